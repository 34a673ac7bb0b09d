// Host runtime above the Newton step: the time loop of the paper's flow chart
// (Sec. 3, steps 4-6: fixed controls within a step, cut on Newton failure),
// a batch engine that runs many scenarios at once, and a serving loop with
// admission by device-memory footprint.
//
// Concurrency model: every scenario owns a pf_sim (its own device arena,
// stream and CUDA graphs); host worker threads drive different scenarios at
// the same time, so their kernels and graphs overlap on the GPU.  Kernels are
// deterministic and a scenario's arithmetic never depends on which stream or
// thread runs it, so a scenario's result is identical alone and in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "polyflood.h"
#include "pf_internal.cuh"

namespace {

thread_local std::string g_rt_error;

pf_status rt_fail(pf_status st, const std::string& m) {
  g_rt_error = m;
  return st;
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Deep copy of a model description and its schedule (the server keeps
// requests after the caller's buffers are gone).
struct OwnedModel {
  pf_model_desc desc{};
  std::vector<double> kx, ky, kz, phi, p0, s0, c0, sat, poly;
  std::vector<std::vector<int64_t>> cells;
  std::vector<std::vector<int>> dirs;
  std::vector<pf_well_desc> wells;
  std::vector<std::vector<pf_well_control>> controls;
  std::vector<pf_period> periods;
  pf_schedule sched{};

  OwnedModel(const pf_model_desc& m, const pf_schedule& s) {
    const size_t n = (size_t)m.nx * m.ny * m.nz;
    auto cp = [n](const double* a) { return std::vector<double>(a, a + n); };
    kx = cp(m.kx); ky = cp(m.ky); kz = cp(m.kz); phi = cp(m.phi); p0 = cp(m.p0); s0 = cp(m.s0); c0 = cp(m.c0);
    desc = m;
    desc.kx = kx.data(); desc.ky = ky.data(); desc.kz = kz.data(); desc.phi = phi.data();
    desc.p0 = p0.data(); desc.s0 = s0.data(); desc.c0 = c0.data();
    wells.assign(m.wells, m.wells + m.n_wells);
    cells.resize(m.n_wells);
    dirs.resize(m.n_wells);
    for (int w = 0; w < m.n_wells; ++w) {
      cells[w].assign(m.wells[w].cells, m.wells[w].cells + m.wells[w].n_perf);
      wells[w].cells = cells[w].data();
      if (m.wells[w].dirs) {
        dirs[w].assign(m.wells[w].dirs, m.wells[w].dirs + m.wells[w].n_perf);
        wells[w].dirs = dirs[w].data();
      }
    }
    desc.wells = wells.empty() ? nullptr : wells.data();
    if (m.n_sat > 0 && m.sat_table) {
      sat.assign(m.sat_table, m.sat_table + 4 * (size_t)m.n_sat);
      desc.sat_table = sat.data();
    }
    if (m.n_poly > 0 && m.poly_table) {
      poly.assign(m.poly_table, m.poly_table + 3 * (size_t)m.n_poly);
      desc.poly_table = poly.data();
    }
    controls.resize(s.n_periods);
    periods.resize(s.n_periods);
    for (int p = 0; p < s.n_periods; ++p) {
      controls[p].assign(s.periods[p].controls, s.periods[p].controls + m.n_wells);
      periods[p] = s.periods[p];
      periods[p].controls = controls[p].empty() ? nullptr : controls[p].data();
    }
    sched.n_periods = s.n_periods;
    sched.periods = periods.empty() ? nullptr : periods.data();
  }
};

bool valid_schedule(const pf_schedule* s, int nw) {
  if (!s || s->n_periods < 0 || (s->n_periods > 0 && !s->periods)) return false;
  for (int p = 0; p < s->n_periods; ++p) {
    const pf_period& q = s->periods[p];
    if (q.n_steps < 0 || !(q.dt > 0.0) || (nw > 0 && !q.controls)) return false;
  }
  return true;
}

}  // namespace

extern "C" {

const char* pf_runtime_last_error(void) { return g_rt_error.c_str(); }

pf_status pf_run_schedule(pf_sim* s, const pf_schedule* sched, int max_cuts, pf_run_report* rep) {
  if (!s) return rt_fail(PF_EINVAL, "pf_sim is NULL");
  int64_t nc = 0, np = 0;
  int nw = 0;
  pf_sizes(s, &nc, &nw, &np);
  if (!valid_schedule(sched, nw)) return rt_fail(PF_EINVAL, "invalid schedule");
  pf_run_report out{};
  const double t0 = now_s();
  pf_status rc = PF_OK;
  for (int p = 0; p < sched->n_periods && rc == PF_OK; ++p) {
    const pf_period& per = sched->periods[p];
    if ((rc = pf_set_controls(s, per.controls, nw)) != PF_OK) {
      rt_fail(rc, pf_last_error());
      break;
    }
    for (int k = 0; k < per.n_steps && rc == PF_OK; ++k) {
      double left = per.dt, dt = per.dt;
      int cuts = 0;
      while (left > 0.0) {
        dt = std::min(dt, left);
        pf_step_report sr{};
        pf_status r = pf_step(s, dt, &sr);
        out.newton_iters += sr.newton_iters;
        out.krylov_iters += sr.krylov_iters;
        if (r == PF_OK) {
          left -= dt;
          dt = std::min(2.0 * dt, per.dt);  // grow back after a cut (Sec. 3 step 4(c)-(d))
        } else if (r == PF_ENOT_CONVERGED && cuts < max_cuts) {
          ++cuts;
          ++out.cuts;
          dt *= 0.5;  // Sec. 3 step 4(a): cut the time step
        } else {
          rc = r;
          rt_fail(r, r == PF_ENOT_CONVERGED ? "time step cut limit reached" : pf_last_error());
          break;
        }
      }
      if (rc == PF_OK) ++out.steps;
    }
  }
  out.status = rc;
  out.seconds = now_s() - t0;
  if (rep) *rep = out;
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batch engine
// ---------------------------------------------------------------------------

// Packed assembly for a batch.  A member that reaches an assembly records an
// event on its stream and queues itself; the first one to find no pack in
// flight becomes the packer: it waits (up to the window) until every member
// inside pf_batch_run is queued, takes the queue, orders the packer stream
// after the queued members' events, launches the packed kernels and records
// one event that each member's stream then waits on.  Members that arrive
// while a pack is in flight are taken by the next packer (one of them).
namespace {

struct EventRef {
  cudaEvent_t e = nullptr;
  ~EventRef() {
    if (e) cudaEventDestroy(e);  // released once its stream work completes
  }
};

struct AsmPacker {
  struct Req {
    pf_sim* s = nullptr;
    cudaEvent_t ready = nullptr;
    std::shared_ptr<EventRef> done;
    pf_status rc = PF_OK;
    bool served = false;
  };
  cudaStream_t st = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::vector<Req*> waiting;
  bool busy = false;
  int running = 0;  // members inside pf_batch_run
  std::chrono::microseconds window{0};
  std::map<pf_sim*, cudaEvent_t> ready;
  int64_t packs = 0, members = 0;
};

pf_status packer_assemble(void* ctx, pf_sim* s) {
  AsmPacker* P = static_cast<AsmPacker*>(ctx);
  AsmPacker::Req r;
  r.s = s;
  const cudaStream_t ms = pf::sim_stream(s);
  std::unique_lock<std::mutex> lk(P->mu);
  r.ready = P->ready.at(s);
  if (cudaEventRecord(r.ready, ms) != cudaSuccess) return rt_fail(PF_ECUDA, "packed assembly: event record");
  P->waiting.push_back(&r);
  P->cv.notify_all();
  while (!r.served) {
    if (P->busy) {
      P->cv.wait(lk);
      continue;
    }
    P->busy = true;
    P->cv.wait_until(lk, std::chrono::steady_clock::now() + P->window,
                     [&] { return (int)P->waiting.size() >= P->running; });
    std::vector<AsmPacker::Req*> pack;
    pack.swap(P->waiting);
    lk.unlock();
    pf_status rc = PF_OK;
    std::vector<pf_sim*> sims;
    for (AsmPacker::Req* q : pack) {
      sims.push_back(q->s);
      if (cudaStreamWaitEvent(P->st, q->ready, 0) != cudaSuccess) rc = PF_ECUDA;
    }
    if (rc == PF_OK) rc = pf::assemble_packed(sims.data(), (int)sims.size(), P->st, nullptr);
    auto ev = std::make_shared<EventRef>();
    if (rc == PF_OK && (cudaEventCreateWithFlags(&ev->e, cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventRecord(ev->e, P->st) != cudaSuccess))
      rc = PF_ECUDA;
    lk.lock();
    for (AsmPacker::Req* q : pack) {
      q->done = ev;
      q->rc = rc;
      q->served = true;
    }
    P->packs += 1;
    P->members += (int64_t)pack.size();
    P->busy = false;
    P->cv.notify_all();
  }
  std::shared_ptr<EventRef> done = std::move(r.done);
  const pf_status rc = r.rc;
  lk.unlock();
  if (rc != PF_OK) return rt_fail(rc, "packed assembly failed");
  if (cudaStreamWaitEvent(ms, done->e, 0) != cudaSuccess) return rt_fail(PF_ECUDA, "packed assembly: stream wait");
  return PF_OK;
}

}  // namespace

struct pf_batch {
  int device = 0;
  int n_threads = 1;
  std::vector<pf_sim*> sims;
  std::vector<cudaStream_t> streams;
  AsmPacker* packer = nullptr;
};

namespace {

void packing_off(pf_batch* b) {
  AsmPacker* P = b->packer;
  if (!P) return;
  for (pf_sim* s : b->sims) pf::set_assembly_packer(s, nullptr, nullptr);
  if (P->st) cudaStreamSynchronize(P->st);
  for (auto& kv : P->ready)
    if (kv.second) cudaEventDestroy(kv.second);
  if (P->st) cudaStreamDestroy(P->st);
  delete P;
  b->packer = nullptr;
}

}  // namespace

extern "C" {

pf_status pf_batch_destroy(pf_batch* b) {
  if (!b) return PF_OK;
  cudaSetDevice(b->device);
  packing_off(b);
  for (pf_sim* s : b->sims) pf_destroy(s);
  for (cudaStream_t st : b->streams) if (st) cudaStreamDestroy(st);
  delete b;
  return PF_OK;
}

pf_status pf_batch_create(const pf_model_desc* const* models, int n, const pf_solver_opts* o, int n_threads,
                          pf_batch** out) {
  if (!out || !models || n < 1 || n_threads < 1) return rt_fail(PF_EINVAL, "invalid batch arguments");
  *out = nullptr;
  // the members overlap on the GPU, so an Arnoldi step run ahead of the host's
  // check would only take time from the others (measured: 64 members, mixed
  // precision, 147.0M with the lookahead off against 143.3M on)
  pf_solver_opts mo;
  if (o) mo = *o;
  else pf_default_opts(&mo);
  mo.krylov_lookahead = 0;
  pf_batch* b = new pf_batch();
  cudaGetDevice(&b->device);
  b->n_threads = n_threads;
  for (int i = 0; i < n; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      pf_batch_destroy(b);
      return rt_fail(PF_ECUDA, "stream creation failed");
    }
    b->streams.push_back(st);
    pf_sim* s = nullptr;
    pf_status rc = pf_create(models[i], &mo, st, &s);
    if (rc != PF_OK) {
      std::string msg = std::string("member ") + std::to_string(i) + ": " + pf_last_error();
      pf_batch_destroy(b);
      return rt_fail(rc, msg);
    }
    b->sims.push_back(s);
  }
  *out = b;
  return PF_OK;
}

pf_status pf_batch_member(pf_batch* b, int i, pf_sim** out) {
  if (!b || !out || i < 0 || i >= (int)b->sims.size()) return rt_fail(PF_EINVAL, "invalid member");
  *out = b->sims[i];
  return PF_OK;
}

pf_status pf_batch_run(pf_batch* b, const pf_schedule* const* schedules, int max_cuts, pf_run_report* reports) {
  if (!b || !schedules) return rt_fail(PF_EINVAL, "invalid batch run arguments");
  const int n = (int)b->sims.size();
  std::atomic<int> next{0};
  std::vector<pf_run_report> rep(n);
  AsmPacker* P = b->packer;
  auto worker = [&]() {
    cudaSetDevice(b->device);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      if (P) {
        std::lock_guard<std::mutex> lk(P->mu);
        P->running += 1;
      }
      pf_run_schedule(b->sims[i], schedules[i], max_cuts, &rep[i]);
      if (P) {
        std::lock_guard<std::mutex> lk(P->mu);
        P->running -= 1;
        P->cv.notify_all();  // a packer waiting for this member stops waiting
      }
    }
  };
  std::vector<std::thread> th;
  const int nt = std::min(b->n_threads, n);
  for (int t = 0; t < nt; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  pf_status rc = PF_OK;
  for (int i = 0; i < n; ++i) {
    if (reports) reports[i] = rep[i];
    if (rep[i].status != PF_OK && rc == PF_OK) rc = rep[i].status;
  }
  if (rc != PF_OK) g_rt_error = "at least one member failed (see its report status)";
  return rc;
}

pf_status pf_batch_set_packing(pf_batch* b, int on, double window_us) {
  if (!b || !(window_us >= 0.0)) return rt_fail(PF_EINVAL, "invalid packing arguments");
  cudaSetDevice(b->device);
  packing_off(b);
  if (!on) return PF_OK;
  AsmPacker* P = new AsmPacker();
  b->packer = P;
  P->window = std::chrono::microseconds((long long)window_us);
  if (cudaStreamCreateWithFlags(&P->st, cudaStreamNonBlocking) != cudaSuccess) {
    packing_off(b);
    return rt_fail(PF_ECUDA, "packing: stream creation failed");
  }
  for (pf_sim* s : b->sims) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      packing_off(b);
      return rt_fail(PF_ECUDA, "packing: event creation failed");
    }
    P->ready[s] = e;
  }
  for (pf_sim* s : b->sims) pf::set_assembly_packer(s, packer_assemble, P);
  return PF_OK;
}

pf_status pf_batch_packing_stats(pf_batch* b, int64_t* packs, int64_t* members) {
  if (!b) return rt_fail(PF_EINVAL, "batch is NULL");
  int64_t p = 0, m = 0;
  if (b->packer) {
    std::lock_guard<std::mutex> lk(b->packer->mu);
    p = b->packer->packs;
    m = b->packer->members;
  }
  if (packs) *packs = p;
  if (members) *members = m;
  return PF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// serving loop
// ---------------------------------------------------------------------------

struct Request {
  uint64_t ticket = 0;
  std::unique_ptr<OwnedModel> model;
  size_t footprint = 0;
  int state = PF_REQ_QUEUED;
  pf_status status = PF_OK;
  pf_run_report report{};
  double t_submit = 0.0, t_start = 0.0, t_end = 0.0;
  std::vector<double> P, S, C, Pb;
  int64_t n = 0;
  int nw = 0;
};

struct pf_server {
  int device = 0;
  size_t budget = 0, in_use = 0;
  pf_solver_opts opts{};
  int max_cuts = 6;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  int running = 0;
  std::vector<std::thread> workers;
};

static void serve_one(pf_server* srv, Request* r) {
  cudaStream_t st = nullptr;
  pf_sim* s = nullptr;
  pf_status rc = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess ? PF_OK : PF_ECUDA;
  if (rc == PF_OK) rc = pf_create(&r->model->desc, &srv->opts, st, &s);
  pf_run_report rep{};
  if (rc == PF_OK) rc = pf_run_schedule(s, &r->model->sched, srv->max_cuts, &rep);
  if (s) {
    r->P.resize(r->n); r->S.resize(r->n); r->C.resize(r->n); r->Pb.resize(std::max(1, r->nw));
    if (pf_get_state(s, r->P.data(), r->S.data(), r->C.data(), r->Pb.data()) != PF_OK && rc == PF_OK) rc = PF_ECUDA;
    pf_destroy(s);
  }
  if (st) cudaStreamDestroy(st);
  r->report = rep;
  r->status = rc;
}

static void server_worker(pf_server* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  for (;;) {
    Request* pick = nullptr;
    srv->cv.wait(lk, [&] {
      if (srv->stop) return true;
      // first queued request (arrival order) whose footprint fits the free budget
      for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it) {
        Request* r = srv->reqs[*it].get();
        if (srv->in_use + r->footprint <= srv->budget) {
          pick = r;
          srv->queue.erase(it);
          return true;
        }
      }
      return false;
    });
    if (!pick) return;  // stop requested and nothing picked
    srv->in_use += pick->footprint;
    pick->state = PF_REQ_RUNNING;
    pick->t_start = now_s();
    srv->running++;
    lk.unlock();
    serve_one(srv, pick);
    lk.lock();
    pick->t_end = now_s();
    pick->state = pick->status == PF_OK ? PF_REQ_DONE : PF_REQ_FAILED;
    pick->model.reset();  // host copy of the inputs is no longer needed
    srv->in_use -= pick->footprint;
    srv->running--;
    srv->cv.notify_all();
    srv->done_cv.notify_all();
  }
}

extern "C" {

pf_status pf_server_create(size_t hbm_budget, int n_workers, const pf_solver_opts* o, int max_cuts,
                           pf_server** out) {
  if (!out || hbm_budget == 0 || n_workers < 1 || max_cuts < 0) return rt_fail(PF_EINVAL, "invalid server arguments");
  pf_server* srv = new pf_server();
  cudaGetDevice(&srv->device);
  srv->budget = hbm_budget;
  srv->max_cuts = max_cuts;
  if (o) srv->opts = *o;
  else pf_default_opts(&srv->opts);
  srv->opts.krylov_lookahead = 0;  // requests overlap on the GPU, as in pf_batch
  for (int i = 0; i < n_workers; ++i) srv->workers.emplace_back(server_worker, srv);
  *out = srv;
  return PF_OK;
}

pf_status pf_server_submit(pf_server* srv, const pf_model_desc* m, const pf_schedule* sched, uint64_t* ticket) {
  if (!srv || !m || !ticket) return rt_fail(PF_EINVAL, "invalid submit arguments");
  if (!valid_schedule(sched, m->n_wells)) return rt_fail(PF_EINVAL, "invalid schedule");
  size_t fp = 0;
  pf_status rc = pf_footprint(m, &srv->opts, &fp);
  if (rc != PF_OK) return rt_fail(rc, pf_last_error());
  if (fp > srv->budget)
    return rt_fail(PF_EBUSY, "request needs " + std::to_string(fp) + " bytes, more than the server budget of " +
                                 std::to_string(srv->budget));
  auto r = std::make_unique<Request>();
  r->model = std::make_unique<OwnedModel>(*m, *sched);
  r->footprint = fp;
  r->n = (int64_t)m->nx * m->ny * m->nz;
  r->nw = m->n_wells;
  std::lock_guard<std::mutex> lk(srv->mu);
  r->ticket = srv->next_ticket++;
  r->t_submit = now_s();
  *ticket = r->ticket;
  srv->queue.push_back(r->ticket);
  srv->reqs[r->ticket] = std::move(r);
  srv->cv.notify_all();
  return PF_OK;
}

static void fill_result(const Request* r, pf_result* out) {
  out->state = r->state;
  out->status = r->status;
  out->report = r->report;
  out->t_submit = r->t_submit;
  out->t_start = r->t_start;
  out->t_end = r->t_end;
  out->footprint = r->footprint;
}

pf_status pf_server_poll(pf_server* srv, uint64_t ticket, pf_result* out) {
  if (!srv || !out) return rt_fail(PF_EINVAL, "invalid poll arguments");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return rt_fail(PF_EINVAL, "unknown ticket");
  fill_result(it->second.get(), out);
  return PF_OK;
}

pf_status pf_server_wait(pf_server* srv, uint64_t ticket, double timeout_s, pf_result* out) {
  if (!srv) return rt_fail(PF_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return rt_fail(PF_EINVAL, "unknown ticket");
  Request* r = it->second.get();
  const bool ok = srv->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [&] { return r->state == PF_REQ_DONE || r->state == PF_REQ_FAILED; });
  if (out) fill_result(r, out);
  return ok ? PF_OK : rt_fail(PF_ETIMEOUT, "request not finished within the timeout");
}

pf_status pf_server_fetch_state(pf_server* srv, uint64_t ticket, double* P, double* S, double* C, double* Pb) {
  if (!srv) return rt_fail(PF_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return rt_fail(PF_EINVAL, "unknown ticket");
  const Request* r = it->second.get();
  if (r->state != PF_REQ_DONE) return rt_fail(PF_EINVAL, "request is not done");
  if (P) std::copy(r->P.begin(), r->P.end(), P);
  if (S) std::copy(r->S.begin(), r->S.end(), S);
  if (C) std::copy(r->C.begin(), r->C.end(), C);
  if (Pb) std::copy(r->Pb.begin(), r->Pb.begin() + r->nw, Pb);
  return PF_OK;
}

pf_status pf_server_stats(pf_server* srv, size_t* in_use, int* running, int* queued) {
  if (!srv) return rt_fail(PF_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(srv->mu);
  if (in_use) *in_use = srv->in_use;
  if (running) *running = srv->running;
  if (queued) *queued = (int)srv->queue.size();
  return PF_OK;
}

pf_status pf_server_destroy(pf_server* srv) {
  if (!srv) return PF_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->queue.clear();
  }
  srv->cv.notify_all();
  for (auto& t : srv->workers) t.join();
  delete srv;
  return PF_OK;
}

}  // extern "C"
