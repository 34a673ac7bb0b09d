// C ABI of the polyflood library: model set-up, device arena, Newton driver
// (Alg. 1 with the forcing term of Sec. 3.3) and the restarted flexible GMRES
// with a right preconditioner (block-Jacobi or CPR, Alg. 2).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "pf_cpr.cuh"
#include "pf_internal.cuh"

using namespace pf;

static thread_local std::string g_last_error;

static pf_status fail(pf_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

static std::atomic<bool> g_pdl{false};

// Host-side fault injection (pf_inject_create_failure): the k-th guarded CUDA
// call of the next pf_create reports an error instead of running.
static std::atomic<int> g_inject_k{0};

static bool inject_hit(int* site) {
  ++*site;
  int k = g_inject_k.load(std::memory_order_relaxed);
  return k > 0 && *site == k && g_inject_k.compare_exchange_strong(k, 0);
}

namespace pf {
void set_last_error(const std::string& msg) { g_last_error = msg; }
bool pdl_enabled() { return g_pdl.load(std::memory_order_relaxed); }
}  // namespace pf

#define PF_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      if (s) s->dead = true;                                                                \
      return fail(PF_ECUDA, std::string("CUDA error in ") + #call + ": " + cudaGetErrorString(e_)); \
    }                                                                                       \
  } while (0)

#define PF_LAUNCHED(k)                                                                      \
  do {                                                                                      \
    s->launches += (k);                                                                     \
    cudaError_t e_ = cudaGetLastError();                                                    \
    if (e_ != cudaSuccess) {                                                                \
      s->dead = true;                                                                       \
      return fail(PF_ECUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e_)); \
    }                                                                                       \
  } while (0)

struct pf_sim {
  cudaStream_t stream = nullptr;
  // assembly through a packer (several simulators per launch, set by the
  // batch engine); null: this simulator's own launches
  pf_status (*packer)(void*, pf_sim*) = nullptr;
  void* packer_ctx = nullptr;
  int device = 0;
  bool dead = false;
  bool mixed = false;
  pf_solver_opts opts;
  Grid g;
  Phys ph;
  int nw = 0;
  long long npf = 0;
  long long nunk = 0, ld = 0;
  int nblocks = 0;
  int64_t launches = 0;
  // host copies
  std::vector<int> h_kind, h_ptr;
  std::vector<long long> h_cell;
  std::vector<double> h_W;
  std::vector<pf_well_control> h_ctl;   // user controls
  std::vector<char> switched;           // rate well running on its BHP limit
  bool have_controls = false;
  // arena
  char* arena = nullptr;
  size_t arena_bytes = 0;
  // device arrays
  double *wL3 = nullptr, *inv_pv = nullptr;
  double *phi_r = nullptr, *T3 = nullptr, *x = nullptr, *x_old = nullptr, *Mold = nullptr, *R = nullptr;
  double *pv = nullptr, *Fbuf = nullptr, *dx = nullptr, *b = nullptr, *r = nullptr, *tmp = nullptr;
  void *pd = nullptr, *J = nullptr, *Bw = nullptr, *Cw = nullptr, *Dw = nullptr;
  void *Dinv = nullptr, *Dwinv = nullptr;
  int *w_ptr = nullptr, *w_kind = nullptr, *w_ctrl = nullptr;
  long long* w_cell = nullptr;
  double *w_wi = nullptr, *w_dzb = nullptr, *w_target = nullptr, *w_cinj = nullptr, *w_W = nullptr;
  double *w_sw = nullptr, *w_so = nullptr, *w_scale = nullptr, *w_gamma = nullptr;
  float* Zf = nullptr;  // mixed precision: FP32 copies of the preconditioned vectors
  float* Vf = nullptr;  // mixed precision: FP32 copy of the Krylov vector the preconditioner takes next
  double *V = nullptr, *Z = nullptr, *hbuf = nullptr, *partial = nullptr, *norms = nullptr, *ydev = nullptr;
  double* vs = nullptr;  // [128] the Krylov basis vector j is vs[j] V_j (V_j is kept before normalisation)
  double* wtot = nullptr;  // [3 nw] well totals
  unsigned int* red_counter = nullptr;  // last-block reduction counter (zeroed)
  double* h_pinned = nullptr;
  CprData cpr;
  Tuning tune;  // block sizes of the per-cell kernels
  // opt-in CUDA-event timing of selected kernels
  bool kt_on = false;
  std::vector<cudaEvent_t> kt_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> kt_pending;
  int64_t kt_count[PF_KT_COUNT] = {0};
  double kt_ms[PF_KT_COUNT] = {0.0};
  int switch_attempt = 0;
  // CUDA graphs of the Krylov iteration, per Arnoldi index j: preconditioner,
  // SpMV, orthogonalisation (captured once, replayed every iteration)
  cudaStream_t cap_stream = nullptr;
  bool capturing = false;
  bool use_graphs = true;
  struct IterGraphs {
    cudaGraphExec_t pre = nullptr, spmv = nullptr, ortho = nullptr;
    int k_pre = 0, k_spmv = 0, k_ortho = 0;
  };
  std::vector<IterGraphs> graphs;
  // completion of the Arnoldi steps in flight, by the parity of j (at most two:
  // step j and the step enqueued ahead of it)
  cudaEvent_t step_done[2] = {nullptr, nullptr};
  double krylov_rate = 0.5;  // mean residual reduction per Arnoldi step of the last solve
  // step state
  double dt = 0.0;
  bool in_step = false;
  bool assembled = false;
  double prev_norm = -1.0;      // |b^{l-1}| of the previous Newton iteration (< 0: none)
  double prev_lin_norm = 0.0;   // |r^{l-1}| (forcing form 2)
  double* rlin = nullptr;       // r^{l-1} (forcing form 1)
  int* w_perf_of = nullptr;     // [N] perforation of each cell, -1 if none
  int* w_pwell = nullptr;       // [npf] well of each perforation
  double* d_sat = nullptr;      // saturation table (structure of arrays with slopes)
  double* d_poly = nullptr;     // polymer table
  int iter_in_step = 0;
  double res0 = 0.0;            // scaled residual at the first iteration of the step
};

namespace {

cudaEvent_t kt_event(pf_sim* s) {
  if (!s->kt_pool.empty()) {
    cudaEvent_t e = s->kt_pool.back();
    s->kt_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one launch of kernel class `which` with events on the sim's stream.
// Pinned host buffer: [0, 8) norms read by the host right away; two slots of
// one Arnoldi step's Hessenberg data (h1, h2, |w|^2 and 1/|w|, second-pass
// flag), by the parity of j, so the step enqueued ahead never overwrites the
// one the host is reading; then the least-squares solution y of a cycle.
constexpr int kPinStep = 8, kPinStepStride = 392, kPinY = kPinStep + 2 * kPinStepStride, kPinTotal = kPinY + 128;

struct KtScope {
  pf_sim* s;
  int which;
  cudaEvent_t a = nullptr, b = nullptr;
  KtScope(pf_sim* s_, int w) : s(s_), which(w) {
    if (s->kt_on && !s->capturing) {
      a = kt_event(s);
      b = kt_event(s);
      cudaEventRecord(a, s->stream);
    }
  }
  ~KtScope() {
    if (a) {
      cudaEventRecord(b, s->stream);
      s->kt_pending.push_back({which, {a, b}});
    }
  }
};

void kt_collect(pf_sim* s) {
  if (s->kt_pending.empty()) return;
  cudaStreamSynchronize(s->stream);
  for (auto& p : s->kt_pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    s->kt_count[p.first] += 1;
    s->kt_ms[p.first] += ms;
    s->kt_pool.push_back(p.second.first);
    s->kt_pool.push_back(p.second.second);
  }
  s->kt_pending.clear();
}

Wells wells_view(const pf_sim* s) {
  Wells w;
  w.nw = s->nw;
  w.npf = s->npf;
  w.ptr = s->w_ptr;
  w.cell = s->w_cell;
  w.wi = s->w_wi;
  w.dzb = s->w_dzb;
  w.kind = s->w_kind;
  w.ctrl = s->w_ctrl;
  w.target = s->w_target;
  w.cinj = s->w_cinj;
  w.W = s->w_W;
  w.sw = s->w_sw;
  w.so = s->w_so;
  w.scale = s->w_scale;
  w.gamma = s->w_gamma;
  w.perf_of = s->w_perf_of;
  w.pwell = s->w_pwell;
  return w;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Peaceman well index of Sec. 2.4 with its equivalent radius and permeability;
// the printed form is for a well along x, whose perpendicular directions are y
// and z.
double well_index(double kx, double ky, double kz, double dx, double dy, double dz, int dir, double rw, double skin,
                  double gf, double f, double fh) {
  double k1, k2, h1, h2, h;
  if (dir == PF_DIR_X) { k1 = ky; k2 = kz; h1 = dy; h2 = dz; h = dx; }
  else if (dir == PF_DIR_Y) { k1 = kx; k2 = kz; h1 = dx; h2 = dz; h = dy; }
  else { k1 = kx; k2 = ky; h1 = dx; h2 = dy; h = dz; }
  const double r21 = k2 / k1, r12 = k1 / k2;
  const double re = 2.0 * gf / sqrt(M_PI) * sqrt(sqrt(r21) * h1 * h1 + sqrt(r12) * h2 * h2) /
                    (pow(r21, 0.25) + pow(r12, 0.25));
  const double ka = sqrt(k1 * k2);
  return 2.0 * M_PI * f * h * fh * ka / (log(re / rw) + skin);
}

Phys derive_phys(const pf_physics& p) {
  Phys ph;
  ph.rho_w = p.rho_w; ph.rho_o = p.rho_o; ph.c_w = p.c_w; ph.c_o = p.c_o; ph.p_ref = p.p_ref;
  ph.mu_w = p.mu_w; ph.mu_o = p.mu_o; ph.c_r = p.c_r; ph.p_r = p.p_r;
  ph.swc = p.swc; ph.sor = p.sor; ph.nw = p.nw; ph.no = p.no; ph.krw_max = p.krw_max; ph.kro_max = p.kro_max;
  ph.pc_e = p.pc_e; ph.pc_n = p.pc_n; ph.ads_a = p.ads_a; ph.ads_b = p.ads_b; ph.rrf = p.rrf; ph.ipv = p.ipv;
  ph.omega = p.omega; ph.mu_p0 = p.mu_p0; ph.c_ref = p.c_ref; ph.g = p.g; ph.mixing = p.mixing;
  ph.inv_den = 1.0 / (1.0 - p.swc - p.sor);
  ph.ln_mu_w = log(p.mu_w);
  ph.ln_mu_ratio = log(p.mu_p0) - log(p.mu_w);
  const double ads_max = p.ads_b > 0.0 ? p.ads_a / p.ads_b : 0.0;
  ph.rk_coef = ads_max > 0.0 ? (p.rrf - 1.0) / ads_max : 0.0;
  ph.mu_p0_pow = pow(p.mu_p0, 1.0 - p.omega);
  ph.mu_w_pow = pow(p.mu_w, 1.0 - p.omega);
  ph.inv_c_ref = 1.0 / p.c_ref;
  ph.inv_rho_w = 1.0 / p.rho_w;
  ph.inv_mu_o = 1.0 / p.mu_o;
  return ph;
}

// Table sizes and, with a polymer table, A_d,max = the largest tabulated A_d
// (the device pointers are set once the arena exists).
void set_tables(Phys& ph, const pf_model_desc& m) {
  ph.n_sat = m.n_sat;
  ph.n_poly = m.n_poly;
  if (m.n_poly > 0) {
    double amax = 0.0;
    for (int k = 0; k < m.n_poly; ++k) amax = std::max(amax, m.poly_table[3 * k + 2]);
    ph.rk_coef = amax > 0.0 ? (m.phys.rrf - 1.0) / amax : 0.0;
  }
}

// Structure-of-arrays copy of a table with its segment slopes: `cols` value
// columns after the abscissa; out = [x, y_1..y_cols, slope_1..slope_cols],
// each K long (the last slope, beyond the table, is 0).
std::vector<double> table_soa(const double* rows, int K, int cols) {
  const int w = cols + 1;
  std::vector<double> out((size_t)(2 * cols + 1) * K, 0.0);
  for (int k = 0; k < K; ++k)
    for (int c = 0; c <= cols; ++c) out[(size_t)c * K + k] = rows[w * k + c];
  for (int k = 0; k + 1 < K; ++k)
    for (int c = 1; c <= cols; ++c)
      out[(size_t)(cols + c) * K + k] = (rows[w * (k + 1) + c] - rows[w * k + c]) / (rows[w * (k + 1)] - rows[w * k]);
  return out;
}

pf_status validate(const pf_model_desc* m, const pf_solver_opts* o) {
  if (!m) return fail(PF_EINVAL, "model description is NULL");
  if (m->nx < 1 || m->ny < 1 || m->nz < 1) return fail(PF_EINVAL, "grid dimensions must be >= 1");
  const long long n = (long long)m->nx * m->ny * m->nz;
  if (n > (1LL << 31) / 4) return fail(PF_EINVAL, "grid too large (more than 2^29 cells)");
  if (!finite_pos(m->dx) || !finite_pos(m->dy) || !finite_pos(m->dz) || !std::isfinite(m->top))
    return fail(PF_EINVAL, "cell sizes must be finite and positive");
  if (!m->kx || !m->ky || !m->kz || !m->phi || !m->p0 || !m->s0 || !m->c0)
    return fail(PF_EINVAL, "per-cell host arrays must not be NULL");
  for (long long i = 0; i < n; ++i) {
    if (!finite_pos(m->kx[i]) || !finite_pos(m->ky[i]) || !finite_pos(m->kz[i]))
      return fail(PF_EINVAL, "permeability must be finite and positive at cell " + std::to_string(i));
    if (!finite_pos(m->phi[i]) || m->phi[i] > 1.0) return fail(PF_EINVAL, "porosity must lie in (0, 1]");
    if (!std::isfinite(m->p0[i]) || !std::isfinite(m->s0[i]) || !std::isfinite(m->c0[i]))
      return fail(PF_EINVAL, "initial state must be finite");
  }
  const pf_physics& p = m->phys;
  if (!finite_pos(p.rho_w) || !finite_pos(p.rho_o) || !finite_pos(p.mu_w) || !finite_pos(p.mu_o) ||
      !finite_pos(p.mu_p0) || !finite_pos(p.c_ref) || !(1.0 - p.swc - p.sor > 0.0) || !std::isfinite(p.g))
    return fail(PF_EINVAL, "invalid fluid or polymer constants");
  if (p.ads_a < 0.0 || p.ads_b < 0.0 || p.ipv < 0.0 || p.ipv >= 1.0 || p.rrf < 1.0 || p.nw < 1.0 || p.no < 1.0)
    return fail(PF_EINVAL, "invalid adsorption, IPV, RRF or Corey exponent");
  if (m->n_sat < 0 || m->n_sat > PF_MAX_KNOTS || (m->n_sat > 0 && !m->sat_table))
    return fail(PF_EINVAL, "invalid saturation table size");
  for (int k = 0; k < m->n_sat; ++k) {
    const double* r = m->sat_table + 4 * k;
    if (!std::isfinite(r[0]) || !std::isfinite(r[1]) || !std::isfinite(r[2]) || !std::isfinite(r[3]) || r[0] < 0.0 ||
        r[0] > 1.0 || r[1] < 0.0 || r[2] < 0.0 || (k > 0 && !(r[0] > r[-4])))
      return fail(PF_EINVAL, "saturation table row " + std::to_string(k) + " is invalid");
  }
  if (m->n_poly < 0 || m->n_poly > PF_MAX_KNOTS || (m->n_poly > 0 && !m->poly_table))
    return fail(PF_EINVAL, "invalid polymer table size");
  for (int k = 0; k < m->n_poly; ++k) {
    const double* r = m->poly_table + 3 * k;
    if (!std::isfinite(r[0]) || !std::isfinite(r[1]) || !std::isfinite(r[2]) || r[0] < 0.0 || !(r[1] > 0.0) ||
        r[2] < 0.0 || (k > 0 && !(r[0] > r[-3])))
      return fail(PF_EINVAL, "polymer table row " + std::to_string(k) + " is invalid");
  }
  if (m->n_wells < 0 || (m->n_wells > 0 && !m->wells)) return fail(PF_EINVAL, "invalid well list");
  std::vector<char> seen((size_t)n, 0);
  for (int w = 0; w < m->n_wells; ++w) {
    const pf_well_desc& d = m->wells[w];
    if (d.n_perf < 1 || !d.cells) return fail(PF_EINVAL, "well without perforations");
    if (d.kind != PF_WELL_INJECTOR && d.kind != PF_WELL_PRODUCER) return fail(PF_EINVAL, "invalid well kind");
    if (!finite_pos(d.rw) || !std::isfinite(d.skin) || !finite_pos(d.gf) || !finite_pos(d.f) || !finite_pos(d.fh) ||
        !std::isfinite(d.pb0))
      return fail(PF_EINVAL, "invalid well index parameters");
    for (int q = 0; q < d.n_perf; ++q) {
      const int64_t c = d.cells[q];
      if (c < 0 || c >= n) return fail(PF_EINVAL, "perforation outside the grid");
      if (seen[(size_t)c]) return fail(PF_EINVAL, "a cell carries more than one perforation");
      seen[(size_t)c] = 1;
      if (d.dirs && (d.dirs[q] < 0 || d.dirs[q] > 2)) return fail(PF_EINVAL, "invalid perforation direction");
    }
  }
  if (o) {
    if (o->gmres_restart < 1 || o->gmres_restart > 64) return fail(PF_EINVAL, "gmres_restart must be in [1, 64]");
    if (o->precision != PF_PREC_FP64 && o->precision != PF_PREC_MIXED) return fail(PF_EINVAL, "invalid precision");
    if (o->precond != PF_PC_BJACOBI && o->precond != PF_PC_CPR) return fail(PF_EINVAL, "invalid preconditioner");
    if (o->amg_cycle != 1 && o->amg_cycle != 2) return fail(PF_EINVAL, "amg_cycle must be 1 or 2");
    if (o->amg_pre_sweeps < 0 || o->amg_post_sweeps < 0 || o->amg_coarse_size < 1 || o->amg_coarse_sweeps < -1)
      return fail(PF_EINVAL, "invalid multigrid parameters");
    if (o->forcing_form < 1 || o->forcing_form > 3) return fail(PF_EINVAL, "forcing_form must be 1, 2 or 3");
    if (o->stage1 != PF_S1_BJACOBI && o->stage1 != PF_S1_ILU0) return fail(PF_EINVAL, "invalid stage1");
    if (!(o->reorth_eta >= 0.0 && o->reorth_eta <= 1.0)) return fail(PF_EINVAL, "reorth_eta must lie in [0, 1]");
    if (std::isnan(o->ilu_guard)) return fail(PF_EINVAL, "ilu_guard is NaN");
    if (!(o->newton_div >= 0.0)) return fail(PF_EINVAL, "newton_div must be >= 0");
    if (o->ilu_store < -1 || o->ilu_store > 2 || (o->ilu_store == 2 && o->precision != PF_PREC_MIXED))
      return fail(PF_EINVAL, "ilu_store must be -1, 0, 1, or 2 (BF16, mixed precision only)");
    if (o->krylov_lookahead != 0 && o->krylov_lookahead != 1) return fail(PF_EINVAL, "krylov_lookahead must be 0 or 1");
  }
  return PF_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Carver {
  size_t off = 0;
  char* base = nullptr;
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Whether the preconditioned Krylov vectors are kept in FP32 only (mixed
// precision with CPR, whose output is FP32 values).
bool fp32_basis(const pf_sim* s) { return s->mixed && s->opts.precond == PF_PC_CPR; }

// Lays out every device array in one arena; with base == nullptr only sizes it.
size_t carve(pf_sim* s, char* base) {
  Carver c;
  c.base = base;
  const long long n = s->g.n;
  const size_t dts = s->mixed ? sizeof(float) : sizeof(double);
  const int m = s->opts.gmres_restart;
  s->phi_r = c.take<double>(n);
  s->T3 = c.take<double>(3 * n);
  s->wL3 = c.take<double>(3 * n);
  s->inv_pv = c.take<double>(n);
  s->x = c.take<double>(s->nunk);
  s->x_old = c.take<double>(s->nunk);
  s->Mold = c.take<double>(3 * n);
  s->R = c.take<double>(s->nunk);
  s->pv = c.take<double>((size_t)PV_COUNT * n);
  s->pd = c.take<char>((size_t)PD_COUNT * n * dts);
  s->Fbuf = c.take<double>(9 * (size_t)n);
  s->J = c.take<char>((size_t)SL_COUNT * 9 * n * dts);
  s->Bw = c.take<char>(3 * (size_t)std::max(1LL, s->npf) * dts);
  s->Cw = c.take<char>(3 * (size_t)std::max(1LL, s->npf) * dts);
  s->Dw = c.take<char>((size_t)std::max(1, s->nw) * dts);
  // the ILU(0) block copies' kind: 0 none, 1 J's type, 2 BF16
  int ilu_kind = s->opts.ilu_store;
  if (ilu_kind < 0) ilu_kind = s->g.n >= 1000000 ? (s->mixed ? 2 : 1) : 0;  // automatic: pays off on large grids
  if (s->opts.stage1 != PF_S1_ILU0) ilu_kind = 0;
  // the block inverses by cell; in FP64 with the copies they are kept per
  // colour slot instead (27M cells: preconditioner apply 6.30 -> 6.07 ms; in
  // mixed precision the same layout measured slower in both ILU(0) forms
  // although it moved fewer bytes, so there they stay by cell)
  const bool inv_by_slot = ilu_kind != 0 && !s->mixed;
  s->Dinv = inv_by_slot ? nullptr : c.take<char>(9 * (size_t)n * dts);
  s->Dwinv = c.take<char>((size_t)std::max(1, s->nw) * dts);
  s->w_ptr = c.take<int>(s->nw + 1);
  s->w_kind = c.take<int>(std::max(1, s->nw));
  s->w_ctrl = c.take<int>(std::max(1, s->nw));
  s->w_cell = c.take<long long>(std::max(1LL, s->npf));
  s->w_wi = c.take<double>(std::max(1LL, s->npf));
  s->w_dzb = c.take<double>(std::max(1LL, s->npf));
  s->w_target = c.take<double>(std::max(1, s->nw));
  s->w_cinj = c.take<double>(std::max(1, s->nw));
  s->w_W = c.take<double>(std::max(1, s->nw));
  s->w_sw = c.take<double>(std::max(1, s->nw));
  s->w_so = c.take<double>(std::max(1, s->nw));
  s->w_scale = c.take<double>(std::max(1, s->nw));
  s->w_gamma = c.take<double>(std::max(1, s->nw));
  s->dx = c.take<double>(s->nunk);
  s->b = c.take<double>(s->nunk);
  s->r = c.take<double>(s->nunk);
  s->tmp = c.take<double>(s->nunk);
  s->rlin = (s->opts.use_forcing && s->opts.forcing_form == 1) ? c.take<double>(s->nunk) : nullptr;
  s->V = c.take<double>((size_t)(m + 1) * s->ld);
  // the mixed CPR preconditioner computes z in FP32: its vectors are kept in
  // FP32 only (the FP64 copy would hold the same values)
  s->Z = fp32_basis(s) ? nullptr : c.take<double>((size_t)m * s->ld);
  s->Zf = s->mixed ? c.take<float>((size_t)m * s->ld) : nullptr;
  s->Vf = s->mixed ? c.take<float>((size_t)s->ld) : nullptr;
  s->hbuf = c.take<double>(4 * 128 + 8);
  s->partial = c.take<double>((size_t)s->nblocks * 72);
  s->norms = c.take<double>(4);
  s->ydev = c.take<double>(128);
  s->vs = c.take<double>(128);
  s->wtot = c.take<double>(3 * (size_t)std::max(1, s->nw));
  s->red_counter = c.take<unsigned int>(64);
  {
    // compact ILU block copies: 2 colours x 54 values per colour slot
    const int kind = ilu_kind;
    const size_t es = kind == 2 ? 2 : dts;
    const size_t slots = (size_t)((s->g.nx + 1) / 2) * s->g.ny * s->g.nz;
    s->cpr.ilu_cp.kind = kind;
    // with the copies the black copy holds the set-up's J_bj D_j^-1, which the
    // black sweep reads (below 1M cells, without the copies, an array of them
    // cost more in L2 residency than it saved: 100k cells FP64, preconditioner
    // apply 123.7 -> 130 us)
    // the finest multigrid smoother's per-colour stencil copies follow the same size rule (any first stage)
    s->cpr.rb_copy = s->opts.ilu_store < 0 ? s->g.n >= 1000000 : s->opts.ilu_store != 0;
    for (int q = 0; q < 2; ++q) s->cpr.ilu_cp.c[q] = kind ? (void*)c.take<char>(54 * slots * es) : nullptr;
    // with CPR after ILU(0): the black rows' pressure combination for stage 2
    // (18 values per black slot in the copy's type, or J's without a copy; 3
    // for the diagonal block)
    const bool cpr_p = s->opts.stage1 == PF_S1_ILU0 && s->opts.precond == PF_PC_CPR;
    s->cpr.ilu_cp.p = cpr_p ? (void*)c.take<char>(18 * slots * es) : nullptr;
    s->cpr.ilu_cp.pd = cpr_p ? (void*)c.take<char>(3 * slots * dts) : nullptr;
    // FP64 with the copies: both colours' block inverses per colour slot (red, then black)
    s->cpr.ilu_cp.dr = inv_by_slot ? (void*)c.take<char>(18 * slots * dts) : nullptr;
  }
  s->w_perf_of = c.take<int>(n);
  s->w_pwell = c.take<int>(std::max(1LL, s->npf));
  s->d_sat = s->ph.n_sat > 0 ? c.take<double>((size_t)7 * s->ph.n_sat) : nullptr;
  s->d_poly = s->ph.n_poly > 0 ? c.take<double>((size_t)5 * s->ph.n_poly) : nullptr;
  if (s->opts.precond == PF_PC_CPR) cpr_carve(s->cpr, s->g, s->mixed, c.off, base);
  return align_up(c.off, 256);
}

template <typename DT>
pf_status assemble_t(pf_sim* s) {
  const Wells w = wells_view(s);
  cudaStream_t st = s->stream;
  {
    KtScope t(s, PF_KT_PROPS);
    launch_cell_props<DT>(s->g, s->ph, s->phi_r, s->x, s->pv, (DT*)s->pd, s->Mold, s->R, (DT*)s->J, nullptr, 0, st,
                          s->tune.props);
  }
  {
    KtScope t(s, PF_KT_FACE);
    launch_face_flux<DT>(s->g, s->ph, s->wL3, s->T3, s->x, s->pv, (const DT*)s->pd, s->dt, (DT*)s->J, s->Fbuf, st,
                         s->tune.face);
  }
  {
    KtScope t(s, PF_KT_GATHER);
    launch_gather<DT>(s->g, s->Fbuf, s->R, (DT*)s->J, st, s->tune.gather);
  }
  {
    KtScope t(s, PF_KT_WELLS);
    launch_wells<DT>(s->g, s->ph, w, s->x, s->pv, (const DT*)s->pd, s->dt, s->R, (DT*)s->J, (DT*)s->Bw, (DT*)s->Cw,
                     (DT*)s->Dw, st);
  }
  PF_LAUNCHED(3 + (s->nw > 0));
  return PF_OK;
}

pf_status assemble(pf_sim* s) {
  pf_status rc = s->packer ? s->packer(s->packer_ctx, s) : s->mixed ? assemble_t<float>(s) : assemble_t<double>(s);
  if (rc == PF_OK) s->assembled = true;
  return rc;
}

template <typename DT>
void fill_asm_member(pf_sim* s, AsmMember<DT>& a) {
  a.g = s->g;
  a.ph = s->ph;
  a.w = wells_view(s);
  a.phi_r = s->phi_r;
  a.x = s->x;
  a.Mold = s->Mold;
  a.wL3 = s->wL3;
  a.T3 = s->T3;
  a.pv = s->pv;
  a.R = s->R;
  a.Fbuf = s->Fbuf;
  a.pd = (DT*)s->pd;
  a.J = (DT*)s->J;
  a.Bw = (DT*)s->Bw;
  a.Cw = (DT*)s->Cw;
  a.Dw = (DT*)s->Dw;
  a.dt = s->dt;
}

template <typename DT>
pf_status assemble_packed_t(pf_sim* const* sims, int n, cudaStream_t st, int* launches) {
  AsmPack<DT> pk;
  int kernels = 0;
  for (int done = 0; done < n;) {
    const int k = std::min(kPackMax, n - done);
    pk.nm = k;
    pk.cblock0[0] = 0;
    pk.wblock0[0] = 0;
    for (int q = 0; q < k; ++q) {
      pf_sim* s = sims[done + q];
      fill_asm_member<DT>(s, pk.m[q]);
      pk.cblock0[q + 1] = pk.cblock0[q] + (int)((s->g.n + 255) / 256);
      pk.wblock0[q + 1] = pk.wblock0[q] + s->nw;
    }
    kernels += launch_assemble_packed<DT>(pk, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      for (int q = 0; q < k; ++q) sims[done + q]->dead = true;
      return fail(PF_ECUDA, std::string("packed assembly launch: ") + cudaGetErrorString(e));
    }
    done += k;
  }
  if (launches) *launches = kernels;
  return PF_OK;
}

// y = J x on device vectors
pf_status spmv(pf_sim* s, const double* xin, double* y) {
  const Wells w = wells_view(s);
  KtScope t(s, PF_KT_SPMV);
  if (s->mixed)
    launch_spmv<float>(s->g, w, (const float*)s->J, (const float*)s->Bw, (const float*)s->Cw, (const float*)s->Dw, xin,
                       y, s->stream, s->tune.spmv);
  else
    launch_spmv<double>(s->g, w, (const double*)s->J, (const double*)s->Bw, (const double*)s->Cw,
                        (const double*)s->Dw, xin, y, s->stream, s->tune.spmv);
  PF_LAUNCHED(1);
  return PF_OK;
}

pf_status precond_setup(pf_sim* s) {
  const Wells w = wells_view(s);
  const bool ilu = s->opts.stage1 == PF_S1_ILU0;
  if (s->opts.precond == PF_PC_CPR) cpr_weights(s->cpr, s->ph);  // read by the ILU(0) set-up below
  if (s->mixed) {
    if (ilu)
      launch_ilu_setup<float, float>(s->g, w, (const float*)s->J, (const float*)s->Dw, (float*)s->Dinv,
                                     (float*)s->Dwinv, s->opts.ilu_guard, s->cpr.ilu_cp, s->stream, s->cpr.w_o,
                                     s->cpr.w_w);
    else
      launch_bjacobi_setup<float, float>(s->g, w, (const float*)s->J, (const float*)s->Dw, (float*)s->Dinv,
                                         (float*)s->Dwinv, s->stream);
  } else {
    if (ilu)
      launch_ilu_setup<double, double>(s->g, w, (const double*)s->J, (const double*)s->Dw, (double*)s->Dinv,
                                       (double*)s->Dwinv, s->opts.ilu_guard, s->cpr.ilu_cp, s->stream, s->cpr.w_o,
                                       s->cpr.w_w);
    else
      launch_bjacobi_setup<double, double>(s->g, w, (const double*)s->J, (const double*)s->Dw, (double*)s->Dinv,
                                           (double*)s->Dwinv, s->stream);
  }
  PF_LAUNCHED(1 + (s->nw > 0) + (ilu ? 1 : 0));
  if (s->opts.precond == PF_PC_CPR) {
    int k = 0;
    cpr_setup(s->cpr, s->g, s->ph, s->phi_r, wells_view(s), s->mixed, s->J, s->Bw, s->Dw, s->stream, &k);
    PF_LAUNCHED(k);
  }
  return PF_OK;
}

// z = M^{-1} v (and, in mixed precision, an FP32 copy zf of z when zf != null).
// vf: the FP32 copy of v when the caller has it (the Arnoldi steps: the
// normalisation that wrote v wrote it too); otherwise the mixed CPR form makes
// it first.
pf_status precond_apply(pf_sim* s, const double* v, double* z, float* zf = nullptr, const float* vf = nullptr) {
  if (s->opts.precond == PF_PC_CPR) {
    int k = 0;
    KtScope t(s, PF_KT_PRECOND);
    if (s->mixed && !vf) {
      launch_to_f32(s->nunk, v, s->Vf, s->stream);
      k += 1;
      vf = s->Vf;
    }
    int k2 = 0;
    cpr_apply(s->cpr, s->g, wells_view(s), s->mixed, s->J, s->Bw, s->Cw, s->Dw, s->Dinv, s->Dwinv, v, vf, z, s->tmp,
              zf, s->stream, &k2);
    PF_LAUNCHED(k + k2);
    return PF_OK;
  }
  if (s->opts.stage1 == PF_S1_ILU0) {
    int nl;
    if (s->mixed)
      nl = launch_ilu_apply<float, float, double, double>(s->g, s->nw, (const float*)s->J, (const float*)s->Dinv,
                                                          (const float*)s->Dwinv, v, z, s->tune.ilu_fused,
                                                          s->cpr.ilu_cp, s->stream);
    else
      nl = launch_ilu_apply<double, double, double, double>(s->g, s->nw, (const double*)s->J, (const double*)s->Dinv,
                                                            (const double*)s->Dwinv, v, z, s->tune.ilu_fused,
                                                            s->cpr.ilu_cp, s->stream);
    PF_LAUNCHED(nl);
  } else {
    if (s->mixed)
      launch_bjacobi_apply<float>(s->g, s->nw, (const float*)s->Dinv, (const float*)s->Dwinv, v, z, s->stream);
    else
      launch_bjacobi_apply<double>(s->g, s->nw, (const double*)s->Dinv, (const double*)s->Dwinv, v, z, s->stream);
    PF_LAUNCHED(1);
  }
  if (s->mixed && zf) {
    launch_to_f32(s->nunk, z, zf, s->stream);
    PF_LAUNCHED(1);
  }
  return PF_OK;
}

// FP32 copy of the Krylov vectors for the mixed CPR preconditioner (null otherwise)
float* precond_vf(pf_sim* s) { return s->mixed && s->opts.precond == PF_PC_CPR ? s->Vf : nullptr; }

pf_status dev_norm2(pf_sim* s, const double* a, double* out_host) {
  launch_dot(s->nunk, a, a, s->partial, s->nblocks, s->norms, s->red_counter, s->stream);
  PF_LAUNCHED(1);
  PF_CUDA(cudaMemcpyAsync(s->h_pinned, s->norms, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  *out_host = sqrt(s->h_pinned[0]);
  return PF_OK;
}

// The first basis vector of a Krylov cycle: V_0 = a (a copy; in mixed
// precision with CPR also the FP32 copy the preconditioner takes) and its
// normalisation vs[0] = 1 / |a|, given as inv_norm.
void start_basis(pf_sim* s, const double* a, double inv_norm) {
  launch_fill(1, 1.0, s->norms + 3, s->stream);
  launch_scale_by_dev(s->nunk, a, s->norms + 3, 0, s->V, s->stream, precond_vf(s));
  launch_fill(1, inv_norm, s->vs, s->stream);
  s->launches += 3;
}

// Work of Arnoldi step j, in three pieces: z_j = M^{-1} V_j; w = J z_j into
// V_{j+1}; two classical Gram-Schmidt passes against v_0..v_j (fused) and the
// copy of the Hessenberg column to pinned host memory.  The basis is kept
// before normalisation: V_j holds the orthogonalised vector and vs[j] = 1 /
// |V_j|, so v_j = vs[j] V_j.  The dot products and the projection carry vs[j]
// (one multiply per basis vector), and the preconditioner takes V_j itself:
// with z_j = M^{-1} V_j the flexible Arnoldi relation J z_j = sum_i h_ij v_i
// holds as before, and no pass over the vector normalises it.
pf_status piece_pre(pf_sim* s, int j) {
  return precond_apply(s, s->V + (size_t)j * s->ld, fp32_basis(s) ? nullptr : s->Z + (size_t)j * s->ld,
                       s->mixed ? s->Zf + (size_t)j * s->ld : nullptr, precond_vf(s));
}
pf_status piece_spmv(pf_sim* s, int j) {
  if (!s->mixed) return spmv(s, s->Z + (size_t)j * s->ld, s->V + (size_t)(j + 1) * s->ld);
  // mixed precision: FP32 operator on the FP32 copy of z_j
  KtScope t(s, PF_KT_SPMV);
  launch_spmv_f32(s->g, wells_view(s), (const float*)s->J, (const float*)s->Bw, (const float*)s->Cw,
                  (const float*)s->Dw, s->Zf + (size_t)j * s->ld, s->V + (size_t)(j + 1) * s->ld, s->stream,
                  s->tune.spmv);
  PF_LAUNCHED(1);
  return PF_OK;
}
pf_status piece_ortho(pf_sim* s, int j) {
  const long long n = s->nunk, ld = s->ld;
  const int k = j + 1;
  double* w = s->V + (size_t)(j + 1) * ld;
  cudaStream_t st = s->stream;
  KtScope t(s, PF_KT_ORTHO);
  // pass 1: hbuf[0..k) = h_i = vs[i] <V_i, w> and hbuf[k] = |w|^2; the
  // projected norm by Pythagoras, |w|^2 - sum_i h_i^2, and its 1/sqrt at
  // hbuf[256..257] (and into vs[j+1]), with the reorthogonalisation flag at
  // hbuf+384 when it falls below eta^2 |w|^2; then w -= sum_i h_i vs[i] V_i
  // (no norm pass).  pass 2 runs only if flagged: hbuf[128..128+k) the same
  // dots, w -= the same projection, and its measured |w|^2 and 1/|w|
  // overwrite hbuf[256..257] and vs[j+1].  Without the flag the first pass
  // kept more than eta^2 of |w|^2, so the Pythagorean value carries a relative
  // error of at most about k eps / eta^2.
  const double eta2 = s->opts.reorth_eta * s->opts.reorth_eta;
  int* reorth = reinterpret_cast<int*>(s->hbuf + 384);
  float* wf = precond_vf(s);  // the FP32 copy of V_{j+1} for the next step's preconditioner (mixed CPR)
  launch_multidot(n, k, s->V, ld, w, s->partial, s->nblocks, s->hbuf, s->red_counter, st, 1, nullptr, s->vs,
                  s->hbuf + 256, s->vs + j + 1, reorth, eta2);
  launch_axpy_norm(n, k, s->V, ld, s->hbuf, w, s->partial, s->nblocks, nullptr, s->red_counter, nullptr, nullptr,
                   nullptr, st, eta2, s->vs, wf, nullptr);
  launch_multidot(n, k, s->V, ld, w, s->partial, s->nblocks, s->hbuf + 128, s->red_counter, st, 0, reorth, s->vs);
  launch_axpy_norm(n, k, s->V, ld, s->hbuf + 128, w, s->partial, s->nblocks, s->hbuf + 256, s->red_counter, nullptr,
                   nullptr, reorth, st, 0.5, s->vs, wf, s->vs + j + 1);
  PF_LAUNCHED(4);
  PF_CUDA(cudaMemcpyAsync(s->h_pinned + kPinStep + (j & 1) * kPinStepStride, s->hbuf, (3 * 128 + 1) * sizeof(double),
                          cudaMemcpyDeviceToHost, st));
  return PF_OK;
}

// Captures one piece into an executable graph on the private capture stream.
pf_status capture(pf_sim* s, pf_status (*piece)(pf_sim*, int), int j, cudaGraphExec_t* exec, int* kernels) {
  cudaStream_t orig = s->stream;
  const int64_t l0 = s->launches;
  s->stream = s->cap_stream;
  s->capturing = true;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
  pf_status rc = PF_OK;
  if (e == cudaSuccess) {
    rc = piece(s, j);
    cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &graph);
    if (e2 != cudaSuccess && rc == PF_OK) e = e2;
  }
  s->capturing = false;
  s->stream = orig;
  if (rc != PF_OK) return rc;
  PF_CUDA(e);
  PF_CUDA(cudaGraphInstantiate(exec, graph, 0));
  cudaGraphDestroy(graph);
  *kernels = (int)(s->launches - l0);
  s->launches = l0;
  return PF_OK;
}

// Enqueues Arnoldi step j (no host synchronisation) and records its
// completion event; arnoldi_wait blocks until its Hessenberg column is in
// pinned memory.
pf_status arnoldi_enqueue(pf_sim* s, int j) {
  cudaStream_t st = s->stream;
  pf_status rc;
  if (!s->use_graphs) {
    if ((rc = piece_pre(s, j)) != PF_OK) return rc;
    if ((rc = piece_spmv(s, j)) != PF_OK) return rc;
    if ((rc = piece_ortho(s, j)) != PF_OK) return rc;
  } else {
    if ((int)s->graphs.size() <= j) s->graphs.resize(j + 1);
    pf_sim::IterGraphs& G = s->graphs[j];
    if (!G.pre) {
      if ((rc = capture(s, piece_pre, j, &G.pre, &G.k_pre)) != PF_OK) return rc;
      if ((rc = capture(s, piece_spmv, j, &G.spmv, &G.k_spmv)) != PF_OK) return rc;
      if ((rc = capture(s, piece_ortho, j, &G.ortho, &G.k_ortho)) != PF_OK) return rc;
    }
    {
      KtScope t(s, PF_KT_PRECOND);
      PF_CUDA(cudaGraphLaunch(G.pre, st));
    }
    {
      KtScope t(s, PF_KT_SPMV);
      PF_CUDA(cudaGraphLaunch(G.spmv, st));
    }
    {
      KtScope t(s, PF_KT_ORTHO);
      PF_CUDA(cudaGraphLaunch(G.ortho, st));
    }
    s->launches += G.k_pre + G.k_spmv + G.k_ortho;
  }
  PF_CUDA(cudaEventRecord(s->step_done[j & 1], st));
  return PF_OK;
}

pf_status arnoldi_wait(pf_sim* s, int j) {
  PF_CUDA(cudaEventSynchronize(s->step_done[j & 1]));
  return PF_OK;
}

// Restarted flexible GMRES (right preconditioning) for J x = b, x0 = 0.
// bnorm_known > 0 is |b| when the caller has it (the Newton right-hand side
// -R, whose 2-norm the residual check just formed); otherwise it is computed.
// Returns without synchronising the stream: x is ready in stream order.
// Arnoldi with classical Gram-Schmidt applied twice; the second projection
// reuses the pass that applies the first (fused kernel), and the
// Hessenberg column crosses to the host once per iteration for the Givens
// rotations.
pf_status gmres(pf_sim* s, const double* bvec, double* xout, double rtol, int maxit, int* iters, double* relres,
                double bnorm_known = 0.0) {
  const long long n = s->nunk, ld = s->ld;
  const int m = s->opts.gmres_restart;
  cudaStream_t st = s->stream;
  pf_status rc;
  double bnorm = bnorm_known;
  if (!(bnorm > 0.0) && (rc = dev_norm2(s, bvec, &bnorm)) != PF_OK) return rc;
  launch_fill(n, 0.0, xout, st);
  s->launches += 1;
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  if (!(bnorm > 0.0)) {
    if (!std::isfinite(bnorm)) return fail(PF_ENOT_CONVERGED, "non-finite right-hand side");
    return PF_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  int total = 0;
  double beta = bnorm;
  double res = bnorm;
  bool converged = false;
  bool first = true;
  while (total < maxit && !converged) {
    start_basis(s, first ? bvec : s->r, 1.0 / beta);  // the first cycle's residual is b itself
    first = false;
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jdone = 0;
    bool queued = false;       // step j was enqueued ahead, while step j - 1 ran
    double prev = beta;        // residual after the last step the host has read
    double rate = s->krylov_rate;
    for (int j = 0; j < m && total < maxit; ++j) {
      if (!queued && (rc = arnoldi_enqueue(s, j)) != PF_OK) return rc;
      // look ahead: put step j + 1 behind step j before reading step j, unless
      // the residual extrapolated one step (prev * rate) is within 3x of the
      // tolerance, where step j may be the last one
      queued = s->opts.krylov_lookahead && j + 1 < m && total + 1 < maxit && prev * rate > 3.0 * rtol * bnorm;
      if (queued && (rc = arnoldi_enqueue(s, j + 1)) != PF_OK) return rc;
      if ((rc = arnoldi_wait(s, j)) != PF_OK) return rc;
      const int k = j + 1;
      const double* hp = s->h_pinned + kPinStep + (j & 1) * kPinStepStride;
      const double* h1 = hp;
      const double* h2 = hp + 128;
      const bool second_pass = reinterpret_cast<const int*>(hp + 384)[0] != 0;
      const double hn = sqrt(std::max(hp[256], 0.0));
      double* col = &H[(size_t)j * (m + 1)];
      for (int i = 0; i < k; ++i) col[i] = h1[i] + (second_pass ? h2[i] : 0.0);
      col[k] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
      }
      const double den = hypot(col[j], col[j + 1]);
      cs[j] = den > 0.0 ? col[j] / den : 1.0;
      sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
      col[j] = den;
      col[j + 1] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      res = fabs(gv[j + 1]);
      ++total;
      jdone = j + 1;
      if (!std::isfinite(res)) return fail(PF_ENOT_CONVERGED, "Krylov solve produced a non-finite residual");
      if (prev > 0.0) rate = std::min(res / prev, 1.0);
      prev = res;
      if (res <= rtol * bnorm || hn == 0.0) { converged = true; break; }
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double t = gv[i];
      for (int l = i + 1; l < jdone; ++l) t -= H[(size_t)l * (m + 1) + i] * y[l];
      y[i] = t / H[(size_t)i * (m + 1) + i];
    }
    memcpy(s->h_pinned + kPinY, y.data(), jdone * sizeof(double));
    PF_CUDA(cudaMemcpyAsync(s->ydev, s->h_pinned + kPinY, jdone * sizeof(double), cudaMemcpyHostToDevice, st));
    if (fp32_basis(s)) launch_multi_axpy_add_f32(n, jdone, s->Zf, ld, s->ydev, xout, st);
    else launch_multi_axpy_add(n, jdone, s->Z, ld, s->ydev, xout, st);
    s->launches += 1;
    if (!converged && total < maxit) {
      if ((rc = spmv(s, xout, s->r)) != PF_OK) return rc;
      launch_sub(n, bvec, s->r, s->r, st);
      s->launches += 1;
      if ((rc = dev_norm2(s, s->r, &beta)) != PF_OK) return rc;
      res = beta;
      if (beta <= rtol * bnorm) converged = true;
    }
  }
  if (total > 0 && res > 0.0) s->krylov_rate = std::min(pow(res / bnorm, 1.0 / total), 1.0);
  if (iters) *iters = total;
  if (relres) *relres = res / bnorm;
  return PF_OK;
}

pf_status residual_norms(pf_sim* s, double* scaled, double* norm2) {
  launch_residual_norms(s->g, s->ph, s->inv_pv, wells_view(s), s->R, s->dt, s->partial, s->nblocks, s->norms,
                        s->stream);
  PF_LAUNCHED(2);
  PF_CUDA(cudaMemcpyAsync(s->h_pinned, s->norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  *scaled = s->h_pinned[0];
  *norm2 = sqrt(s->h_pinned[1]);
  return PF_OK;
}

pf_status check(pf_sim* s) {
  if (!s) return fail(PF_EINVAL, "pf_sim is NULL");
  if (s->dead) return fail(PF_ECUDA, "pf_sim is unusable after an earlier CUDA error");
  PF_CUDA(cudaSetDevice(s->device));
  return PF_OK;
}

double clamp_eta(double eta) { return std::isnan(eta) ? 0.1 : std::min(std::max(eta, 0.01), 0.1); }

double forcing_term(double nb, double nb_prev) {
  // forcing term of Sec. 3.3, third choice: gamma (|b^l| / |b^{l-1}|)^beta, gamma = 0.5,
  // beta = (sqrt(5) + 1) / 2, restricted to [0.01, 0.1]; first iteration 0.1
  if (!(nb_prev > 0.0)) return 0.1;
  return clamp_eta(0.5 * pow(nb / nb_prev, (sqrt(5.0) + 1.0) / 2.0));
}

}  // namespace

namespace pf {

pf_status assemble_packed(pf_sim* const* sims, int n, cudaStream_t st, int* launches) {
  if (n < 1) return PF_OK;
  for (int i = 0; i < n; ++i)
    if (sims[i]->mixed != sims[0]->mixed) return fail(PF_EINVAL, "a pack mixes precisions");
  return sims[0]->mixed ? assemble_packed_t<float>(sims, n, st, launches)
                        : assemble_packed_t<double>(sims, n, st, launches);
}

void set_assembly_packer(pf_sim* s, pf_status (*fn)(void*, pf_sim*), void* ctx) {
  s->packer = fn;
  s->packer_ctx = ctx;
}

cudaStream_t sim_stream(const pf_sim* s) { return s->stream; }

}  // namespace pf

extern "C" {

pf_status pf_set_programmatic_launch(int on) {
  g_pdl.store(on != 0);
  return PF_OK;
}

pf_status pf_inject_create_failure(int k) {
  if (k < 0) return fail(PF_EINVAL, "pf_inject_create_failure: k must be >= 0");
  g_inject_k.store(k);
  return PF_OK;
}

const char* pf_version(void) { return "polyflood-gb300 0.1 (sm_103a)"; }

const char* pf_last_error(void) { return g_last_error.c_str(); }

pf_status pf_default_opts(pf_solver_opts* o) {
  if (!o) return fail(PF_EINVAL, "opts is NULL");
  o->precision = PF_PREC_FP64;
  o->precond = PF_PC_BJACOBI;
  o->gmres_restart = 30;
  o->gmres_max_iter = 300;
  o->newton_max_iter = 25;
  o->use_forcing = 0;
  o->lin_rtol = 1e-12;
  o->newton_tol = 1e-10;
  o->ds_max = 0.2;
  o->dc_frac = 0.5;
  o->amg_pre_sweeps = 1;
  o->amg_post_sweeps = 1;
  o->amg_coarse_size = 32;
  o->amg_cycle = 1;
  o->autotune = 0;
  o->forcing_form = 3;
  o->stage1 = PF_S1_ILU0;
  o->amg_coarse_sweeps = 2;
  o->reorth_eta = 0.2;
  o->ilu_guard = 0.1;
  o->newton_div = 1e6;
  o->ilu_store = -1;
  o->krylov_lookahead = 1;
  return PF_OK;
}

pf_status pf_create(const pf_model_desc* m, const pf_solver_opts* o, void* stream, pf_sim** out) {
  if (!out) return fail(PF_EINVAL, "out is NULL");
  *out = nullptr;
  pf_solver_opts opts;
  pf_default_opts(&opts);
  if (o) opts = *o;
  pf_status rc = validate(m, &opts);
  if (rc != PF_OK) return rc;
  pf_sim* s = new (std::nothrow) pf_sim();
  if (!s) return fail(PF_ENOMEM, "host allocation failed");
  s->opts = opts;
  s->mixed = opts.precision == PF_PREC_MIXED;
  s->stream = (cudaStream_t)stream;
  {
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) { delete s; return fail(PF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e)); }
  }
  Grid& g = s->g;
  g.nx = m->nx; g.ny = m->ny; g.nz = m->nz;
  g.nxy = (long long)m->nx * m->ny;
  g.n = g.nxy * m->nz;
  g.dx = m->dx; g.dy = m->dy; g.dz = m->dz; g.top = m->top;
  g.V = m->dx * m->dy * m->dz;
  s->ph = derive_phys(m->phys);
  set_tables(s->ph, *m);
  s->nw = m->n_wells;
  s->h_ptr.assign(s->nw + 1, 0);
  for (int w = 0; w < s->nw; ++w) s->h_ptr[w + 1] = s->h_ptr[w] + m->wells[w].n_perf;
  s->npf = s->h_ptr[s->nw];
  s->nunk = 3 * g.n + s->nw;
  s->ld = (long long)align_up((size_t)s->nunk, 64);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  // reduction grids: about 8 entries per thread, from one to four blocks of
  // 256 per SM (the last block of each reduction sums one row per block)
  s->nblocks = (int)std::min<long long>(4LL * sms, std::max<long long>(sms, (s->nunk + 2047) / 2048));
  s->h_ctl.resize(s->nw);
  s->switched.assign(s->nw, 0);
  // host set-up: transmissibilities and well indices
  const long long n = g.n;
  std::vector<double> T3((size_t)3 * n, 0.0);
  for (long long k = 0; k < g.nz; ++k)
    for (long long j = 0; j < g.ny; ++j)
      for (long long i = 0; i < g.nx; ++i) {
        const long long c = i + g.nx * (j + g.ny * k);
        if (i + 1 < g.nx) {  // harmonic sum of half-cell resistances, Sec. 3.2
          const long long h = c + 1;
          T3[c] = (g.dy * g.dz) / (g.dx / (2.0 * m->kx[c]) + g.dx / (2.0 * m->kx[h]));
        }
        if (j + 1 < g.ny) {
          const long long h = c + g.nx;
          T3[n + c] = (g.dx * g.dz) / (g.dy / (2.0 * m->ky[c]) + g.dy / (2.0 * m->ky[h]));
        }
        if (k + 1 < g.nz) {
          const long long h = c + g.nxy;
          T3[2 * n + c] = (g.dx * g.dy) / (g.dz / (2.0 * m->kz[c]) + g.dz / (2.0 * m->kz[h]));
        }
      }
  // pore-volume weights of the face averages (Sec. 3.2) and 1 / (V phi_r)
  std::vector<double> wL3((size_t)3 * n, 0.0), inv_pv((size_t)n);
  for (long long c = 0; c < n; ++c) {
    inv_pv[c] = 1.0 / (g.V * m->phi[c]);
    const long long st3[3] = {1, g.nx, g.nxy};
    for (int d = 0; d < 3; ++d) {
      const long long h = c + st3[d];
      if (T3[d * n + c] != 0.0) wL3[d * n + c] = m->phi[c] / (m->phi[c] + m->phi[h]);
    }
  }
  std::vector<long long> cell(std::max(1LL, s->npf));
  std::vector<double> wi(std::max(1LL, s->npf)), dzb(std::max(1LL, s->npf));
  std::vector<int> kind(std::max(1, s->nw));
  std::vector<double> Wsc(std::max(1, s->nw));
  std::vector<double> pb0(std::max(1, s->nw));
  for (int w = 0; w < s->nw; ++w) {
    const pf_well_desc& d = m->wells[w];
    kind[w] = d.kind;
    pb0[w] = d.pb0;
    double sum = 0.0;
    const double zb = g.top + ((double)(d.cells[0] / g.nxy) + 0.5) * g.dz;
    for (int q = 0; q < d.n_perf; ++q) {
      const long long c = d.cells[q];
      const int dir = d.dirs ? d.dirs[q] : PF_DIR_Z;
      const long long t = s->h_ptr[w] + q;
      cell[t] = c;
      wi[t] = well_index(m->kx[c], m->ky[c], m->kz[c], g.dx, g.dy, g.dz, dir, d.rw, d.skin, d.gf, d.f, d.fh);
      dzb[t] = g.top + ((double)(c / g.nxy) + 0.5) * g.dz - zb;
      sum += wi[t];
    }
    Wsc[w] = sum * m->phys.rho_w / m->phys.mu_w;
  }
  s->h_kind.assign(kind.begin(), kind.begin() + s->nw);
  s->h_cell.assign(cell.begin(), cell.begin() + s->npf);
  s->h_W.assign(Wsc.begin(), Wsc.begin() + s->nw);
  // device arena
  s->cpr.coarse_limit = std::min(std::max(opts.amg_coarse_size, 1), 64);
  s->cpr.ilu = opts.stage1 == PF_S1_ILU0;
  s->arena_bytes = carve(s, nullptr);
  // Every CUDA call from here on goes through PF_CREATE: a failure frees
  // whatever the sim holds so far (pf_destroy handles a partly built sim) and
  // returns the status with the call's message.  inject_hit() lets a test make
  // the k-th of these calls fail on the host (pf_inject_create_failure).
  int site = 0;
#define PF_CREATE(call, inj_err, status)                                                     \
  do {                                                                                      \
    cudaError_t e_ = inject_hit(&site) ? (inj_err) : (call);                                \
    if (e_ != cudaSuccess) {                                                                \
      cudaGetLastError();                                                                   \
      const std::string msg_ = std::string("pf_create: ") + #call + ": " + cudaGetErrorString(e_); \
      pf_destroy(s);                                                                        \
      return fail((status), msg_);                                                          \
    }                                                                                       \
  } while (0)
  {
    // stream-ordered allocation: no device-wide synchronisation, so creating
    // or destroying one simulator does not stall the others' streams
    cudaError_t e = inject_hit(&site) ? cudaErrorMemoryAllocation
                                      : cudaMallocAsync((void**)&s->arena, s->arena_bytes, s->stream);
    if (e != cudaSuccess) s->arena = nullptr;
    else e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      const size_t bytes = s->arena_bytes;
      pf_destroy(s);
      return fail(PF_ENOMEM, "device arena of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
  }
  PF_CREATE(cudaMallocHost((void**)&s->h_pinned, kPinTotal * sizeof(double)), cudaErrorMemoryAllocation, PF_ENOMEM);
  carve(s, s->arena);
  PF_CREATE(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking), cudaErrorInvalidValue, PF_ECUDA);
  for (int q = 0; q < 2; ++q)
    PF_CREATE(cudaEventCreateWithFlags(&s->step_done[q], cudaEventDisableTiming), cudaErrorInvalidValue, PF_ECUDA);
  // upload
  std::vector<double> x0((size_t)s->nunk);
  for (long long i = 0; i < n; ++i) {
    x0[3 * i] = m->p0[i];
    x0[3 * i + 1] = m->s0[i];
    x0[3 * i + 2] = m->c0[i];
  }
  for (int w = 0; w < s->nw; ++w) x0[3 * n + w] = pb0[w];
  cudaStream_t st = s->stream;
  const cudaError_t einv = cudaErrorInvalidValue;
  PF_CREATE(cudaMemsetAsync(s->arena, 0, s->arena_bytes, st), einv, PF_ECUDA);
  PF_CREATE(cudaMemcpyAsync(s->phi_r, m->phi, n * sizeof(double), cudaMemcpyHostToDevice, st), einv, PF_ECUDA);
  PF_CREATE(cudaMemcpyAsync(s->T3, T3.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, st), einv, PF_ECUDA);
  PF_CREATE(cudaMemcpyAsync(s->wL3, wL3.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, st), einv, PF_ECUDA);
  PF_CREATE(cudaMemcpyAsync(s->inv_pv, inv_pv.data(), n * sizeof(double), cudaMemcpyHostToDevice, st), einv,
            PF_ECUDA);
  PF_CREATE(cudaMemcpyAsync(s->x, x0.data(), s->nunk * sizeof(double), cudaMemcpyHostToDevice, st), einv, PF_ECUDA);
  PF_CREATE(cudaMemcpyAsync(s->w_ptr, s->h_ptr.data(), (s->nw + 1) * sizeof(int), cudaMemcpyHostToDevice, st), einv,
            PF_ECUDA);
  std::vector<double> sat_soa, poly_soa;   // live until the stream synchronises below
  if (m->n_sat > 0) {
    sat_soa = table_soa(m->sat_table, m->n_sat, 3);
    PF_CREATE(cudaMemcpyAsync(s->d_sat, sat_soa.data(), sat_soa.size() * sizeof(double), cudaMemcpyHostToDevice, st),
              einv, PF_ECUDA);
    s->ph.sat = s->d_sat;
  }
  if (m->n_poly > 0) {
    poly_soa = table_soa(m->poly_table, m->n_poly, 2);
    PF_CREATE(cudaMemcpyAsync(s->d_poly, poly_soa.data(), poly_soa.size() * sizeof(double), cudaMemcpyHostToDevice,
                              st),
              einv, PF_ECUDA);
    s->ph.poly = s->d_poly;
  }
  std::vector<int> perf_of((size_t)n, -1), pwell((size_t)std::max(1LL, s->npf), 0);
  for (int w = 0; w < s->nw; ++w)
    for (int t = s->h_ptr[w]; t < s->h_ptr[w + 1]; ++t) {
      perf_of[(size_t)cell[t]] = t;
      pwell[(size_t)t] = w;
    }
  PF_CREATE(cudaMemcpyAsync(s->w_perf_of, perf_of.data(), n * sizeof(int), cudaMemcpyHostToDevice, st), einv,
            PF_ECUDA);
  PF_CREATE(cudaMemcpyAsync(s->w_pwell, pwell.data(), pwell.size() * sizeof(int), cudaMemcpyHostToDevice, st), einv,
            PF_ECUDA);
  if (s->nw > 0) {
    PF_CREATE(cudaMemcpyAsync(s->w_kind, kind.data(), s->nw * sizeof(int), cudaMemcpyHostToDevice, st), einv,
              PF_ECUDA);
    PF_CREATE(cudaMemcpyAsync(s->w_cell, cell.data(), s->npf * sizeof(long long), cudaMemcpyHostToDevice, st), einv,
              PF_ECUDA);
    PF_CREATE(cudaMemcpyAsync(s->w_wi, wi.data(), s->npf * sizeof(double), cudaMemcpyHostToDevice, st), einv,
              PF_ECUDA);
    PF_CREATE(cudaMemcpyAsync(s->w_dzb, dzb.data(), s->npf * sizeof(double), cudaMemcpyHostToDevice, st), einv,
              PF_ECUDA);
    PF_CREATE(cudaMemcpyAsync(s->w_W, Wsc.data(), s->nw * sizeof(double), cudaMemcpyHostToDevice, st), einv,
              PF_ECUDA);
  }
  if (s->opts.precond == PF_PC_CPR) {
    pf_status r2 = cpr_init(s->cpr, s->g, s->mixed, s->opts, s->stream);
    if (r2 != PF_OK) { pf_destroy(s); return fail(r2, "CPR set-up failed"); }
  }
  PF_CREATE(cudaStreamSynchronize(st), einv, PF_ECUDA);
#undef PF_CREATE
  g_inject_k.store(0);  // armed for one pf_create only, also when it had fewer guarded calls than k
  if (s->opts.autotune) {
    pf_status r3 = pf_autotune(s, nullptr);
    if (r3 != PF_OK) {
      std::string msg = pf_last_error();
      pf_destroy(s);
      return fail(r3, "launch-shape tuning failed: " + msg);
    }
  }
  *out = s;
  return PF_OK;
}

pf_status pf_footprint(const pf_model_desc* m, const pf_solver_opts* o, size_t* bytes) {
  if (!bytes) return fail(PF_EINVAL, "bytes is NULL");
  pf_solver_opts opts;
  pf_default_opts(&opts);
  if (o) opts = *o;
  pf_status rc = validate(m, &opts);
  if (rc != PF_OK) return rc;
  pf_sim tmp;
  tmp.opts = opts;
  tmp.mixed = opts.precision == PF_PREC_MIXED;
  tmp.g.nx = m->nx; tmp.g.ny = m->ny; tmp.g.nz = m->nz;
  tmp.g.nxy = (long long)m->nx * m->ny;
  tmp.g.n = tmp.g.nxy * m->nz;
  tmp.nw = m->n_wells;
  tmp.ph.n_sat = m->n_sat;
  tmp.ph.n_poly = m->n_poly;
  tmp.npf = 0;
  for (int w = 0; w < m->n_wells; ++w) tmp.npf += m->wells[w].n_perf;
  tmp.nunk = 3 * tmp.g.n + tmp.nw;
  tmp.ld = (long long)align_up((size_t)tmp.nunk, 64);
  tmp.nblocks = 4 * 152;
  tmp.cpr.coarse_limit = std::min(std::max(opts.amg_coarse_size, 1), 64);
  // arena + pinned staging + graph and context overheads (a fixed allowance)
  *bytes = carve(&tmp, nullptr) + ((size_t)8 << 20);
  return PF_OK;
}

pf_status pf_destroy(pf_sim* s) {
  if (!s) return PF_OK;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& G : s->graphs) {
    if (G.pre) cudaGraphExecDestroy(G.pre);
    if (G.spmv) cudaGraphExecDestroy(G.spmv);
    if (G.ortho) cudaGraphExecDestroy(G.ortho);
  }
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  for (cudaEvent_t ev : s->step_done)
    if (ev) cudaEventDestroy(ev);
  if (s->arena) {
    cudaFreeAsync(s->arena, s->stream);
    cudaStreamSynchronize(s->stream);
  }
  if (s->h_pinned) cudaFreeHost(s->h_pinned);
  for (auto& p : s->kt_pending) { s->kt_pool.push_back(p.second.first); s->kt_pool.push_back(p.second.second); }
  for (cudaEvent_t e : s->kt_pool) cudaEventDestroy(e);
  delete s;
  return PF_OK;
}

static pf_status upload_controls(pf_sim* s, const pf_well_control* c, int nwells) {
  std::vector<int> ctrl(std::max(1, nwells));
  std::vector<double> target(std::max(1, nwells)), cinj(std::max(1, nwells)), sw(std::max(1, nwells)),
      so(std::max(1, nwells)), scale(std::max(1, nwells));
  const Phys& ph = s->ph;
  for (int w = 0; w < nwells; ++w) {
    const pf_well_control& k = c[w];
    if (!std::isfinite(k.target) || !std::isfinite(k.c_inj) || k.c_inj < 0.0) return fail(PF_EINVAL, "invalid control");
    const bool inj = s->h_kind[w] == PF_WELL_INJECTOR;
    ctrl[w] = k.ctrl;
    cinj[w] = k.c_inj;
    sw[w] = so[w] = 0.0;
    double rho_t = 1.0;
    switch (k.ctrl) {
      case PF_CTRL_BHP:
        target[w] = k.target;
        scale[w] = s->h_W[w] * 1.0e5;
        break;
      case PF_CTRL_WRATE:
        sw[w] = inj ? 1.0 : -1.0;
        rho_t = ph.rho_w;
        break;
      case PF_CTRL_ORATE:
        if (inj) return fail(PF_EINVAL, "oil-rate control on an injector");
        so[w] = -1.0;
        rho_t = ph.rho_o;
        break;
      case PF_CTRL_LRATE:
        if (inj) return fail(PF_EINVAL, "liquid-rate control on an injector");
        sw[w] = -1.0;
        so[w] = -ph.rho_w / ph.rho_o;
        rho_t = ph.rho_w;
        break;
      default:
        return fail(PF_EINVAL, "unknown control");
    }
    if (k.ctrl != PF_CTRL_BHP) {
      if (!(k.target >= 0.0)) return fail(PF_EINVAL, "rate targets are non-negative volume rates");
      target[w] = rho_t * k.target;
      scale[w] = rho_t * std::max(fabs(k.target), 1e-30);
    }
  }
  cudaStream_t st = s->stream;
  if (nwells > 0) {
    PF_CUDA(cudaMemcpyAsync(s->w_ctrl, ctrl.data(), nwells * sizeof(int), cudaMemcpyHostToDevice, st));
    PF_CUDA(cudaMemcpyAsync(s->w_target, target.data(), nwells * sizeof(double), cudaMemcpyHostToDevice, st));
    PF_CUDA(cudaMemcpyAsync(s->w_cinj, cinj.data(), nwells * sizeof(double), cudaMemcpyHostToDevice, st));
    PF_CUDA(cudaMemcpyAsync(s->w_sw, sw.data(), nwells * sizeof(double), cudaMemcpyHostToDevice, st));
    PF_CUDA(cudaMemcpyAsync(s->w_so, so.data(), nwells * sizeof(double), cudaMemcpyHostToDevice, st));
    PF_CUDA(cudaMemcpyAsync(s->w_scale, scale.data(), nwells * sizeof(double), cudaMemcpyHostToDevice, st));
    PF_CUDA(cudaStreamSynchronize(st));
  }
  return PF_OK;
}

pf_status pf_set_controls(pf_sim* s, const pf_well_control* c, int nwells) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (nwells != s->nw || (nwells > 0 && !c)) return fail(PF_EINVAL, "control count must equal the well count");
  if ((rc = upload_controls(s, c, nwells)) != PF_OK) return rc;
  for (int w = 0; w < nwells; ++w) {
    // a well keeps its switched state only while its constraint is unchanged
    if (c[w].ctrl != s->h_ctl[w].ctrl || c[w].target != s->h_ctl[w].target || c[w].limit != s->h_ctl[w].limit)
      s->switched[w] = 0;
    s->h_ctl[w] = c[w];
  }
  s->have_controls = true;
  return PF_OK;
}

// Controls in force for the next solve: switched rate wells run on BHP = limit.
static std::vector<pf_well_control> effective_controls(const pf_sim* s) {
  std::vector<pf_well_control> e(s->h_ctl);
  for (int w = 0; w < s->nw; ++w)
    if (s->switched[w]) { e[w].ctrl = PF_CTRL_BHP; e[w].target = e[w].limit; }
  return e;
}

pf_status pf_begin_step(pf_sim* s, double dt) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(PF_EINVAL, "dt must be finite and positive");
  if (!s->have_controls && s->nw > 0) return fail(PF_EINVAL, "pf_set_controls must precede the first step");
  s->dt = dt;
  if (s->nw > 0) {
    std::vector<pf_well_control> eff = effective_controls(s);
    if ((rc = upload_controls(s, eff.data(), s->nw)) != PF_OK) return rc;
  }
  cudaStream_t st = s->stream;
  launch_copy(s->nunk, s->x, s->x_old, st);
  if (s->mixed)
    launch_cell_props<float>(s->g, s->ph, s->phi_r, s->x, s->pv, (float*)s->pd, nullptr, nullptr, nullptr, s->Mold, 1, st);
  else
    launch_cell_props<double>(s->g, s->ph, s->phi_r, s->x, s->pv, (double*)s->pd, nullptr, nullptr, nullptr, s->Mold, 1,
                              st);
  launch_well_gamma(s->g, s->ph, wells_view(s), s->x, s->pv, s->w_gamma, st);
  PF_LAUNCHED(2 + (s->nw > 0));
  s->in_step = true;
  s->assembled = false;
  s->prev_norm = -1.0;
  s->iter_in_step = 0;
  return PF_OK;
}

pf_status pf_assemble(pf_sim* s) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!s->in_step) return fail(PF_EINVAL, "pf_begin_step must precede pf_assemble");
  rc = assemble(s);
  if (rc != PF_OK) return rc;
  PF_CUDA(cudaStreamSynchronize(s->stream));
  return PF_OK;
}

static bool has_limits(const pf_sim* s);

// In-iteration limit check after an update: a rate well whose P_b crosses its
// BHP limit (above for an injector, below for a producer) moves onto BHP =
// limit for the rest of the step; the effective controls are re-uploaded.
static pf_status limit_crossings(pf_sim* s) {
  if (!has_limits(s)) return PF_OK;
  std::vector<double> pb(s->nw);
  PF_CUDA(cudaMemcpyAsync(pb.data(), s->x + 3 * s->g.n, s->nw * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  bool changed = false;
  for (int w = 0; w < s->nw; ++w) {
    const pf_well_control& c = s->h_ctl[w];
    if (c.ctrl == PF_CTRL_BHP || c.limit == 0.0 || s->switched[w]) continue;
    const int kind = s->h_kind[w];
    if ((kind == PF_WELL_INJECTOR && pb[w] > c.limit) || (kind == PF_WELL_PRODUCER && pb[w] < c.limit)) {
      s->switched[w] = 1;
      changed = true;
    }
  }
  if (!changed) return PF_OK;
  std::vector<pf_well_control> eff = effective_controls(s);
  return upload_controls(s, eff.data(), s->nw);
}

static pf_status newton_iteration(pf_sim* s, pf_iter_report* rep, bool allow_update) {
  pf_status rc;
  if ((rc = assemble(s)) != PF_OK) return rc;
  double scaled, nrm;
  if ((rc = residual_norms(s, &scaled, &nrm)) != PF_OK) return rc;
  pf_iter_report r{};
  r.res_scaled = scaled;
  r.res_norm2 = nrm;
  if (!std::isfinite(scaled) || !std::isfinite(nrm)) {
    if (rep) *rep = r;
    return fail(PF_ENOT_CONVERGED, "non-finite residual");
  }
  if (scaled <= s->opts.newton_tol) {
    r.converged = 1;
    if (rep) *rep = r;
    return PF_OK;
  }
  if (s->iter_in_step == 0) {
    s->res0 = scaled;
  } else if (s->opts.newton_div > 0.0 && scaled > s->opts.newton_div * s->res0) {
    // the iterates run away (a step too long for the start of a transient):
    // give up now rather than at the iteration cap, so that the caller cuts
    // the step before Krylov solves on runaway states cost hundreds of
    // iterations each
    if (rep) *rep = r;
    return fail(PF_ENOT_CONVERGED, "Newton iteration diverged");
  }
  if (!allow_update) {
    if (rep) *rep = r;
    return fail(PF_ENOT_CONVERGED, "Newton iteration cap reached");
  }
  // b = -R
  launch_fill(1, -1.0, s->norms + 3, s->stream);
  launch_scale_by_dev(s->nunk, s->R, s->norms + 3, 0, s->b, s->stream);
  s->launches += 2;
  const int form = s->opts.forcing_form;
  double eta = s->opts.lin_rtol;
  if (s->opts.use_forcing) {
    if (!(s->prev_norm > 0.0)) {
      eta = 0.1;                                          // first iteration of the step
    } else if (form == 1) {                               // |b^l - r^{l-1}| / |b^{l-1}|
      double d = 0.0;
      launch_sub(s->nunk, s->b, s->rlin, s->tmp, s->stream);
      s->launches += 1;
      if ((rc = dev_norm2(s, s->tmp, &d)) != PF_OK) return rc;
      eta = clamp_eta(d / s->prev_norm);
    } else if (form == 2) {                               // (|b^l| - |r^{l-1}|) / |b^{l-1}|
      eta = clamp_eta((nrm - s->prev_lin_norm) / s->prev_norm);
    } else {
      eta = forcing_term(nrm, s->prev_norm);
    }
  }
  r.eta = eta;
  if ((rc = precond_setup(s)) != PF_OK) return rc;
  int its = 0;
  double rr = 0.0;
  rc = gmres(s, s->b, s->dx, eta, s->opts.gmres_max_iter, &its, &rr, nrm);  // |b| = |R|
  r.krylov_iters = its;
  r.lin_rel_res = rr;
  if (rc != PF_OK) {
    if (rep) *rep = r;
    return rc;
  }
  if (s->opts.use_forcing && form != 3) {
    // r^l = b^l - J dx^l, the residual this linear solve left (forms 1 and 2)
    double* rl = form == 1 ? s->rlin : s->tmp;
    if ((rc = spmv(s, s->dx, rl)) != PF_OK) return rc;
    launch_sub(s->nunk, s->b, rl, rl, s->stream);
    s->launches += 1;
    if (form == 2 && (rc = dev_norm2(s, rl, &s->prev_lin_norm)) != PF_OK) return rc;
  }
  launch_newton_update(s->g, s->nw, s->x, s->dx, s->opts.ds_max, s->opts.dc_frac * s->ph.c_ref, s->stream);
  PF_LAUNCHED(1);
  if ((rc = limit_crossings(s)) != PF_OK) return rc;
  s->prev_norm = nrm;
  s->iter_in_step++;
  if (rep) *rep = r;
  return PF_OK;
}

pf_status pf_newton_iteration(pf_sim* s, pf_iter_report* rep) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!s->in_step) return fail(PF_EINVAL, "pf_begin_step must precede pf_newton_iteration");
  return newton_iteration(s, rep, true);
}

// Per-well water, oil and polymer mass rates and reference BHP at the current
// state into host arrays (any may be NULL).
static pf_status well_totals(pf_sim* s, std::vector<double>& tot, std::vector<double>& pb) {
  cudaStream_t st = s->stream;
  if (s->mixed)
    launch_cell_props<float>(s->g, s->ph, s->phi_r, s->x, s->pv, (float*)s->pd, nullptr, nullptr, nullptr, nullptr, 2, st);
  else
    launch_cell_props<double>(s->g, s->ph, s->phi_r, s->x, s->pv, (double*)s->pd, nullptr, nullptr, nullptr, nullptr, 2,
                              st);
  launch_well_totals(s->g, s->ph, wells_view(s), s->x, s->pv, s->wtot, st);
  PF_LAUNCHED(1 + (s->nw > 0));
  tot.assign(3 * (size_t)std::max(1, s->nw), 0.0);
  pb.assign(std::max(1, s->nw), 0.0);
  if (s->nw > 0) {
    PF_CUDA(cudaMemcpyAsync(tot.data(), s->wtot, 3 * s->nw * sizeof(double), cudaMemcpyDeviceToHost, st));
    PF_CUDA(cudaMemcpyAsync(pb.data(), s->x + 3 * s->g.n, s->nw * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  PF_CUDA(cudaStreamSynchronize(st));
  return PF_OK;
}

// The volume rate a rate constraint refers to (Sec. 2.4), positive.
static double controlled_rate(const Phys& ph, int kind, int ctrl, double qw, double qo) {
  if (kind == PF_WELL_INJECTOR) return qw / ph.rho_w;
  if (ctrl == PF_CTRL_WRATE) return -qw / ph.rho_w;
  if (ctrl == PF_CTRL_ORATE) return -qo / ph.rho_o;
  return -(qw / ph.rho_w + qo / ph.rho_o);
}

// Limit check after a converged step: a rate well whose BHP crosses its limit
// (above for an injector, below for a producer) moves onto BHP = limit; a
// switched well whose rate at the limit exceeds its target returns to rate
// control.  Returns true if a switch changed.
static bool update_switches(pf_sim* s, const std::vector<double>& tot, const std::vector<double>& pb) {
  bool changed = false;
  for (int w = 0; w < s->nw; ++w) {
    const pf_well_control& c = s->h_ctl[w];
    if (c.ctrl == PF_CTRL_BHP || c.limit == 0.0) continue;
    const int kind = s->h_kind[w];
    if (!s->switched[w]) {
      if ((kind == PF_WELL_INJECTOR && pb[w] > c.limit) || (kind == PF_WELL_PRODUCER && pb[w] < c.limit)) {
        s->switched[w] = 1;
        changed = true;
      }
    } else if (controlled_rate(s->ph, kind, c.ctrl, tot[3 * w], tot[3 * w + 1]) > c.target) {
      s->switched[w] = 0;
      changed = true;
    }
  }
  return changed;
}

static bool has_limits(const pf_sim* s) {
  for (int w = 0; w < s->nw; ++w)
    if (s->h_ctl[w].ctrl != PF_CTRL_BHP && s->h_ctl[w].limit != 0.0) return true;
  return false;
}

pf_status pf_end_step(pf_sim* s, int* resolve) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!resolve) return fail(PF_EINVAL, "resolve is NULL");
  *resolve = 0;
  const int max_switch_solves = 2;
  if (s->switch_attempt < max_switch_solves && has_limits(s)) {
    std::vector<double> tot, pb;
    if ((rc = well_totals(s, tot, pb)) != PF_OK) return rc;
    if (update_switches(s, tot, pb)) {
      launch_copy(s->nunk, s->x_old, s->x, s->stream);
      s->launches += 1;
      s->switch_attempt++;
      *resolve = 1;
      return PF_OK;
    }
  }
  s->switch_attempt = 0;
  s->in_step = false;
  return PF_OK;
}

pf_status pf_abort_step(pf_sim* s) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!s->in_step) return fail(PF_EINVAL, "no step in progress");
  launch_copy(s->nunk, s->x_old, s->x, s->stream);
  s->launches += 1;
  PF_CUDA(cudaStreamSynchronize(s->stream));
  s->switch_attempt = 0;
  s->in_step = false;
  return PF_OK;
}

pf_status pf_step(pf_sim* s, double dt, pf_step_report* rep) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  pf_step_report out{};
  for (;;) {
    if ((rc = pf_begin_step(s, dt)) != PF_OK) return rc;
    bool converged = false;
    for (int it = 0; it <= s->opts.newton_max_iter; ++it) {
      pf_iter_report ir{};
      rc = newton_iteration(s, &ir, it < s->opts.newton_max_iter);
      out.krylov_iters += ir.krylov_iters;
      out.res_scaled = ir.res_scaled;
      if (rc == PF_ECUDA) return rc;
      if (rc == PF_OK && ir.converged) {
        converged = true;
        out.newton_iters += it;
        break;
      }
      if (rc != PF_OK) break;
    }
    if (!converged) {
      out.newton_iters += s->opts.newton_max_iter;
      if (rep) *rep = out;
      pf_abort_step(s);
      return fail(PF_ENOT_CONVERGED, "Newton did not converge; state restored to the start of the step");
    }
    int resolve = 0;
    if ((rc = pf_end_step(s, &resolve)) != PF_OK) return rc;
    if (!resolve) break;
  }
  out.converged = 1;
  if (rep) *rep = out;
  return PF_OK;
}

pf_status pf_well_rates(pf_sim* s, double* q_w, double* q_o, double* q_p, double* pb) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  std::vector<double> tot, pbv;
  if ((rc = well_totals(s, tot, pbv)) != PF_OK) return rc;
  for (int w = 0; w < s->nw; ++w) {
    if (q_w) q_w[w] = tot[3 * w];
    if (q_o) q_o[w] = tot[3 * w + 1];
    if (q_p) q_p[w] = tot[3 * w + 2];
    if (pb) pb[w] = pbv[w];
  }
  return PF_OK;
}

pf_status pf_well_switched(const pf_sim* s, int* switched) {
  if (!s || (!switched && s->nw > 0)) return fail(PF_EINVAL, "NULL argument");
  for (int w = 0; w < s->nw; ++w) switched[w] = s->switched[w];
  return PF_OK;
}

pf_status pf_export_system(pf_sim* s, double* R, double* Jc, double* Jw_b, double* Jw_c, double* Jw_d) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!s->assembled) return fail(PF_EINVAL, "nothing assembled");
  cudaStream_t st = s->stream;
  PF_CUDA(cudaStreamSynchronize(st));
  const long long n = s->g.n;
  auto fetch = [&](const void* src, double* dst, size_t count) -> pf_status {
    if (!dst) return PF_OK;
    if (!s->mixed) {
      PF_CUDA(cudaMemcpy(dst, src, count * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
      std::vector<float> tmp(count);
      PF_CUDA(cudaMemcpy(tmp.data(), src, count * sizeof(float), cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < count; ++i) dst[i] = tmp[i];
    }
    return PF_OK;
  };
  if (R) PF_CUDA(cudaMemcpy(R, s->R, s->nunk * sizeof(double), cudaMemcpyDeviceToHost));
  if ((rc = fetch(s->J, Jc, (size_t)SL_COUNT * 9 * n)) != PF_OK) return rc;
  if (s->npf > 0) {
    if ((rc = fetch(s->Bw, Jw_b, 3 * (size_t)s->npf)) != PF_OK) return rc;
    if ((rc = fetch(s->Cw, Jw_c, 3 * (size_t)s->npf)) != PF_OK) return rc;
  }
  if (s->nw > 0 && (rc = fetch(s->Dw, Jw_d, s->nw)) != PF_OK) return rc;
  return PF_OK;
}

pf_status pf_apply_jacobian(pf_sim* s, const double* xh, double* yh) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!s->assembled) return fail(PF_EINVAL, "nothing assembled");
  if (!xh || !yh) return fail(PF_EINVAL, "NULL vector");
  PF_CUDA(cudaMemcpyAsync(s->tmp, xh, s->nunk * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  if ((rc = spmv(s, s->tmp, s->r)) != PF_OK) return rc;
  PF_CUDA(cudaMemcpyAsync(yh, s->r, s->nunk * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  return PF_OK;
}

pf_status pf_apply_preconditioner(pf_sim* s, const double* vh, double* zh) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!s->assembled) return fail(PF_EINVAL, "nothing assembled");
  if (!vh || !zh) return fail(PF_EINVAL, "NULL vector");
  if ((rc = precond_setup(s)) != PF_OK) return rc;
  PF_CUDA(cudaMemcpyAsync(s->b, vh, s->nunk * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  if ((rc = precond_apply(s, s->b, s->dx)) != PF_OK) return rc;
  PF_CUDA(cudaMemcpyAsync(zh, s->dx, s->nunk * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  return PF_OK;
}

pf_status pf_solve_linear(pf_sim* s, const double* bh, double* xh, double rtol, int* iters, double* rel_res) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!s->assembled) return fail(PF_EINVAL, "nothing assembled");
  if (!bh || !xh || !(rtol > 0.0)) return fail(PF_EINVAL, "invalid arguments");
  if ((rc = precond_setup(s)) != PF_OK) return rc;
  PF_CUDA(cudaMemcpyAsync(s->b, bh, s->nunk * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  if ((rc = gmres(s, s->b, s->dx, rtol, s->opts.gmres_max_iter, iters, rel_res)) != PF_OK) return rc;
  PF_CUDA(cudaMemcpyAsync(xh, s->dx, s->nunk * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  return PF_OK;
}

pf_status pf_get_state(pf_sim* s, double* P, double* S, double* C, double* Pb) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  const long long n = s->g.n;
  std::vector<double> xh((size_t)s->nunk);
  PF_CUDA(cudaMemcpyAsync(xh.data(), s->x, s->nunk * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  for (long long i = 0; i < n; ++i) {
    if (P) P[i] = xh[3 * i];
    if (S) S[i] = xh[3 * i + 1];
    if (C) C[i] = xh[3 * i + 2];
  }
  if (Pb) for (int w = 0; w < s->nw; ++w) Pb[w] = xh[3 * n + w];
  return PF_OK;
}

pf_status pf_set_state(pf_sim* s, const double* P, const double* S, const double* C, const double* Pb) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  const long long n = s->g.n;
  std::vector<double> xh((size_t)s->nunk);
  PF_CUDA(cudaMemcpyAsync(xh.data(), s->x, s->nunk * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  for (long long i = 0; i < n; ++i) {
    if (P) xh[3 * i] = P[i];
    if (S) xh[3 * i + 1] = S[i];
    if (C) xh[3 * i + 2] = C[i];
  }
  if (Pb) for (int w = 0; w < s->nw; ++w) xh[3 * n + w] = Pb[w];
  for (long long i = 0; i < s->nunk; ++i)
    if (!std::isfinite(xh[i])) return fail(PF_EINVAL, "state must be finite");
  PF_CUDA(cudaMemcpyAsync(s->x, xh.data(), s->nunk * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  s->assembled = false;
  return PF_OK;
}

pf_status pf_sizes(const pf_sim* s, int64_t* n_cells, int* n_wells, int64_t* n_perf) {
  if (!s) return fail(PF_EINVAL, "pf_sim is NULL");
  if (n_cells) *n_cells = s->g.n;
  if (n_wells) *n_wells = s->nw;
  if (n_perf) *n_perf = s->npf;
  return PF_OK;
}

pf_status pf_device_state(pf_sim* s, double** x_dev) {
  if (!s || !x_dev) return fail(PF_EINVAL, "NULL argument");
  *x_dev = s->x;
  return PF_OK;
}

}  // extern "C"

// Mean time of `reps` launches issued by fn on the sim's stream (after one warm-up).
template <typename F>
static float time_launch(pf_sim* s, F fn, int reps) {
  fn();
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, s->stream);
  for (int r = 0; r < reps; ++r) fn();
  cudaEventRecord(b, s->stream);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

template <typename F>
static int pick_from(pf_sim* s, const int* cand, int nc, F fn_of_block) {
  int best = cand[nc - 1];
  float tbest = 1e30f;
  for (int q = 0; q < nc; ++q) {
    const float t = time_launch(s, [&] { fn_of_block(cand[q]); }, 3);
    if (t < tbest) { tbest = t; best = cand[q]; }
  }
  return best;
}

// For candidates whose times differ by a few percent (whole preconditioner
// applications): the candidates take turns over `rounds` rounds and each
// keeps its fastest round, so a slow stretch of the device in one round does
// not decide the choice.
template <typename F>
static int pick_interleaved(pf_sim* s, const int* cand, int nc, int rounds, F fn) {
  float tmin[8];
  for (int q = 0; q < nc; ++q) tmin[q] = 1e30f;
  for (int r = 0; r < rounds; ++r)
    for (int q = 0; q < nc; ++q) tmin[q] = std::min(tmin[q], time_launch(s, [&] { fn(cand[q]); }, 3));
  int best = nc - 1;
  for (int q = 0; q < nc; ++q)
    if (tmin[q] < tmin[best]) best = q;
  return cand[best];
}

template <typename F>
static int pick_block(pf_sim* s, F fn_of_block) {
  static const int cand[3] = {64, 128, 256};
  return pick_from(s, cand, 3, fn_of_block);
}

extern "C" {

pf_status pf_autotune(pf_sim* s, pf_tuning* out) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  cudaStream_t st = s->stream;
  Tuning t;
  const double dt = s->dt > 0.0 ? s->dt : 86400.0;
  // the kernels run on the current buffers; what they write is scratch for
  // the next assembly (residual, Jacobian, property scratch, multigrid vectors)
  if (s->mixed) {
    t.props = pick_block(s, [&](int b) { launch_cell_props<float>(s->g, s->ph, s->phi_r, s->x, s->pv, (float*)s->pd,
                                                                 s->Mold, s->R, (float*)s->J, nullptr, 0, st, b); });
    t.face = pick_block(s, [&](int b) { launch_face_flux<float>(s->g, s->ph, s->wL3, s->T3, s->x, s->pv,
                                                               (const float*)s->pd, dt, (float*)s->J, s->Fbuf, st, b); });
    t.gather = pick_block(s, [&](int b) { launch_gather<float>(s->g, s->Fbuf, s->R, (float*)s->J, st, b); });
    t.spmv = pick_block(s, [&](int b) {
      launch_spmv_f32(s->g, wells_view(s), (const float*)s->J, (const float*)s->Bw, (const float*)s->Cw,
                      (const float*)s->Dw, s->Zf, s->r, st, b);
    });
    if (s->opts.precond == PF_PC_CPR)
      t.stage2 = pick_block(s, [&](int b) {
        cpr_time_stage2(s->cpr, s->g, wells_view(s), true, s->J, s->Bw, s->x, s->tmp, b, st);
      });
  } else {
    t.props = pick_block(s, [&](int b) { launch_cell_props<double>(s->g, s->ph, s->phi_r, s->x, s->pv,
                                                                  (double*)s->pd, s->Mold, s->R, (double*)s->J,
                                                                  nullptr, 0, st, b); });
    t.face = pick_block(s, [&](int b) { launch_face_flux<double>(s->g, s->ph, s->wL3, s->T3, s->x, s->pv,
                                                                (const double*)s->pd, dt, (double*)s->J, s->Fbuf, st,
                                                                b); });
    t.gather = pick_block(s, [&](int b) { launch_gather<double>(s->g, s->Fbuf, s->R, (double*)s->J, st, b); });
    // one thread per cell (64/128/256) or one per block row (-96/-192/-384)
    if (s->opts.precond == PF_PC_CPR)
      t.stage2 = pick_block(s, [&](int b) {
        cpr_time_stage2(s->cpr, s->g, wells_view(s), false, s->J, s->Bw, s->x, s->tmp, b, st);
      });
    static const int cand_spmv[6] = {64, 128, 256, -96, -192, -384};
    t.spmv = pick_from(s, cand_spmv, 6, [&](int b) {
      launch_spmv<double>(s->g, wells_view(s), (const double*)s->J, (const double*)s->Bw, (const double*)s->Cw,
                          (const double*)s->Dw, s->b, s->r, st, b);
    });
  }
  if (s->opts.precond == PF_PC_CPR) {
    // the finest smoother's block size, timed as whole preconditioner
    // applications (on small grids one smoother pass takes a few microseconds,
    // about what it takes to enqueue it, so timing the pass alone measures the
    // enqueueing), in turns over five rounds
    s->cpr.block_stage2 = t.stage2;
    static const int cand_rbgs[3] = {64, 128, 256};
    t.rbgs = pick_interleaved(s, cand_rbgs, 3, 5, [&](int b) {
      s->cpr.block_rbgs0 = b;
      precond_apply(s, s->b, s->dx, s->mixed ? s->Zf : nullptr);
    });
    s->cpr.block_rbgs0 = t.rbgs;
    // whole preconditioner applications: ILU(0) solve in two or three launches
    // (with the copies there is one form, through the set-up's products J_bj D_j^-1)
    if (s->opts.stage1 == PF_S1_ILU0 && s->cpr.ilu_cp.kind == 0) {
      static const int cand_fused[2] = {1, 0};
      t.ilu_fused = pick_interleaved(s, cand_fused, 2, 5, [&](int f) {
        s->cpr.ilu_fused = f;
        precond_apply(s, s->b, s->dx, s->mixed ? s->Zf : nullptr);
      });
      s->cpr.ilu_fused = t.ilu_fused;
    }
    // the single-block threshold keeps its default: timed on the set-up's
    // placeholder data the two candidates differ by less than the noise, and
    // measured on live systems the default was the faster (256 cells in FP64,
    // 4096 in FP32); pf_set_tuning can still change it
    t.block_cells = (int)s->cpr.block_cells;
    t.cluster_cells = (int)s->cpr.cluster_cells;
  }
  PF_CUDA(cudaGetLastError());
  PF_CUDA(cudaStreamSynchronize(st));
  s->tune = t;
  s->cpr.block_rbgs0 = t.rbgs;
  s->cpr.block_stage2 = t.stage2;
  if (t.block_cells > 0) s->cpr.block_cells = t.block_cells;
  if (t.cluster_cells >= 0) s->cpr.cluster_cells = t.cluster_cells;
  s->cpr.ilu_fused = t.ilu_fused;
  // captured graphs hold the old launch shapes
  for (auto& G : s->graphs) {
    if (G.pre) cudaGraphExecDestroy(G.pre);
    if (G.spmv) cudaGraphExecDestroy(G.spmv);
    if (G.ortho) cudaGraphExecDestroy(G.ortho);
  }
  s->graphs.clear();
  s->assembled = false;
  if (out) {
    out->props = t.props; out->face = t.face; out->gather = t.gather;
    out->spmv = t.spmv; out->stage2 = t.stage2; out->rbgs = t.rbgs;
    out->block_cells = (int)s->cpr.block_cells;
    out->cluster_cells = (int)s->cpr.cluster_cells;
    out->ilu_fused = t.ilu_fused;
  }
  return PF_OK;
}

pf_status pf_get_tuning(const pf_sim* s, pf_tuning* t) {
  if (!s) return fail(PF_EINVAL, "pf_sim is NULL");
  if (!t) return fail(PF_EINVAL, "tuning is NULL");
  const Tuning& u = s->tune;
  t->props = u.props; t->face = u.face; t->gather = u.gather;
  t->spmv = u.spmv; t->stage2 = u.stage2; t->rbgs = u.rbgs;
  t->block_cells = (int)s->cpr.block_cells;
  t->cluster_cells = (int)s->cpr.cluster_cells;
  t->ilu_fused = s->cpr.ilu_fused;
  return PF_OK;
}

pf_status pf_set_tuning(pf_sim* s, const pf_tuning* t) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!t) return fail(PF_EINVAL, "tuning is NULL");
  auto ok = [](int b) { return b >= 32 && b <= 256 && b % 32 == 0; };
  const bool spmv_ok = ok(t->spmv) || (!s->mixed && (t->spmv == -96 || t->spmv == -192 || t->spmv == -384));
  if (!ok(t->props) || !ok(t->face) || !ok(t->gather) || !spmv_ok || !ok(t->stage2) || !ok(t->rbgs) ||
      t->block_cells < 1 || t->block_cells > 65536 || (t->ilu_fused != 0 && t->ilu_fused != 1) ||
      t->cluster_cells < 0 || t->cluster_cells > 16384)
    return fail(PF_EINVAL, "invalid launch shape");
  PF_CUDA(cudaStreamSynchronize(s->stream));
  Tuning& u = s->tune;
  u.props = t->props; u.face = t->face; u.gather = t->gather;
  u.spmv = t->spmv; u.stage2 = t->stage2; u.rbgs = t->rbgs;
  u.block_cells = t->block_cells;
  u.cluster_cells = t->cluster_cells;
  s->cpr.cluster_cells = t->cluster_cells;
  u.ilu_fused = t->ilu_fused;
  s->cpr.ilu_fused = t->ilu_fused;
  s->cpr.block_rbgs0 = u.rbgs;
  s->cpr.block_stage2 = u.stage2;
  s->cpr.block_cells = t->block_cells;
  for (auto& G : s->graphs) {
    if (G.pre) cudaGraphExecDestroy(G.pre);
    if (G.spmv) cudaGraphExecDestroy(G.spmv);
    if (G.ortho) cudaGraphExecDestroy(G.ortho);
  }
  s->graphs.clear();
  return PF_OK;
}

pf_status pf_get_x(pf_sim* s, double* x) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!x) return fail(PF_EINVAL, "x is NULL");
  PF_CUDA(cudaMemcpyAsync(x, s->x, s->nunk * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  return PF_OK;
}

pf_status pf_set_x(pf_sim* s, const double* x) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (!x) return fail(PF_EINVAL, "x is NULL");
  PF_CUDA(cudaMemcpyAsync(s->x, x, s->nunk * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  PF_CUDA(cudaStreamSynchronize(s->stream));
  s->assembled = false;
  return PF_OK;
}

pf_status pf_kernel_timing_enable(pf_sim* s, int on) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  kt_collect(s);
  s->kt_on = on != 0;
  for (int k = 0; k < PF_KT_COUNT; ++k) { s->kt_count[k] = 0; s->kt_ms[k] = 0.0; }
  return PF_OK;
}

pf_status pf_kernel_timing(pf_sim* s, int which, int64_t* launches, double* total_ms) {
  pf_status rc = check(s);
  if (rc != PF_OK) return rc;
  if (which < 0 || which >= PF_KT_COUNT) return fail(PF_EINVAL, "unknown kernel class");
  kt_collect(s);
  if (launches) *launches = s->kt_count[which];
  if (total_ms) *total_ms = s->kt_ms[which];
  return PF_OK;
}

pf_status pf_launch_count(const pf_sim* s, int64_t* count) {
  if (!s || !count) return fail(PF_EINVAL, "NULL argument");
  *count = s->launches;
  return PF_OK;
}

}  // extern "C"
