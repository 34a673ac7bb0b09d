"""Native time loop, batch engine and serving loop on the GPU.

* pf_run_schedule reproduces the oracle's time loop (1e-6 per step field).
* A scenario gives bit-identical states alone and as a member of a batch or
  of a server's mix (deterministic kernels; streams and host threads do not
  enter the arithmetic).
* The server never holds more device memory than its budget and refuses a
  request that can never fit with PF_EBUSY.
"""

import time

import numpy as np
import pytest

from oracle import model as M
from scenarios import generate as G

pytestmark = pytest.mark.gpu

DAY = G.DAY


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    from paper_1807_05298_gb300 import build as bld
    bld.build()
    from paper_1807_05298_gb300 import binding
    binding.lib()
    return binding


def small_members(k, n_steps=3):
    out = []
    for i in range(k):
        nx = 12 + 5 * i
        sc = G.scenario_c2(seed=200 + i, nx=nx, ny=nx + 3, nz=3 + (i % 3), n_steps=n_steps, slug_steps=2,
                           c_slug=0.5 + 0.3 * i, rrf=1.2 + 0.1 * i, dt_days=2.0)
        out.append(sc)
    return out


def alone(B, sc, n_steps, **opt):
    sim = B.Simulator(sc, **opt)
    B.run_schedule(sim, B.Schedule(sc["schedule"], n_steps))
    x = sim.get_x()
    sim.close()
    return x


def test_native_time_loop_matches_oracle(B):
    sc = G.scenario_c1(n_steps=10)
    sim = B.Simulator(sc, precond=B.PF_PC_CPR, use_forcing=1)
    rep = B.run_schedule(sim, B.Schedule(sc["schedule"]))
    x = sim.get_x()
    sim.close()
    st, xo, hist = M.run(sc)
    assert rep.steps == 10 and rep.status == 0
    n = st.n
    for a in range(3):
        ref = max(np.abs(xo[a:3 * n:3]).max(), 1e-12)
        assert np.abs(x[a:3 * n:3] - xo[a:3 * n:3]).max() <= 1e-6 * ref


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_members_equal_alone(B, precision):
    scs = small_members(5)
    opt = dict(precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=precision)
    batch = B.Batch(scs, n_threads=4, **opt)
    reps = batch.run(n_steps=3)
    assert all(r.status == 0 and r.steps == 3 for r in reps)
    xs = [batch.member_x(i) for i in range(len(scs))]
    batch.close()
    for sc, xb in zip(scs, xs):
        xa = alone(B, sc, 3, **opt)
        assert np.array_equal(xa, xb)


@pytest.mark.parametrize("precision,window_us", [(0, 0.0), (1, 0.0), (1, 2000.0)])
def test_packed_batch_members_equal_alone(B, precision, window_us):
    """Packed assembly (one launch per assembly kernel over the members that
    reach an assembly together): every member's final state is bit-identical
    to its own run alone, with no waiting window and with a window long enough
    that the members inside the run meet at their assemblies; the packs did
    take several members at once."""
    scs = small_members(5)
    opt = dict(precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=precision)
    batch = B.Batch(scs, n_threads=4, packed=True, pack_window_us=window_us, **opt)
    reps = batch.run(n_steps=3)
    assert all(r.status == 0 and r.steps == 3 for r in reps)
    packs, members = batch.packing_stats()
    xs = [batch.member_x(i) for i in range(len(scs))]
    batch.close()
    assert packs >= 1 and members >= packs
    if window_us > 0.0:
        assert members > packs          # some packs held more than one member
    for sc, xb in zip(scs, xs):
        xa = alone(B, sc, 3, **opt)
        assert np.array_equal(xa, xb)


def test_packing_turned_off_between_runs(B):
    """Two batch runs, the first packed and the second with packing turned
    off (the members' own launches again): each member ends where the same
    two runs of it alone end, bit for bit, and the stats reset."""
    scs = small_members(3)
    opt = dict(precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=B.PF_PREC_MIXED)
    batch = B.Batch(scs, n_threads=3, packed=True, pack_window_us=5000.0, **opt)
    with pytest.raises(B.PfError):
        batch.set_packing(True, -1.0)             # a negative window is rejected (packing stays as it was)
    batch.set_packing(True, 5000.0)               # turning it on again replaces the packer
    assert all(r.status == 0 for r in batch.run(n_steps=2))
    assert batch.packing_stats()[0] >= 1
    batch.set_packing(False)
    assert batch.packing_stats() == (0, 0)
    assert all(r.status == 0 for r in batch.run(n_steps=2))
    xs = [batch.member_x(i) for i in range(len(scs))]
    batch.close()
    for sc, xb in zip(scs, xs):
        sim = B.Simulator(sc, **opt)
        for _ in range(2):
            B.run_schedule(sim, B.Schedule(sc["schedule"], 2))
        xa = sim.get_x()
        sim.close()
        assert np.array_equal(xa, xb)


def test_server_same_alone_and_in_mix_and_admission(B):
    scs = small_members(6, n_steps=2)
    opt = dict(precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=B.PF_PREC_MIXED)
    fps = [B.footprint(sc, precond=B.PF_PC_CPR, precision=B.PF_PREC_MIXED) for sc in scs]
    budget = int(sorted(fps)[-1] + sorted(fps)[-2])   # at most about two requests resident
    srv = B.Server(budget, n_workers=4, **opt)
    tickets = []
    peak = 0
    for sc in scs:
        tickets.append(srv.submit(sc, n_steps=2))
        peak = max(peak, srv.stats()[0])
    done = False
    t0 = time.time()
    while not done and time.time() - t0 < 300:
        used, running, queued = srv.stats()
        peak = max(peak, used)
        done = all(srv.poll(t).state in (B.PF_REQ_DONE, B.PF_REQ_FAILED) for t in tickets)
        time.sleep(0.001)
    assert done
    assert peak <= budget
    results = [srv.wait(t) for t in tickets]
    assert all(r.state == B.PF_REQ_DONE and r.report.steps == 2 for r in results)
    assert all(r.t_end >= r.t_start >= r.t_submit for r in results)
    for sc, t in zip(scs, tickets):
        P, S, C, Pb = srv.state(t)
        xa = alone(B, sc, 2, **opt)
        n = sc["nx"] * sc["ny"] * sc["nz"]
        assert np.array_equal(P, xa[0:3 * n:3]) and np.array_equal(S, xa[1:3 * n:3])
        assert np.array_equal(C, xa[2:3 * n:3]) and np.array_equal(Pb, xa[3 * n:])
    big = G.scenario_c2(nx=60, ny=60, nz=10)
    with pytest.raises(B.PfError) as e:
        srv.submit(big)
    assert e.value.status == B.PF_EBUSY
    srv.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_launch_shapes_give_identical_results(B, precision):
    sc = G.scenario_c1(nx=17, ny=11, nz=3, n_steps=3)
    opt = dict(precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=precision)
    base = alone(B, sc, 3, **opt)
    sim = B.Simulator(sc, autotune=1, **opt)
    t = sim.autotune()
    assert sim.tuning() == t
    assert all(v in (64, 128, 256) for k, v in t.items()
               if k not in ("spmv", "block_cells", "ilu_fused", "cluster_cells"))
    assert t["ilu_fused"] in (0, 1)
    assert t["spmv"] in ((64, 128, 256, -96, -192, -384) if precision == 0 else (64, 128, 256))
    assert t["block_cells"] == (512 if precision == 0 else 4096)
    B.run_schedule(sim, B.Schedule(sc["schedule"], 3))
    x = sim.get_x()
    sim.close()
    assert np.array_equal(base, x)


def test_native_time_loop_cuts_and_grows_like_oracle(B):
    """A 30-day step with at most 6 Newton iterations fails and is cut; the
    native loop cuts, grows the step back and lands on the oracle's state."""
    sc = G.scenario_c1(n_steps=2, dt_days=30.0)
    sim = B.Simulator(sc, precond=B.PF_PC_CPR, use_forcing=0, lin_rtol=1e-12, newton_max_iter=6)
    rep = B.run_schedule(sim, B.Schedule(sc["schedule"]))
    x = sim.get_x()
    sim.close()
    st, xo, hist = M.run(sc, max_iter=6)
    assert rep.status == 0 and rep.steps == 2
    assert rep.cuts == sum(h["cuts"] for h in hist)
    n = st.n
    for a in range(3):
        ref = max(np.abs(xo[a:3 * n:3]).max(), 1e-12)
        assert np.abs(x[a:3 * n:3] - xo[a:3 * n:3]).max() <= 1e-6 * ref


@pytest.mark.parametrize("shape", [-96, -192, -384])
def test_row_split_spmv_gives_identical_results(B, shape):
    """One thread per block row (FP64 SpMV) against one thread per cell: the
    product and a whole 3-step run are bit-identical; shapes outside the
    documented set are refused."""
    sc = G.scenario_c1(nx=17, ny=11, nz=3, n_steps=3)
    opt = dict(precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=0)
    base = alone(B, sc, 3, **opt)
    ref = B.Simulator(sc, **opt)
    sim = B.Simulator(sc, **opt)
    sim.set_tuning(spmv=shape)
    v = np.random.default_rng(3).standard_normal(ref.nunk)
    ref.set_controls(sc["schedule"][0]["controls"])
    sim.set_controls(sc["schedule"][0]["controls"])
    ref.begin_step(DAY)
    sim.begin_step(DAY)
    ref.assemble()
    sim.assemble()
    assert np.array_equal(ref.apply_jacobian(v), sim.apply_jacobian(v))
    ref.close()
    sim.close()
    sim = B.Simulator(sc, **opt)
    # also every multigrid level in one block, and the ILU(0) solve in three launches
    sim.set_tuning(spmv=shape, block_cells=2048, ilu_fused=0)
    B.run_schedule(sim, B.Schedule(sc["schedule"], 3))
    assert np.array_equal(base, sim.get_x())
    with pytest.raises(B.PfError) as e:
        sim.set_tuning(spmv=-100)
    assert e.value.status == B.PF_EINVAL
    sim.close()
    mixed = B.Simulator(sc, **dict(opt, precision=1))
    with pytest.raises(B.PfError):
        mixed.set_tuning(spmv=shape)
    mixed.close()


def test_programmatic_launch_gives_identical_results(B):
    """Kernels launched with programmatic dependent launch wait for their
    predecessor before reading, so a run is bit-identical with the launch
    attribute on and off (FP64 and mixed precision, CPR + ILU(0))."""
    sc = G.scenario_c1(nx=13, ny=9, nz=3, n_steps=3)
    for precision in (0, 1):
        opt = dict(precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=precision)
        off = alone(B, sc, 3, **opt)
        try:
            B.set_programmatic_launch(True)
            on = alone(B, sc, 3, **opt)
        finally:
            B.set_programmatic_launch(False)
        assert np.array_equal(off, on)


@pytest.mark.parametrize("precision", [0, 1])
def test_cluster_cycle_gives_identical_results(B, precision):
    """The multigrid levels run by one thread-block cluster (cluster barriers
    between phases) round exactly like the per-level kernels: a run is
    bit-identical with the cluster path on and off."""
    sc = G.scenario_c1(nx=40, ny=36, nz=6, n_steps=2)        # finest 8640 cells, next 1080
    opt = dict(precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=precision)
    base = B.Simulator(sc, **opt)
    base.set_tuning(block_cells=64, cluster_cells=0)
    B.run_schedule(base, B.Schedule(sc["schedule"], 2))
    xb = base.get_x()
    base.close()
    for cells in (2048, 16384):
        sim = B.Simulator(sc, **opt)
        sim.set_tuning(block_cells=64, cluster_cells=cells)
        B.run_schedule(sim, B.Schedule(sc["schedule"], 2))
        assert np.array_equal(sim.get_x(), xb)
        sim.close()


def test_runaway_step_fails_early_and_restores_the_state(B):
    """The library's divergence test: with near-exact linear solves (the
    oracle's Newton path) a 30000-day first step runs away, so the step
    fails with PF_ENOT_CONVERGED before the Newton cap and the state is
    restored; with the test off it fails only at the cap."""
    dt = 30000.0 * DAY
    sc = G.scenario_c1(n_steps=1, dt_days=30000.0)
    ctl = sc["schedule"][0]["controls"]
    its = {}
    for div in (1e6, 0.0):
        sim = B.Simulator(sc, precond=B.PF_PC_CPR, use_forcing=0, lin_rtol=1e-12, gmres_max_iter=600,
                          newton_div=div)
        sim.set_controls(ctl)
        x0 = sim.get_x()
        rc, rep = sim.step(dt, raise_on_failure=False)
        assert rc == B.PF_ENOT_CONVERGED
        assert np.array_equal(sim.get_x(), x0)
        sim.begin_step(dt)
        n = 0
        while True:
            try:
                r = sim.newton_iteration()
            except B.PfError as e:
                assert e.status == B.PF_ENOT_CONVERGED
                break
            assert not r.converged
            n += 1
        sim.abort_step()
        its[div] = n
        sim.close()
    assert its[1e6] < its[0.0] and its[1e6] < 25


@pytest.mark.parametrize("precision", [0, 1])
def test_krylov_lookahead_gives_identical_results(B, precision):
    """Arnoldi step j + 1 enqueued before the host reads step j (and left
    unused when step j meets the tolerance) changes no result: the same
    states, Newton and Krylov counts bit for bit, with a launch count at
    least as large (the unused steps ran)."""
    sc = G.scenario_c1(nx=17, ny=11, nz=3, n_steps=4)
    out = []
    for look in (0, 1):
        sim = B.Simulator(sc, precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=precision,
                          krylov_lookahead=look)
        l0 = sim.launch_count()
        rep = B.run_schedule(sim, B.Schedule(sc["schedule"], 4))
        out.append((sim.get_x(), (rep.newton_iters, rep.krylov_iters, rep.cuts), sim.launch_count() - l0))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    assert out[1][2] >= out[0][2]


@pytest.mark.parametrize("precision,shape", [(0, (17, 13, 4)), (1, (24, 18, 12))])
def test_per_colour_copies_give_identical_results(B, precision, shape):
    """ilu_store = 1: the ILU(0) sweeps, stage 2 and the finest multigrid
    smoother read per-colour copies of their blocks and stencil (grids above
    the single-block size, so the finest level runs as separate passes), and
    the black sweep goes through the set-up's products J_bj D_j^-1 (another
    rounding order of the same ILU(0) solve): against the natural layout a
    3-step run has the same cuts, Newton and Krylov totals within one
    iteration and 5%, and states equal far inside the oracle's 1e-6
    tolerance."""
    nx, ny, nz = shape
    sc = G.scenario_c1(nx=nx, ny=ny, nz=nz, n_steps=3)
    outs = []
    for store in (0, 1):
        sim = B.Simulator(sc, precond=B.PF_PC_CPR, use_forcing=1, newton_tol=1e-8, precision=precision,
                          ilu_store=store)
        rep = B.run_schedule(sim, B.Schedule(sc["schedule"], 3))
        outs.append((sim.get_x(), (rep.newton_iters, rep.krylov_iters, rep.cuts)))
        sim.close()
    (x0, (n0, k0, c0)), (x1, (n1, k1, c1)) = outs
    assert c0 == c1 and abs(n0 - n1) <= 1
    assert abs(k0 - k1) <= max(2, 0.05 * k0)
    n = nx * ny * nz
    for a in range(3):
        ref = max(np.abs(x0[a:3 * n:3]).max(), 1e-12)
        assert np.abs(x0[a:3 * n:3] - x1[a:3 * n:3]).max() <= 1e-7 * ref


def test_create_failure_paths_free_everything(B):
    """Failure detection on the host (no GPU fault): the fault-injection hook
    makes each CUDA call of pf_create fail in turn, from the device arena's
    allocation through the uploads to the closing synchronisation.  Every
    failure reports its status (PF_ENOMEM for the two allocations, PF_ECUDA
    after them) with the failed call in the message, leaves no device memory
    behind, and a pf_create that follows still works and steps."""
    import torch
    sc = G.scenario_c2(seed=7, nx=64, ny=64, nz=16, n_steps=1)
    arena = B.footprint(sc)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    statuses = []
    for k in range(1, 200):
        B.inject_create_failure(k)
        try:
            sim = B.Simulator(sc, stream=B.current_stream_handle(), autotune=0)
        except B.PfError as e:
            statuses.append(e.status)
            msg = str(e)
            assert "device arena" in msg if k == 1 else "pf_create: cuda" in msg, msg
            torch.cuda.synchronize()
            free, _ = torch.cuda.mem_get_info()
            assert free0 - free < arena // 4, (k, free0 - free, arena)
            continue
        # k is past the last guarded call: the hook did not fire and is disarmed
        sim.close()
        break
    assert statuses[:2] == [B.PF_ENOMEM, B.PF_ENOMEM]
    assert len(statuses) >= 12 and all(s == B.PF_ECUDA for s in statuses[2:]), statuses
    B.inject_create_failure(0)
    sim = B.Simulator(sc, stream=B.current_stream_handle(), autotune=0)
    sim.set_controls(sc["schedule"][0]["controls"])
    rc, rep = sim.step(sc["schedule"][0]["dt"], raise_on_failure=False)
    assert rc == B.PF_OK and rep.newton_iters > 0
    sim.close()
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    assert free0 - free < arena // 4
