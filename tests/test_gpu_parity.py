"""GPU path versus the FP64 oracle, through the C ABI (needs a GB300).

Assembly (R and every Jacobian entry), SpMV, the preconditioned Krylov solve
and whole time steps are compared element by element with the oracle on the
same seeded inputs; grids span several 256-thread tiles with a ragged tail,
plus the degenerate shapes.  Tolerances:
  * R and J at one state: 1e-11 relative to the row scale (FP64 rounding of
    different but equivalent evaluation orders; both sides are FP64);
  * per-timestep P, S, C: 1e-6 relative to the field's maximum (the oracle's
    Newton tolerance is 1e-10 in scaled residual units).
"""

import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import model as M
from scenarios import generate as G
from gpu_helpers import (gpu_system_to_csr, perforated_cells, rb_block_ilu0_apply, rel_matrix_error,
                         window_around, window_state)

pytestmark = pytest.mark.gpu

DAY, BAR = G.DAY, G.BAR


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


def ragged_scenario(nx=23, ny=13, nz=5, physics=None, seed=4):
    sc = G.scenario_c1(seed=seed, nx=nx, ny=ny, nz=nz)
    if physics is not None:
        sc["physics"] = physics
    n = nx * ny * nz
    col = lambda i, j, k0, k1: [i + nx * (j + ny * k) for k in range(k0, k1)]
    wells = [dict(kind="inj", cells=col(0, 0, 0, min(3, nz))),
             dict(kind="prod", cells=col(nx - 1, ny - 1, 0, nz)),
             dict(kind="prod", cells=col(nx // 2, ny // 2, max(0, nz - 2), nz))]
    for w in wells:
        w.update(rw=0.1, skin=0.0, gf=0.249, f=1.0, fh=1.0, dirs=["z"] * len(w["cells"]))
        w["cells"] = np.asarray(w["cells"], dtype=np.int64)
        w["Pb0"] = float(sc["P0"][w["cells"][0]])
    sc["wells"] = wells
    ctl = [dict(ctrl="wrate", target=60.0 / DAY, limit=None, c_inj=1.2),
           dict(ctrl="bhp", target=150.0 * BAR, limit=None, c_inj=0.0),
           dict(ctrl="lrate", target=20.0 / DAY, limit=None, c_inj=0.0)]
    sc["schedule"] = [dict(n_steps=5, dt=2.0 * DAY, controls=ctl)]
    return sc, ctl


def random_state(st, rng, x0):
    x = x0.copy()
    n = st.n
    x[0:3 * n:3] += rng.normal(0.0, 2.0 * BAR, n)
    x[1:3 * n:3] = rng.uniform(0.22, 0.78, n)
    x[2:3 * n:3] = rng.uniform(0.0, 1.6, n)
    x[3 * n:] += rng.normal(0.0, 5.0 * BAR, st.nw)
    return x


def assemble_both(B, sc, ctl, x_old, x, dt, **opt):
    st = M.Setup(sc)
    gam = M.well_gamma(st, x_old, ctl)
    R_o, J_o = M.assemble(st, x, M.masses(st, x_old), dt, ctl, gam)
    sim = B.Simulator(sc, stream=B.current_stream_handle(), **opt)
    sim.set_controls(ctl)
    sim.set_x(x_old)
    sim.begin_step(dt)
    sim.set_x(x)
    sim.assemble()
    R_g, Jc, Bw, Cw, Dw = sim.export_system()
    J_g = gpu_system_to_csr(sc, Jc, Bw, Cw, Dw, [w["cells"] for w in sc["wells"]])
    return st, sim, R_o, J_o, R_g, J_g


def residual_error(st, R_g, R_o, dt, ctl):
    n = st.n
    pv = st.V * st.phi_r
    ph = st.ph
    err = 0.0
    for a, ref in enumerate((ph["rho_o"], ph["rho_w"], ph["c_ref"])):
        err = max(err, float(np.max(np.abs(R_g[a:3 * n:3] - R_o[a:3 * n:3]) / (pv * ref))))
    for w in range(st.nw):
        scale = abs(R_o[3 * n + w]) + dt * st.wells[w]["W"] * BAR
        err = max(err, abs(R_g[3 * n + w] - R_o[3 * n + w]) / scale)
    return err


PHYS_VARIANTS = [
    G.default_physics(),
    G.default_physics(omega=0.6, pc_e=0.4 * BAR, mixing=1, ads_a=0.8, ads_b=4.0, rrf=2.3, ipv=0.15),
    G.default_physics(omega=0.3, nw=2.5, no=1.7, c_r=0.0, krw_max=0.6, kro_max=0.9),
    # tabulated k_rw, k_ro, P_c (Sec. 2.2) and A_d, viscosity multiplier (Sec. 2.3)
    G.default_physics(omega=0.7, rrf=1.9,
                      sat_table=np.array([[0.1, 0.0, 1.0, 0.9 * BAR], [0.25, 0.02, 0.7, 0.5 * BAR],
                                          [0.4, 0.1, 0.4, 0.3 * BAR], [0.6, 0.3, 0.12, 0.12 * BAR],
                                          [0.85, 0.8, 0.0, 0.01 * BAR]]),
                      poly_table=np.array([[0.0, 1.0, 0.0], [0.3, 1.8, 0.02], [1.0, 3.5, 0.05],
                                           [2.5, 6.0, 0.065]])),
]


@pytest.mark.parametrize("pi", range(len(PHYS_VARIANTS)))
def test_assembly_matches_oracle(B, pi):
    sc, ctl = ragged_scenario(physics=PHYS_VARIANTS[pi])
    st = M.Setup(sc)
    rng = np.random.default_rng(10 + pi)
    x0 = M.initial_state(st)
    x_old, x = random_state(st, rng, x0), random_state(st, rng, x0)
    dt = 3.0 * DAY
    st, sim, R_o, J_o, R_g, J_g = assemble_both(B, sc, ctl, x_old, x, dt)
    assert residual_error(st, R_g, R_o, dt, ctl) <= 1e-11
    assert rel_matrix_error(J_g, J_o) <= 1e-11
    # the oil row's polymer column of every block is exactly zero (the block
    # products skip it; the oracle pins the same structure)
    Jc = sim.export_system()[1]          # [slot][entry][cell]; entry 2 = oil row, polymer column
    assert not np.any(Jc[:, 2, :])
    # SpMV with the assembled Jacobian
    v = rng.normal(size=st.nunk) * np.tile([1e5, 0.1, 0.5], st.n + 1)[:st.nunk]
    y_g = sim.apply_jacobian(v)
    y_o = J_o @ v
    bound = abs(J_o) @ np.abs(v)
    assert np.all(np.abs(y_g - y_o) <= 1e-12 * bound + 1e-300)
    sim.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 6), (7, 1, 1), (1, 5, 3), (2, 2, 2), (33, 9, 1)])
def test_assembly_degenerate_grids(B, shape):
    nx, ny, nz = shape
    sc = G.scenario_c1(nx=nx, ny=ny, nz=nz)
    n = nx * ny * nz
    if n == 1:
        sc["wells"] = []
        ctl = []
    else:
        sc["wells"] = [dict(kind="inj", cells=np.array([0], dtype=np.int64), dirs=["z"], rw=0.1, skin=0.0,
                            gf=0.249, f=1.0, fh=1.0, Pb0=210 * BAR),
                       dict(kind="prod", cells=np.array([n - 1], dtype=np.int64), dirs=["x"], rw=0.1, skin=1.0,
                            gf=0.249, f=1.0, fh=1.0, Pb0=190 * BAR)]
        ctl = [dict(ctrl="wrate", target=10.0 / DAY, limit=None, c_inj=0.5),
               dict(ctrl="bhp", target=180 * BAR, limit=None, c_inj=0.0)]
    st = M.Setup(sc)
    rng = np.random.default_rng(sum(shape))
    x0 = M.initial_state(st)
    x_old, x = random_state(st, rng, x0), random_state(st, rng, x0)
    st, sim, R_o, J_o, R_g, J_g = assemble_both(B, sc, ctl, x_old, x, DAY)
    assert residual_error(st, R_g, R_o, DAY, ctl) <= 1e-11
    assert rel_matrix_error(J_g, J_o) <= 1e-11
    sim.close()


@pytest.mark.parametrize("precond,cycle,stage1,sweeps", [("bjacobi", 1, 0, 1), ("cpr", 1, 0, 1), ("cpr", 2, 0, 1),
                                                          ("bjacobi", 1, 1, 1), ("cpr", 1, 1, 1), ("cpr", 1, 1, 0)])
def test_linear_solve_matches_direct(B, precond, cycle, stage1, sweeps):
    """GMRES with each preconditioner against a direct solve of the oracle's
    system; sweeps = 0: no pre-smoothing on any multigrid level (the levels
    start from the zero initial guess) and no post-smoothing below the finest."""
    sc, ctl = ragged_scenario(nx=17, ny=9, nz=4)
    st = M.Setup(sc)
    rng = np.random.default_rng(3)
    x0 = M.initial_state(st)
    x_old = random_state(st, rng, x0)
    x = x_old + 0.0
    x[0:3 * st.n:3] += rng.normal(0.0, 0.5 * BAR, st.n)
    dt = 0.5 * DAY
    pc = B.PF_PC_CPR if precond == "cpr" else B.PF_PC_BJACOBI
    sw = {} if sweeps else dict(amg_pre_sweeps=0, amg_coarse_sweeps=0)
    st, sim, R_o, J_o, R_g, J_g = assemble_both(B, sc, ctl, x_old, x, dt, gmres_max_iter=2000, precond=pc,
                                                amg_cycle=cycle, stage1=stage1, **sw)
    b = -R_o
    xg, its, rr = sim.solve_linear(b, 1e-12)
    xo = spla.spsolve(J_o.tocsc(), b)
    assert rr <= 1e-12
    assert np.linalg.norm(J_o @ xg - b) <= 1e-10 * np.linalg.norm(b)
    n = st.n
    for a in range(3):
        ref = np.abs(xo[a:3 * n:3]).max()
        assert np.abs(xg[a:3 * n:3] - xo[a:3 * n:3]).max() <= 1e-6 * ref + 1e-300
    sim.close()


@pytest.mark.parametrize("eta,restart", [(0.0, 30), (1.0, 30), (0.2, 5)])
def test_gram_schmidt_variants_match_direct(B, eta, restart):
    """The Arnoldi step's Gram-Schmidt under each reorthogonalisation rule:
    eta = 0 keeps one classical pass (the second only where the projected
    norm, taken by Pythagoras from the first pass's dots, is not positive),
    eta = 1 always takes the second pass with its measured norm, and the
    default 0.2 with a short restart (every cycle restarts from the true
    residual).  Each solve must reach the direct solution of the oracle's
    system (FP64: the mixed form solves with its FP32 operator)."""
    sc, ctl = ragged_scenario(nx=17, ny=9, nz=4)
    st = M.Setup(sc)
    rng = np.random.default_rng(5)
    x_old = random_state(st, rng, M.initial_state(st))
    x = x_old + 0.0
    x[0:3 * st.n:3] += rng.normal(0.0, 0.5 * BAR, st.n)
    dt = 0.5 * DAY
    st, sim, R_o, J_o, R_g, J_g = assemble_both(B, sc, ctl, x_old, x, dt, gmres_max_iter=2000, precond=B.PF_PC_CPR,
                                                reorth_eta=eta, gmres_restart=restart)
    b = -R_o
    xg, its, rr = sim.solve_linear(b, 1e-12)
    xo = spla.spsolve(J_o.tocsc(), b)
    assert rr <= 1e-12
    assert np.linalg.norm(J_o @ xg - b) <= 1e-10 * np.linalg.norm(b)
    n = st.n
    for a in range(3):
        ref = np.abs(xo[a:3 * n:3]).max()
        assert np.abs(xg[a:3 * n:3] - xo[a:3 * n:3]).max() <= 1e-6 * ref + 1e-300
    sim.close()


def field_errors(n, x_g, x_o):
    out = []
    for a in range(3):
        ref = max(np.abs(x_o[a:3 * n:3]).max(), 1e-12)
        out.append(float(np.abs(x_g[a:3 * n:3] - x_o[a:3 * n:3]).max() / ref))
    return out


def run_both(B, sc, n_steps, **opt):
    sim = B.Simulator(sc, stream=B.current_stream_handle(), **opt)
    states = []
    sim.run_schedule(n_steps=n_steps, callback=lambda s, rec: states.append(s.get_x()))
    st, _, hist = M.run(sc, n_steps=n_steps)
    sim.close()
    return st, states, hist


def test_timesteps_match_oracle_c1(B):
    """The 10x10x3 workload, all 30 daily steps: P, S, C per step to 1e-6."""
    sc = G.scenario_c1()
    st, states, hist = run_both(B, sc, 30)
    assert len(states) == len(hist) == 30
    worst = [0.0, 0.0, 0.0]
    for xg, h in zip(states, hist):
        errs = field_errors(st.n, xg, h["x"])
        worst = [max(a, b) for a, b in zip(worst, errs)]
    assert max(worst) <= 1e-6, worst


def test_timesteps_match_oracle_c1_cpr(B):
    """Same root under the CPR preconditioner and the inexact-Newton forcing
    term (Sec. 3.3): the Newton tolerance decides, not the linear path."""
    sc = G.scenario_c1()
    st, states, hist = run_both(B, sc, 30, precond=B.PF_PC_CPR, use_forcing=1)
    for xg, h in zip(states, hist):
        assert max(field_errors(st.n, xg, h["x"])) <= 1e-6


def test_timesteps_match_oracle_ragged_mixed_precision(B):
    """FP32 Jacobian and preconditioner, FP64 residual: the root is the same."""
    sc, _ = ragged_scenario(nx=19, ny=11, nz=3)
    st, states, hist = run_both(B, sc, 4, precision=B.PF_PREC_MIXED, precond=B.PF_PC_CPR)
    for xg, h in zip(states, hist):
        assert max(field_errors(st.n, xg, h["x"])) <= 1e-6


def test_step_failure_restores_state(B):
    """A Newton cap of one iteration cannot converge a rate-driven step: the
    library reports PF_ENOT_CONVERGED and restores x^n bit for bit."""
    sc = G.scenario_c1(nx=6, ny=6, nz=2)
    sim = B.Simulator(sc, stream=B.current_stream_handle(), newton_max_iter=1)
    sim.set_controls(sc["schedule"][0]["controls"])
    x0 = sim.get_x()
    rc, rep = sim.step(DAY, raise_on_failure=False)
    assert rc == B.PF_ENOT_CONVERGED
    assert np.array_equal(sim.get_x(), x0)
    sim.close()


def test_full_size_100k_root_is_oracle_root(B):
    """100x100x10 (100,000 cells) under the benchmark's solver settings (CPR,
    forcing term): past the start-up transient, one GPU time step lands on a
    root of the oracle's own equations (oracle residual at the GPU state below
    the Newton tolerance), and a GPU assembly at that state matches the
    oracle's R and J entry by entry."""
    sc = G.scenario_c2()
    tol = 1e-8
    sim = B.Simulator(sc, stream=B.current_stream_handle(), use_forcing=1, newton_tol=tol,
                      precond=B.PF_PC_CPR)
    sim.run_schedule(n_steps=2)
    x_old = sim.get_x()
    dt = sc["schedule"][0]["dt"]
    rc, rep = sim.step(dt)
    # the last solve of the step ran under the switch state the step ended with
    ctl = [dict(c) for c in sc["schedule"][0]["controls"]]
    for w, sw in enumerate(sim.switched()):
        if sw:
            ctl[w] = dict(ctl[w], ctrl="bhp", target=ctl[w]["limit"])
    x = sim.get_x()
    st = M.Setup(sc)
    gam = M.well_gamma(st, x_old, ctl)
    R_o, J_o = M.assemble(st, x, M.masses(st, x_old), dt, ctl, gam)
    assert M.scaled_residual(st, R_o, dt, ctl) <= tol * 1.01
    sim.set_controls(ctl)
    sim.set_x(x_old)
    sim.begin_step(dt)
    sim.set_x(x)
    sim.assemble()
    R_g, Jc, Bw, Cw, Dw = sim.export_system()
    J_g = gpu_system_to_csr(sc, Jc, Bw, Cw, Dw, [w["cells"] for w in sc["wells"]])
    assert residual_error(st, R_g, R_o, dt, ctl) <= 1e-11
    assert rel_matrix_error(J_g, J_o) <= 1e-11
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c2_trajectory_matches_the_oracle_run(B, precision):
    """100x100x10 (100,000 cells, the 5-spot recipe with the polymer slug):
    the first three time steps of 10 days from the initial state, under the
    schedule's controls and BHP limits, against the oracle's own run of the
    same steps (tests/golden/c2_trajectory.json, written by
    make_c2_trajectory.py, which runs only oracle/): per step, P, S, C at the
    sampled cells to 1e-6 of each field's max-norm, every bottom-hole
    pressure to 1e-6 relative, the same number of step cuts and the same
    wells switched onto their BHP limits.  In both precisions: the mixed
    form's FP32 Jacobian and preconditioner change the Newton path, not the
    root its FP64 residual defines."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c2_trajectory.json")))
    sc = G.scenario_c2()
    prec = B.PF_PREC_MIXED if precision == "mixed" else B.PF_PREC_FP64
    sim = B.Simulator(sc, stream=B.current_stream_handle(), precond=B.PF_PC_CPR, use_forcing=0,
                      newton_tol=g["newton_tol"], precision=prec)
    states = []
    hist = sim.run_schedule(n_steps=g["n_steps"],
                            callback=lambda s, rec: states.append((s.get_x(), [bool(v) for v in s.switched()])))
    sim.close()
    cells = np.asarray(g["cells"])
    n = sc["nx"] * sc["ny"] * sc["nz"]
    assert len(states) == len(g["steps"])
    for (x, sw), rec, want in zip(states, hist, g["steps"]):
        for name, a in (("P", 0), ("S", 1), ("C", 2)):
            got = x[a:3 * n:3][cells]
            err = np.abs(got - np.asarray(want[name])).max() / want["max_abs"][name]
            assert err <= 1e-6, (name, err)
            assert abs(np.abs(x[a:3 * n:3]).max() - want["max_abs"][name]) <= 1e-6 * want["max_abs"][name]
        pb = np.asarray(want["Pb"])
        assert np.abs(x[3 * n:] - pb).max() <= 1e-6 * np.abs(pb).max()
        assert rec["cuts"] == want["cuts"]
        assert sw == want["switched"]


def sampled_window_check(B, sc, precision, seed, n_sample=48, layer_cells=0):
    """One GPU assembly of the full grid at a perturbed state; at n_sample
    seeded interior cells away from the wells (layer_cells of them next to a
    change of rock properties between layers), the FP64 residual and the
    action of the Jacobian (FP32 in mixed precision) on a random vector match
    the oracle, which assembles the 3x3x3 window around each cell (the window
    reproduces the full grid's rows of its centre: tests/test_window_oracle.py)."""
    import scipy.sparse as sp
    ctl = sc["schedule"][0]["controls"]
    dt = sc["schedule"][0]["dt"]
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    n = nx * ny * nz
    x_old = np.empty(3 * n + len(sc["wells"]))
    x_old[0:3 * n:3], x_old[1:3 * n:3], x_old[2:3 * n:3] = sc["P0"], sc["S0"], sc["C0"]
    x_old[3 * n:] = [w["Pb0"] for w in sc["wells"]]
    rng = np.random.default_rng(seed)
    x = x_old.copy()
    x[0:3 * n:3] += rng.normal(0.0, 2.0 * BAR, n)
    x[1:3 * n:3] = rng.uniform(0.22, 0.78, n)
    x[2:3 * n:3] = rng.uniform(0.0, 1.6, n)
    prec = B.PF_PREC_MIXED if precision == "mixed" else B.PF_PREC_FP64
    jv_tol = 3e-5 if precision == "mixed" else 1e-12  # FP32 Jacobian in mixed precision
    sim = B.Simulator(sc, stream=B.current_stream_handle(), precision=prec, precond=B.PF_PC_CPR)
    sim.set_controls(ctl)
    sim.set_x(x_old)
    sim.begin_step(dt)
    sim.set_x(x)
    sim.assemble()
    R_g = sim.export_residual()
    v = rng.standard_normal(sim.nunk) * np.concatenate([np.tile([1e5, 0.1, 0.5], n), np.full(len(sc["wells"]), 1e5)])  # P, S, C scales
    y_g = sim.apply_jacobian(v)
    sim.close()
    perf = perforated_cells(sc)
    kz = sc["kz"]
    cells = []
    while len(cells) < n_sample:
        i, j, k = int(rng.integers(1, nx - 1)), int(rng.integers(1, ny - 1)), int(rng.integers(1, nz - 1))
        c = i + nx * (j + ny * k)
        if len(cells) < layer_cells:       # a layer interface above or below c
            nxy = nx * ny
            if kz[c] == kz[c - nxy] and kz[c] == kz[c + nxy]:
                continue
        if c not in perf and c not in cells:
            cells.append(c)
    ph = sc["physics"]
    V = sc["dx"] * sc["dy"] * sc["dz"]
    for c in cells:
        w, idx = window_around(sc, c)
        stw = M.Setup(w)
        xw, xw_old = window_state(x, idx), window_state(x_old, idx)
        Rw, Jw = M.assemble(stw, xw, M.masses(stw, xw_old), dt, [], M.well_gamma(stw, xw_old, []))
        Jw = sp.csr_matrix(Jw)
        vw = window_state(v, idx)
        for a, ref in enumerate((ph["rho_o"], ph["rho_w"], ph["c_ref"])):
            scale = V * sc["phi"][c] * ref
            assert abs(R_g[3 * c + a] - Rw[3 * 13 + a]) <= 1e-11 * scale
            row = Jw[3 * 13 + a]
            yo = row @ vw
            mag = abs(row) @ np.abs(vw)
            assert abs(y_g[3 * c + a] - yo[0]) <= jv_tol * mag[0]
    return cells


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_27m_sampled_cells_match_the_oracle(B, precision):
    """600x450x100 (27M cells, 120 wells), in mixed precision and in FP64 as
    the benchmark runs them: 48 sampled cells against the oracle's windows."""
    sampled_window_check(B, G.scenario_c3(n_steps=3), precision, 27)


def step_lands_on_oracle_root(B, sc, seed):
    """One half-day time step from the initial state under the benchmark's
    solver settings (CPR, forcing term, Newton tolerance 1e-8 on the scaled
    residual), in mixed precision and in FP64.  At 48 sampled interior cells
    away from the wells the oracle's residual of the end state (assembled on
    the cell's 3x3x3 window, with the initial state as x^n) is within the
    Newton tolerance in the oracle's own scaled units, in both precisions; and
    the two end states agree to 1e-6 of each field's max-norm."""
    ctl = sc["schedule"][0]["controls"]
    dt = 0.5 * DAY
    tol = 1e-8
    ends = {}
    for precision in ("mixed", "fp64"):
        prec = B.PF_PREC_MIXED if precision == "mixed" else B.PF_PREC_FP64
        sim = B.Simulator(sc, stream=B.current_stream_handle(), precision=prec, precond=B.PF_PC_CPR, use_forcing=1,
                          newton_tol=tol)
        sim.set_controls(ctl)
        x_old = sim.get_x()
        rc, rep = sim.step(dt)
        assert rc == B.PF_OK and rep.converged
        ends[precision] = sim.get_x()
        sim.close()
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    n = nx * ny * nz
    for a in range(3):
        ref = np.abs(ends["fp64"][a:3 * n:3]).max()
        assert np.abs(ends["mixed"][a:3 * n:3] - ends["fp64"][a:3 * n:3]).max() <= 1e-6 * ref
    perf = perforated_cells(sc)
    rng = np.random.default_rng(seed)
    cells = []
    while len(cells) < 48:
        i, j, k = int(rng.integers(1, nx - 1)), int(rng.integers(1, ny - 1)), int(rng.integers(1, nz - 1))
        c = i + nx * (j + ny * k)
        if c not in perf and c not in cells:
            cells.append(c)
    ph = sc["physics"]
    V = sc["dx"] * sc["dy"] * sc["dz"]
    for precision, x in ends.items():
        worst = 0.0
        for c in cells:
            w, idx = window_around(sc, c)
            stw = M.Setup(w)
            xw, xw_old = window_state(x, idx), window_state(x_old, idx)
            Rw, _ = M.assemble(stw, xw, M.masses(stw, xw_old), dt, [], M.well_gamma(stw, xw_old, []),
                               with_jacobian=False)
            for a, ref in enumerate((ph["rho_o"], ph["rho_w"], ph["c_ref"])):
                worst = max(worst, abs(Rw[3 * 13 + a]) / (V * sc["phi"][c] * ref))
        assert worst <= 1.01 * tol, (precision, worst)


def test_full_size_27m_time_step_lands_on_the_oracle_root(B):
    """600x450x100 (27M cells, 120 wells): see step_lands_on_oracle_root."""
    step_lands_on_oracle_root(B, G.scenario_c3(n_steps=1), 2727)


def test_odd_rows_1m_time_step_lands_on_the_oracle_root(B):
    """201x105x50 (1,055,250 cells) of the channelised recipe: an odd number
    of colour slots per row (101) on the levels from 1M cells, whose smoother
    passes take two slots of a row per thread (the last thread of a row takes
    one), and per-colour copies with ragged rows; see
    step_lands_on_oracle_root."""
    step_lands_on_oracle_root(B, G.scenario_c3(nx=201, ny=105, nz=50, n_steps=1), 1055)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_paper_scale_sampled_cells_match_the_oracle(B, precision):
    """The paper's high-resolution grid, 951x1920x15 (27,388,800 cells, Sec.
    4.2.2) over the Table 4 layers each split in three (the benchmark's paper
    workload), in mixed precision and FP64: 48 sampled cells against the
    oracle's windows, 16 of them next to a change of layer properties."""
    sc = G.scenario_layered_table4(nx=951, ny=1920, refine_z=3, dt_days=1.0)
    cells = sampled_window_check(B, sc, precision, 44, layer_cells=16)
    assert len(cells) == 48


def test_bhp_limit_switching_matches_oracle(B):
    """A rate injector that hits its BHP limit: both sides switch it onto the
    limit in the same step and the states agree to 1e-6."""
    from test_oracle_pins import limited_injector_scenario
    sc = limited_injector_scenario(2000.0, 260.0, n_steps=5)
    sim = B.Simulator(sc, stream=B.current_stream_handle())
    states, flags = [], []

    def cb(s, rec):
        states.append(s.get_x())
        flags.append(bool(s.switched()[0]))

    sim.run_schedule(callback=cb)
    st, _, hist = M.run(sc)
    assert flags == [h["switched"][0] for h in hist]
    assert any(flags)
    for xg, h in zip(states, hist):
        assert max(field_errors(st.n, xg, h["x"])) <= 1e-6
    sim.close()


@pytest.mark.parametrize("form", [1, 2, 3])
def test_forcing_term_forms_match_oracle(B, form):
    """All three choices of the Sec. 3.3 forcing term (the third is the
    paper's and the library's default): the tolerance the library picks at
    each Newton iteration equals the oracle's formula evaluated on the
    iterates the library produced (for the first two, the previous linear
    residual rebuilt as b - J dx from the oracle's own R and J), and the step
    still lands on the oracle's root.  Polymer is present everywhere at the
    start so no update is clipped and dx is the difference of consecutive
    iterates."""
    sc = G.scenario_c1(nx=9, ny=7, nz=3)
    sc["C0"] = np.full(sc["C0"].shape, 0.5)
    dt = 2.0 * DAY
    ctl = M.controls_with_defaults(sc["schedule"][0]["controls"])
    sim = B.Simulator(sc, precond=B.PF_PC_CPR, use_forcing=1, forcing_form=form)
    sim.set_controls(sc["schedule"][0]["controls"])
    st = M.Setup(sc)
    x_old = sim.get_x()
    sim.begin_step(dt)
    xs, etas = [x_old], []
    for _ in range(12):
        rep = sim.newton_iteration()
        if rep.converged:
            break
        etas.append(rep.eta)
        xs.append(sim.get_x())
    assert rep.converged and len(etas) >= 3
    assert not any(sim.switched())
    sim.close()
    n = st.n
    gam = M.well_gamma(st, x_old, ctl)
    Mold = M.masses(st, x_old)
    assert etas[0] == 0.1
    for l in range(1, len(etas)):
        a, b = xs[l - 1], xs[l]
        assert np.abs(b[1:3 * n:3] - a[1:3 * n:3]).max() < 0.2 and b[2:3 * n:3].min() > 0.0
        assert 0.0 < b[1:3 * n:3].min() and b[1:3 * n:3].max() < 1.0
        R_a, J_a = M.assemble(st, a, Mold, dt, ctl, gam)
        R_b, _ = M.assemble(st, b, Mold, dt, ctl, gam)
        r_prev = -R_a - J_a @ (b - a)
        nb_prev = np.linalg.norm(R_a)
        if form == 1:
            want = M.forcing_term_difference(-R_b, r_prev, nb_prev)
        elif form == 2:
            want = M.forcing_term_norms(np.linalg.norm(R_b), np.linalg.norm(r_prev), nb_prev)
        else:
            want = M.forcing_term(np.linalg.norm(R_b), nb_prev)
        assert etas[l] == pytest.approx(want, rel=1e-6, abs=1e-12)
    x_o, ok, _ = M.newton_step(st, x_old, dt, ctl)
    assert ok
    err = field_errors(n, xs[-1], x_o)
    assert max(err) <= 1e-6


def test_equilibrium_state_is_a_rest_state_on_the_gpu(B):
    """Capillary-gravity equilibrium (Sec. 4.1.3) from the library's host
    initialiser, tabulated P_c: with no wells the GPU residual at that state
    vanishes and a time step leaves it unchanged (Newton converges before
    any update)."""
    sat = np.array([[0.2, 0.0, 1.0, 1.2 * BAR], [0.45, 0.08, 0.45, 0.35 * BAR], [0.8, 0.6, 0.0, 0.0],
                    [1.0, 1.0, 0.0, 0.0]])
    ph = G.default_physics(sat_table=sat)
    nx, ny, nz = 5, 4, 30
    n = nx * ny * nz
    phi = np.repeat(np.linspace(0.12, 0.3, nz), nx * ny)
    k = np.repeat(np.exp(np.linspace(np.log(20.0), np.log(500.0), nz)), nx * ny) * G.MD
    sched = [dict(n_steps=2, dt=10.0 * DAY, controls=[])]
    sc = G.make_scenario(nx, ny, nz, 20.0, 20.0, 1.0, 2000.0, k, k, 0.1 * k, phi, ph, [], sched)
    P, S = B.equilibrium_init(sc, 2005.0, 200.0 * BAR, 2022.0)
    sc["P0"], sc["S0"] = P, S
    st = M.Setup(sc)
    x0 = M.initial_state(st)
    sim = B.Simulator(sc, stream=B.current_stream_handle(), newton_tol=1e-10)
    sim.set_controls([])
    sim.begin_step(10.0 * DAY)
    sim.assemble()
    R_g = sim.export_system()[0]
    assert M.scaled_residual(st, R_g, 10.0 * DAY, []) < 1e-11
    sim.abort_step()
    rc, rep = sim.step(10.0 * DAY)
    assert rep.newton_iters == 0
    assert np.array_equal(sim.get_x(), x0)
    sim.close()


@pytest.mark.parametrize("shape", [(7, 5, 4), (9, 1, 3), (3, 3, 5), (4, 3, 1)])
def test_block_ilu0_matches_its_definition(B, shape):
    """The red-black block ILU(0) first stage (PF_S1_ILU0) against a dense
    reference of the same factorisation on the GPU's own Jacobian, FP64."""
    nx, ny, nz = shape
    sc, ctl = ragged_scenario(nx=nx, ny=ny, nz=nz)
    st = M.Setup(sc)
    rng = np.random.default_rng(8)
    x0 = M.initial_state(st)
    x_old, x = random_state(st, rng, x0), random_state(st, rng, x0)
    st, sim, R_o, J_o, R_g, J_g = assemble_both(B, sc, ctl, x_old, x, DAY, precond=B.PF_PC_BJACOBI, stage1=1)
    v = rng.normal(size=st.nunk)
    z_g = sim.apply_preconditioner(v)
    z_r = rb_block_ilu0_apply(sc, J_g, v)
    assert np.allclose(z_g, z_r, rtol=1e-10, atol=1e-12 * np.abs(z_r).max())
    sim.close()


def test_compact_ilu_copies(B):
    """ilu_store: with the per-colour copies (FP64: the red blocks, the black
    products J_bj D_j^-1 and the block inverses per colour slot) the
    preconditioner output equals the by-cell one to rounding, alone and inside
    CPR (whose stage 2 reads the black rows' pressure combination that the
    set-up writes in either case); the two- and the three-launch ILU(0) solve
    give it bit for bit in each layout; with a BF16 copy (mixed precision) the
    time steps still land on the oracle's root."""
    sc, ctl = ragged_scenario(nx=9, ny=7, nz=4)
    st = M.Setup(sc)
    rng = np.random.default_rng(12)
    x0 = M.initial_state(st)
    x_old, x = random_state(st, rng, x0), random_state(st, rng, x0)
    v = rng.normal(size=st.nunk)
    for precond in (B.PF_PC_BJACOBI, B.PF_PC_CPR):  # the ILU(0) solve alone; the CPR apply (stage 2 too)
        outs = []
        for store in (0, 1):
            per_form = []
            for fused in (0, 1):
                _, sim, _, _, _, _ = assemble_both(B, sc, ctl, x_old, x, DAY, precond=precond, stage1=1,
                                                   ilu_store=store)
                sim.set_tuning(ilu_fused=fused)
                assert sim.tuning()["ilu_fused"] == fused
                per_form.append(sim.apply_preconditioner(v))
                sim.close()
            assert np.array_equal(per_form[0], per_form[1])
            outs.append(per_form[0])
        scale = np.abs(outs[0]).max()
        assert np.abs(outs[0] - outs[1]).max() <= 1e-10 * scale
    sc1 = G.scenario_c1(nx=12, ny=10, nz=3, n_steps=4)
    sim = B.Simulator(sc1, stream=B.current_stream_handle(), precision=B.PF_PREC_MIXED, precond=B.PF_PC_CPR,
                      use_forcing=1, ilu_store=2)
    states = []
    sim.run_schedule(n_steps=4, callback=lambda s, rec: states.append(s.get_x()))
    sim.close()
    st1, _, hist = M.run(sc1, n_steps=4)
    for k in range(4):
        assert max(field_errors(st1.n, states[k], hist[k]["x"])) <= 1e-6


@pytest.mark.parametrize("shape", [(9, 7, 4), (8, 1, 3)])
def test_red_rows_of_the_ilu_residual_are_their_well_columns(B, shape):
    """The reading behind the CPR stage 2 after ILU(0): the last (red) sweep
    solves the red rows' cell part exactly, so v - J y on a red cell is its
    well column -B y_w alone, and the stage forms only the black rows.  Checked
    in FP64 with the GPU's own ILU(0) output and Jacobian."""
    nx, ny, nz = shape
    sc, ctl = ragged_scenario(nx=nx, ny=ny, nz=nz)
    st = M.Setup(sc)
    rng = np.random.default_rng(21)
    x0 = M.initial_state(st)
    x_old, x = random_state(st, rng, x0), random_state(st, rng, x0)
    st, sim, _, _, _, J_g = assemble_both(B, sc, ctl, x_old, x, DAY, precond=B.PF_PC_BJACOBI, stage1=1)
    v = rng.normal(size=st.nunk)
    y = sim.apply_preconditioner(v)
    sim.close()
    n = st.n
    J = J_g.tocsr()
    cell_part = v[:3 * n] - J[:3 * n, :3 * n] @ y[:3 * n]
    idx = np.arange(n)
    red = ((idx % nx) + (idx // nx) % ny + idx // (nx * ny)) % 2 == 0
    rows_red = (3 * idx[red][:, None] + np.arange(3)).ravel()
    rows_black = (3 * idx[~red][:, None] + np.arange(3)).ravel()
    scale = np.abs(J[:3 * n, :3 * n]) @ np.abs(y[:3 * n]) + np.abs(v[:3 * n])
    assert np.all(np.abs(cell_part[rows_red]) <= 1e-12 * scale[rows_red])
    # the black rows are where the ILU(0) error lives
    assert np.max(np.abs(cell_part[rows_black]) / scale[rows_black]) > 1e-6
    assert np.count_nonzero(J[:3 * n, 3 * n:][rows_red].toarray()) > 0  # a red cell is perforated: its well column counts
