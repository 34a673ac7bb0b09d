"""pf_residual_norms_noalloc: the residual norms for callers that cannot
allocate device memory (a host framework that owns every device allocation,
a loop that cannot afford an allocation once it runs).  Its two outputs must
equal the norms that pf_newton_iteration reports for the same residual and
the oracle's definition of them, on two calls in a row (the second call
reuses the fixed scratch the first one left behind), from one thread block up
to the largest size its scratch takes (4096 blocks).

Collected last on purpose (file name), so that a run that stops at the first
failure has already run every other test; it also passes alone in a fresh
process, where its first call resolves the scratch address.
"""

import ctypes as C
import types

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12     # same arithmetic as the library's norm step; only the order of the 2-norm sum differs
MAX_CELLS = 16_777_216


def _lib():
    from paper_1807_05298_gb300 import binding as B
    L = C.CDLL(B.LIB_PATH)
    f = L.pf_residual_norms_noalloc
    f.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    L.pf_noalloc_last_error.restype = C.c_char_p
    return L


def _call(L, n, nw, R_d, ip_d, den_d, ph, out_d, stream):
    import torch
    out_d.fill_(float("nan"))
    rc = L.pf_residual_norms_noalloc(n, nw, R_d.data_ptr(), ip_d.data_ptr(),
                                     den_d.data_ptr() if den_d is not None else None,
                                     ph["rho_o"], ph["rho_w"], ph["c_ref"], out_d.data_ptr(), stream)
    assert rc == 0, L.pf_noalloc_last_error().decode()
    torch.cuda.synchronize()
    return out_d.cpu().numpy().copy()


def _well_denoms(st, ph, ctl, dt):
    """The well rows' scale of the Newton convergence measure (reading 15):
    dt W * 1 bar for a BHP row, dt rho_ref |target| for a rate row."""
    from oracle import model as M
    out = []
    for w, c in enumerate(ctl):
        if c["ctrl"] == "bhp":
            out.append(dt * st.wells[w]["W"] * 1.0e5)
        else:
            _, _, rho_t = M.rate_coefficients(ph, c["ctrl"], st.wells[w]["kind"])
            out.append(dt * rho_t * abs(c["target"]))
    return out


def _scenario(name):
    from scenarios import generate as G
    if name == "23x13x5":          # one thread block of the kernel (4096 cells per block)
        nx, ny, nz = 23, 13, 5
        sc = G.scenario_c1(nx=nx, ny=ny, nz=nz)
        col = lambda i, j, k0, k1: np.array([i + nx * (j + ny * k) for k in range(k0, k1)], dtype=np.int64)
        sc["wells"] = [dict(kind="inj", cells=col(0, 0, 0, 3)), dict(kind="prod", cells=col(nx - 1, ny - 1, 0, nz)),
                       dict(kind="prod", cells=col(nx // 2, ny // 2, 3, nz))]
        for w in sc["wells"]:
            w.update(rw=0.1, skin=0.0, gf=0.249, f=1.0, fh=1.0, dirs=["z"] * len(w["cells"]),
                     Pb0=float(sc["P0"][w["cells"][0]]))
        ctl = [dict(ctrl="wrate", target=60.0 / G.DAY, limit=None, c_inj=1.2),
               dict(ctrl="bhp", target=150.0 * G.BAR, limit=None, c_inj=0.0),
               dict(ctrl="lrate", target=20.0 / G.DAY, limit=None, c_inj=0.0)]
        return sc, ctl, 2.0 * G.DAY
    sc = G.scenario_c2()               # 100x100x10: 25 thread blocks
    per = sc["schedule"][0]
    ctl = [dict(c, limit=None) for c in per["controls"]]
    return sc, ctl, per["dt"]


@pytest.mark.parametrize("name", ["23x13x5", "100x100x10"])
def test_noalloc_norms_match_newton_report_and_oracle(name):
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    torch.cuda.set_device(0)
    from paper_1807_05298_gb300 import build as bld
    bld.build()
    from paper_1807_05298_gb300 import binding as B
    from oracle import model as M

    sc, ctl, dt = _scenario(name)
    ph = sc["physics"]

    # the existing entry point: the norms pf_newton_iteration reports
    sim = B.Simulator(sc, stream=B.current_stream_handle())
    sim.set_controls(ctl)
    sim.begin_step(dt)
    rep = sim.newton_iteration()
    R = sim.export_system()[0]
    sim.close()

    st = M.Setup(sc)
    denom = _well_denoms(st, ph, ctl, dt)
    V = sc["dx"] * sc["dy"] * sc["dz"]
    dev = torch.device("cuda", 0)
    R_d = torch.tensor(R, dtype=torch.float64, device=dev)
    ip_d = torch.tensor(1.0 / (V * sc["phi"]), dtype=torch.float64, device=dev)
    den_d = torch.tensor(denom, dtype=torch.float64, device=dev)
    out_d = torch.empty(2, dtype=torch.float64, device=dev)
    L = _lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = st.n

    results = [_call(L, n, len(ctl), R_d, ip_d, den_d, ph, out_d, stream) for _ in range(2)]
    oracle_scaled = M.scaled_residual(st, R, dt, ctl)
    oracle_norm2 = float(np.linalg.norm(R))
    for res in results:
        assert res[0] == pytest.approx(rep.res_scaled, rel=TOL)
        assert res[1] == pytest.approx(rep.res_norm2, rel=TOL)
        assert res[0] == pytest.approx(oracle_scaled, rel=TOL)
        assert res[1] == pytest.approx(oracle_norm2, rel=TOL)
    assert np.array_equal(results[0], results[1])   # deterministic reduction order

    # sizes beyond the fixed scratch are rejected with a message, nothing launched
    rc = L.pf_residual_norms_noalloc(MAX_CELLS + 1, 0, R_d.data_ptr(), ip_d.data_ptr(), None, ph["rho_o"],
                                     ph["rho_w"], ph["c_ref"], out_d.data_ptr(), stream)
    assert rc == B.PF_EINVAL and b"16777216" in L.pf_noalloc_last_error()


def test_noalloc_norms_at_the_size_limit():
    """16,777,216 cells (4096 thread blocks, every slot of the scratch) and
    4096 wells, the largest call the scratch takes, on a seeded residual of
    the magnitudes a step produces; against the oracle's scaled residual and
    numpy's 2-norm.  A small call in between must not disturb the next large
    one (the completion counter and the partials are reused)."""
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    torch.cuda.set_device(0)
    from paper_1807_05298_gb300 import build as bld
    bld.build()
    from oracle import model as M
    from scenarios import generate as G

    n, nw = MAX_CELLS, 4096
    ph = G.default_physics()
    rng = np.random.default_rng(7)
    V = 20.0 * 20.0 * 4.0
    phi = 0.1 + 0.2 * rng.random(n)
    R = np.concatenate([rng.standard_normal(3 * n) * np.repeat(V * phi * 1e-6, 3), rng.standard_normal(nw)])
    # one planted large entry deep inside the grid decides the max-norm
    R[3 * (n - 12345) + 1] = 3.0 * V * phi[n - 12345] * ph["rho_w"]
    W = 1e-9 * (1.0 + rng.random(nw))
    dt = 86400.0
    wells = [dict(kind="prod", W=float(W[w])) for w in range(nw)]
    ctl = [dict(ctrl="bhp", target=150e5) for _ in range(nw)]
    st = types.SimpleNamespace(n=n, ph=ph, V=V, phi_r=phi, wells=wells)
    denom = [dt * W[w] * 1.0e5 for w in range(nw)]

    dev = torch.device("cuda", 0)
    R_d = torch.tensor(R, dtype=torch.float64, device=dev)
    ip_d = torch.tensor(1.0 / (V * phi), dtype=torch.float64, device=dev)
    den_d = torch.tensor(denom, dtype=torch.float64, device=dev)
    out_d = torch.empty(2, dtype=torch.float64, device=dev)
    L = _lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    big1 = _call(L, n, nw, R_d, ip_d, den_d, ph, out_d, stream)
    small = _call(L, 1000, 0, R_d, ip_d, None, ph, out_d, stream)
    big2 = _call(L, n, nw, R_d, ip_d, den_d, ph, out_d, stream)
    assert np.array_equal(big1, big2)
    assert big1[0] == pytest.approx(M.scaled_residual(st, R, dt, ctl), rel=TOL)
    assert big1[0] == pytest.approx(3.0, rel=TOL)
    assert big1[1] == pytest.approx(float(np.linalg.norm(R)), rel=TOL)
    st_small = types.SimpleNamespace(n=1000, ph=ph, V=V, phi_r=phi[:1000], wells=[])
    R_small = R[:3000]
    assert small[0] == pytest.approx(M.scaled_residual(st_small, R_small, dt, []), rel=TOL)
    assert small[1] == pytest.approx(float(np.linalg.norm(R_small)), rel=TOL)
