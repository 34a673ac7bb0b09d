"""pf_residual_norms_noalloc: the residual norms for callers that cannot
allocate device memory (graph capture, frameworks that own all device memory,
allocation-free loops).  Its two outputs must equal the norms that
pf_newton_iteration reports for the same residual, on two calls in a row (the
second call reuses the fixed scratch the first one left behind).

Collected last on purpose (file name), so that a run that stops at the first
failure has already run every other test; it also passes alone in a fresh
process, where its first call resolves the scratch address.
"""

import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12  # same-arithmetic comparison: only the order of the 2-norm sum differs


def test_noalloc_norms_match_newton_report():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    torch.cuda.set_device(0)
    from paper_1807_05298_gb300 import build as bld
    bld.build()
    from paper_1807_05298_gb300 import binding as B
    from oracle import model as M
    from scenarios import generate as G

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
    dt = 2.0 * G.DAY

    # the existing entry point: norms reported by pf_newton_iteration
    sim = B.Simulator(sc, stream=B.current_stream_handle())
    sim.set_controls(ctl)
    sim.begin_step(dt)
    rep = sim.newton_iteration()
    R = sim.export_system()[0]
    sim.close()

    st = M.Setup(sc)
    ph = sc["physics"]
    V = sc["dx"] * sc["dy"] * sc["dz"]
    inv_pv = 1.0 / (V * sc["phi"])
    denom = []
    for w, c in enumerate(ctl):
        if c["ctrl"] == "bhp":
            denom.append(dt * (st.wells[w]["W"] * 1.0e5))
        else:
            rho_t = ph["rho_o"] if c["ctrl"] == "orate" else ph["rho_w"]
            denom.append(dt * (rho_t * abs(c["target"])))

    dev = torch.device("cuda", 0)
    R_d = torch.tensor(R, dtype=torch.float64, device=dev)
    ip_d = torch.tensor(inv_pv, dtype=torch.float64, device=dev)
    den_d = torch.tensor(denom, dtype=torch.float64, device=dev)
    out_d = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)

    L = C.CDLL(B.LIB_PATH)
    f = L.pf_residual_norms_noalloc
    f.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double,
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    L.pf_noalloc_last_error.restype = C.c_char_p
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = nx * ny * nz

    results = []
    for _ in range(2):
        out_d.fill_(float("nan"))
        rc = f(n, len(ctl), R_d.data_ptr(), ip_d.data_ptr(), den_d.data_ptr(), ph["rho_o"], ph["rho_w"],
               ph["c_ref"], out_d.data_ptr(), stream)
        assert rc == 0, L.pf_noalloc_last_error().decode()
        torch.cuda.synchronize()
        results.append(out_d.cpu().numpy().copy())
    for res in results:
        assert res[0] == pytest.approx(rep.res_scaled, rel=TOL)
        assert res[1] == pytest.approx(rep.res_norm2, rel=TOL)
    assert np.array_equal(results[0], results[1])   # deterministic reduction order

    # sizes beyond the fixed scratch are rejected with a message, nothing launched
    rc = f(1 << 25, 0, R_d.data_ptr(), ip_d.data_ptr(), None, ph["rho_o"], ph["rho_w"], ph["c_ref"],
           out_d.data_ptr(), stream)
    assert rc == B.PF_EINVAL and b"16777216" in L.pf_noalloc_last_error()
