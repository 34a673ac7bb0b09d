"""The oracle on a 3x3x3 window reproduces the full oracle's residual and
Jacobian rows of the window's centre cell: the check that lets the GPU's
full-size (27M-cell) assembly be compared with the oracle cell by cell."""

import numpy as np
import scipy.sparse as sp

from gpu_helpers import perforated_cells, window_around, window_state
from oracle import model as M
from scenarios import generate as G

BAR = 1e5


def test_window_rows_equal_full_rows():
    sc = G.scenario_c1(nx=8, ny=7, nz=5, n_steps=2)
    st = M.Setup(sc)
    ctl = sc["schedule"][0]["controls"]
    dt = sc["schedule"][0]["dt"]
    rng = np.random.default_rng(6)
    x_old = M.initial_state(st)
    x = x_old.copy()
    x[0:3 * st.n:3] += rng.normal(0.0, 2.0 * BAR, st.n)
    x[1:3 * st.n:3] = rng.uniform(0.22, 0.78, st.n)
    x[2:3 * st.n:3] = rng.uniform(0.0, 1.6, st.n)
    R, J = M.assemble(st, x, M.masses(st, x_old), dt, ctl, M.well_gamma(st, x_old, ctl))
    J = sp.csr_matrix(J)
    perf = perforated_cells(sc)
    checked = 0
    for c in range(st.n):
        k, rem = divmod(c, sc["nx"] * sc["ny"])
        j, i = divmod(rem, sc["nx"])
        if not (0 < i < sc["nx"] - 1 and 0 < j < sc["ny"] - 1 and 0 < k < sc["nz"] - 1) or c in perf:
            continue
        w, idx = window_around(sc, c)
        stw = M.Setup(w)
        xw, xw_old = window_state(x, idx), window_state(x_old, idx)
        Rw, Jw = M.assemble(stw, xw, M.masses(stw, xw_old), dt, [], M.well_gamma(stw, xw_old, []))
        Jw = sp.csr_matrix(Jw)
        cols_full = (3 * idx[:, None] + np.arange(3)).ravel()
        for a in range(3):
            assert abs(Rw[3 * 13 + a] - R[3 * c + a]) <= 1e-13 * (abs(R[3 * c + a]) + 1e-300)
            row_full = J[3 * c + a].toarray().ravel()
            row_win = Jw[3 * 13 + a].toarray().ravel()
            assert np.allclose(row_win, row_full[cols_full], rtol=1e-13, atol=0.0)
            assert np.count_nonzero(row_full) == np.count_nonzero(row_full[cols_full])  # nothing outside
        checked += 1
    assert checked >= 20
