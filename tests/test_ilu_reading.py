"""The algebra behind CPR stage 2 after the red-black block ILU(0) first stage
(Alg. 2 with the ILU(0) reading of the RAS local solve), pinned on the CPU with
the oracle's own Jacobian and a dense reference of the ILU(0) solve.

The red sweep, the last one, solves each red row's cell part exactly, so the
residual v - J y of a red row is its well column -B y_w alone; stage 2 forms
only the black rows.  A mistake in the colouring, the sweep order or the
sign of the well term fails here.
"""

import numpy as np

from gpu_helpers import rb_block_ilu0_apply
from oracle import model as M
from scenarios import generate as G

DAY = 86400.0
BAR = 1e5


def oracle_system(nx, ny, nz, seed):
    sc = G.scenario_c1(nx=nx, ny=ny, nz=nz, n_steps=2)
    st = M.Setup(sc)
    ctl = sc["schedule"][0]["controls"]
    rng = np.random.default_rng(seed)
    x0 = M.initial_state(st)
    x = x0.copy()
    x[0:3 * st.n:3] += rng.normal(0.0, 2.0 * BAR, st.n)
    x[1:3 * st.n:3] = rng.uniform(0.22, 0.78, st.n)
    x[2:3 * st.n:3] = rng.uniform(0.0, 1.6, st.n)
    gam = M.well_gamma(st, x0, ctl)
    _, J = M.assemble(st, x, M.masses(st, x0), DAY, ctl, gam)
    return sc, st, J.tocsr(), rng


def test_red_rows_of_the_ilu_residual_are_their_well_columns():
    for shape, seed in (((6, 5, 3), 1), ((7, 1, 4), 2)):
        sc, st, J, rng = oracle_system(*shape, seed)
        nx, ny, nz = shape
        n = st.n
        v = rng.normal(size=3 * n + st.nw)
        y = rb_block_ilu0_apply(sc, J, v)
        idx = np.arange(n)
        red = ((idx % nx) + (idx // nx) % ny + idx // (nx * ny)) % 2 == 0
        rows = lambda cells: (3 * cells[:, None] + np.arange(3)).ravel()
        Jcc = J[:3 * n, :3 * n]
        cell_part = v[:3 * n] - Jcc @ y[:3 * n]
        scale = np.abs(Jcc) @ np.abs(y[:3 * n]) + np.abs(v[:3 * n])
        full = cell_part - J[:3 * n, 3 * n:] @ y[3 * n:]   # v - J y on the cell rows
        well_col = -(J[:3 * n, 3 * n:] @ y[3 * n:])
        r_red, r_black = rows(idx[red]), rows(idx[~red])
        assert np.all(np.abs(full[r_red] - well_col[r_red]) <= 1e-12 * scale[r_red])
        assert np.max(np.abs(full[r_black]) / scale[r_black]) > 1e-6      # the ILU(0) error lives here
        assert np.count_nonzero(well_col[r_red]) > 0                       # a perforated red cell counts
