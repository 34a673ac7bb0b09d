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


def test_black_sweep_through_the_products_is_the_same_solve():
    """The two-sweep form of the red-black ILU(0) solve used with the
    per-colour copies: the black sweep takes f_j of its red neighbours through
    T_bj = J_bj D_j^-1 (J_bj t_j = T_bj f_j with t_j = D_j^-1 f_j), so no
    diagonal red sweep is needed.  Same factor, same result to rounding, on the
    oracle's Jacobian against the three-sweep reference.  T's oil row has a
    nonzero polymer column although J_bj's is structurally zero, which is why
    the copy stores all nine entries of T."""
    for shape, seed in (((6, 5, 3), 3), ((5, 4, 2), 4)):
        sc, st, J, rng = oracle_system(*shape, seed)
        nx, ny, nz = shape
        n = st.n
        v = rng.normal(size=3 * n + st.nw)
        ref = rb_block_ilu0_apply(sc, J, v)
        idx = np.arange(n)
        i_, j_, k_ = idx % nx, (idx // nx) % ny, idx // (nx * ny)
        red = (i_ + j_ + k_) % 2 == 0
        blk = lambda r, c: J[3 * r:3 * r + 3, 3 * c:3 * c + 3].toarray()

        def nbrs(c):
            out = []
            for coord, lim, step in ((i_[c], nx, 1), (j_[c], ny, nx), (k_[c], nz, nx * ny)):
                if coord > 0:
                    out.append(c - step)
                if coord < lim - 1:
                    out.append(c + step)
            return out
        Dinv = {c: np.linalg.inv(blk(c, c)) for c in idx[red]}
        T = {(b, r): blk(b, r) @ Dinv[r] for b in idx[~red] for r in nbrs(b)}
        f = v[:3 * n].reshape(n, 3)
        y = np.zeros((n, 3))
        oil_c = []
        for b in idx[~red]:
            D0 = blk(b, b)
            D = D0 - sum(T[b, r] @ blk(r, b) for r in nbrs(b))
            if not np.linalg.det(D) / np.linalg.det(D0) > 0.1:
                D = D0
            y[b] = np.linalg.solve(D, f[b] - sum(T[b, r] @ f[r] for r in nbrs(b)))
            for r in nbrs(b):
                assert blk(b, r)[0, 2] == 0.0
                oil_c.append(abs(T[b, r][0, 2]))
        for r in idx[red]:
            y[r] = Dinv[r] @ (f[r] - sum(blk(r, b) @ y[b] for b in nbrs(r)))
        scale = np.abs(ref[:3 * n]).max()
        assert np.abs(y.ravel() - ref[:3 * n]).max() <= 1e-12 * scale
        assert max(oil_c) > 0.0
