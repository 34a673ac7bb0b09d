"""Helpers shared by the tests: rebuild the library's exported block layout
as a sparse matrix in the oracle's unknown ordering, and a dense reference of
the red-black block ILU(0) solve."""

import numpy as np
import scipy.sparse as sp

SLOT_OFFSETS = ["d", "xm", "xp", "ym", "yp", "zm", "zp"]


def neighbor_cols(nx, ny, nz):
    n = nx * ny * nz
    idx = np.arange(n)
    k, rem = np.divmod(idx, nx * ny)
    j, i = np.divmod(rem, nx)
    out = []
    for s in SLOT_OFFSETS:
        if s == "d":
            out.append((idx, np.ones(n, bool)))
        elif s == "xm":
            out.append((idx - 1, i > 0))
        elif s == "xp":
            out.append((idx + 1, i + 1 < nx))
        elif s == "ym":
            out.append((idx - nx, j > 0))
        elif s == "yp":
            out.append((idx + nx, j + 1 < ny))
        elif s == "zm":
            out.append((idx - nx * ny, k > 0))
        else:
            out.append((idx + nx * ny, k + 1 < nz))
    return out


def gpu_system_to_csr(sc, Jc, Bw, Cw, Dw, well_cells):
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    n = nx * ny * nz
    nw = len(well_cells)
    nunk = 3 * n + nw
    rows, cols, vals = [], [], []
    for s, (col, mask) in enumerate(neighbor_cols(nx, ny, nz)):
        cells = np.nonzero(mask)[0]
        for e in range(9):
            r, c = divmod(e, 3)
            rows.append(3 * cells + r)
            cols.append(3 * col[cells] + c)
            vals.append(Jc[s, e, cells])
    m = 0
    for w, cells in enumerate(well_cells):
        for c in cells:
            for r in range(3):
                rows.append(np.array([3 * c + r])); cols.append(np.array([3 * n + w])); vals.append(np.array([Bw[r, m]]))
                rows.append(np.array([3 * n + w])); cols.append(np.array([3 * c + r])); vals.append(np.array([Cw[r, m]]))
            m += 1
        rows.append(np.array([3 * n + w])); cols.append(np.array([3 * n + w])); vals.append(np.array([Dw[w]]))
    J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nunk, nunk))
    return J.tocsr()


def _row_max_abs(A):
    A = abs(A).tocsr()
    A.sum_duplicates()
    out = np.zeros(A.shape[0])
    nnz = np.diff(A.indptr) > 0
    if A.nnz:
        out[nnz] = np.maximum.reduceat(A.data, A.indptr[:-1][nnz])
    return out


def rel_matrix_error(Jg, Jo):
    """max |Jg - Jo| per row, relative to the row's largest |Jo| entry."""
    dmax = _row_max_abs((Jg - Jo).tocsr())
    amax = _row_max_abs(Jo)
    nz = amax > 0
    if np.any(dmax[~nz] > 0):
        return np.inf
    return float(np.max(dmax[nz] / amax[nz])) if nz.any() else 0.0


def rb_block_ilu0_apply(sc, J_csr, v, guard=0.1):
    """Reference red-black block ILU(0) solve, written from its definition:
    red cells (i + j + k even) first; the factor keeps the red diagonal
    blocks and replaces each black one by D_b - sum_j J_bj D_j^-1 J_jb
    (unless det of the result over det(D_b) is not above `guard`, when the
    cell keeps D_b); then forward and backward substitution.  Well rows:
    v_w / D_w."""
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    n = nx * ny * nz
    J = J_csr.tocsr()
    idx = np.arange(n)
    i_, j_, k_ = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    red = (i_ + j_ + k_) % 2 == 0
    blk = lambda r, c: J[3 * r:3 * r + 3, 3 * c:3 * c + 3].toarray()

    def nbrs(c):
        out = []
        for d, (coord, lim, st_) in enumerate(((i_[c], nx, 1), (j_[c], ny, nx), (k_[c], nz, nx * ny))):
            if coord > 0:
                out.append(c - st_)
            if coord < lim - 1:
                out.append(c + st_)
        return out
    Dinv = {c: np.linalg.inv(blk(c, c)) for c in idx[red]}
    Dp = {}
    for c in idx[~red]:
        D0 = blk(c, c)
        D = D0
        for r in nbrs(c):
            D = D - blk(c, r) @ Dinv[r] @ blk(r, c)
        if not np.linalg.det(D) / np.linalg.det(D0) > guard:
            D = D0
        Dp[c] = np.linalg.inv(D)
    f = v[:3 * n].reshape(n, 3)
    y = np.zeros((n, 3))
    for c in idx[red]:
        y[c] = Dinv[c] @ f[c]
    for c in idx[~red]:
        y[c] = Dp[c] @ (f[c] - sum(blk(c, r) @ y[r] for r in nbrs(c)))
    for c in idx[red]:
        y[c] = Dinv[c] @ (f[c] - sum(blk(c, r) @ y[r] for r in nbrs(c)))
    out = np.empty_like(v)
    out[:3 * n] = y.ravel()
    diag = J.diagonal()
    out[3 * n:] = v[3 * n:] / diag[3 * n:]
    return out


def window_around(sc, c):
    """The 3x3x3 block of cells centred on the interior cell c as a scenario
    of its own (same cell sizes, depth, rock and physics; no wells), with the
    natural indices of its 27 cells.  The centre (window cell 13) has the same
    faces, neighbours and transmissibilities as in the full grid, so the
    oracle's residual row and Jacobian row of the centre are those of cell c:
    only the window's own border rows differ.  Lets the oracle check single
    cells of grids too large for it to assemble whole."""
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    k, rem = divmod(int(c), nx * ny)
    j, i = divmod(rem, nx)
    assert 0 < i < nx - 1 and 0 < j < ny - 1 and 0 < k < nz - 1, "interior cells only"
    ii, jj, kk = np.arange(i - 1, i + 2), np.arange(j - 1, j + 2), np.arange(k - 1, k + 2)
    idx = (ii[None, None, :] + nx * (jj[None, :, None] + ny * kk[:, None, None])).ravel()
    w = dict(sc)
    w.update(nx=3, ny=3, nz=3, top=sc["top"] + (k - 1) * sc["dz"],
             kx=sc["kx"][idx], ky=sc["ky"][idx], kz=sc["kz"][idx], phi=sc["phi"][idx],
             P0=sc["P0"][idx], S0=sc["S0"][idx], C0=sc["C0"][idx], wells=[],
             schedule=[dict(n_steps=1, dt=sc["schedule"][0]["dt"], controls=[])])
    return w, idx


def window_state(x, idx):
    """Cell unknowns (P, S, C) of the window cells idx from a full state x."""
    cols = (3 * idx[:, None] + np.arange(3)).ravel()
    return x[cols]


def perforated_cells(sc):
    return set(int(c) for w in sc["wells"] for c in w["cells"])
