"""Ordering of the unknowns and preconditioner convergence (Sec. 3.4).

The paper arranges the unknowns either point-wise (all P_o, then all S_w, all
C, then the wells) or block-wise (P_o, S_w, C per cell, then the wells) and
states that the preconditioner converges better with the block-wise order,
which is the order this library uses throughout.  This study repeats the
comparison on the oracle's own Jacobians: the same scalar ILU(0) factor, the
same restarted GMRES, the two orderings.  No GPU.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import model as M
from scenarios import generate as G


def ilu0(A):
    """Scalar ILU(0): Gaussian elimination restricted to the pattern of A."""
    A = sp.csr_matrix(A, copy=True)
    A.sort_indices()
    n = A.shape[0]
    ptr, idx, val = A.indptr, A.indices, A.data.astype(np.float64).copy()
    diag = np.array([ptr[i] + np.searchsorted(idx[ptr[i]:ptr[i + 1]], i) for i in range(n)])
    for i in range(n):
        where = {c: ptr[i] + t for t, c in enumerate(idx[ptr[i]:ptr[i + 1]])}
        for t in range(ptr[i], ptr[i + 1]):
            k = idx[t]
            if k >= i:
                break
            val[t] /= val[diag[k]]
            for u in range(diag[k] + 1, ptr[k + 1]):
                pos = where.get(idx[u])
                if pos is not None:
                    val[pos] -= val[t] * val[u]
    LU = sp.csr_matrix((val, idx, ptr), shape=A.shape)
    return sp.tril(LU, -1, format="csr") + sp.eye(n, format="csr"), sp.triu(LU, 0, format="csr")


def gmres_iterations(A, b):
    L, U = ilu0(A)
    prec = spla.LinearOperator(A.shape, matvec=lambda v: spla.spsolve_triangular(
        U, spla.spsolve_triangular(L, v, lower=True), lower=False))
    count = [0]

    def tick(_):
        count[0] += 1
    _, info = spla.gmres(A, b, M=prec, rtol=1e-8, restart=30, maxiter=400, callback=tick,
                         callback_type="pr_norm")
    assert info == 0
    return count[0]


def newton_system(sc, n_steps):
    """The Jacobian and right-hand side one Newton update into the step after
    n_steps steps of the oracle's own time loop."""
    st, x, hist = M.run(sc, n_steps=n_steps)
    ctl = [dict(c) for c in sc["schedule"][0]["controls"]]
    for w, switched in enumerate(hist[-1]["switched"]):
        if switched:
            ctl[w] = dict(ctl[w], ctrl="bhp", target=ctl[w]["limit"])
    dt = sc["schedule"][0]["dt"]
    gam = M.well_gamma(st, x, ctl)
    Mold = M.masses(st, x)
    R, J = M.assemble(st, x, Mold, dt, ctl, gam)
    x1 = M.update(st, x, spla.spsolve(J.tocsc(), -R), 0.2)
    R, J = M.assemble(st, x1, Mold, dt, ctl, gam)
    return st, J.tocsr(), -R


@pytest.mark.parametrize("name", ["10x10x3", "12x12x4 five-spot"])
def test_block_wise_order_converges_no_slower_than_point_wise(name):
    sc, n_steps = (G.scenario_c1(n_steps=10), 5) if name == "10x10x3" else \
        (G.scenario_c2(nx=12, ny=12, nz=4, n_steps=6), 3)
    st, J, b = newton_system(sc, n_steps)
    n, nw = st.n, st.nw
    block_wise = np.arange(3 * n + nw)
    point_wise = np.concatenate([np.arange(0, 3 * n, 3), np.arange(1, 3 * n, 3), np.arange(2, 3 * n, 3),
                                 3 * n + np.arange(nw)])
    its = {}
    for label, p in (("block", block_wise), ("point", point_wise)):
        its[label] = gmres_iterations(J[p][:, p], b[p])
    assert its["block"] <= its["point"], its
