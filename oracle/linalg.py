"""Dense linear algebra written from textbook definitions (oracle test
infrastructure; see the package header for who may import it)."""

import numpy as np


def lu_solve_dense(A, b):
    """Gaussian elimination with partial (row) pivoting, then forward and
    back substitution (Golub & Van Loan, Algorithm 3.4.1)."""
    A = np.array(A, dtype=np.float64, copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    n = A.shape[0]
    for k in range(n - 1):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if A[p, k] == 0.0:
            raise ZeroDivisionError("singular matrix")
        if p != k:
            A[[k, p]] = A[[p, k]]
            b[[k, p]] = b[[p, k]]
        m = A[k + 1:, k] / A[k, k]
        A[k + 1:, k + 1:] -= np.outer(m, A[k, k + 1:])
        A[k + 1:, k] = 0.0
        b[k + 1:] -= m * b[k]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (b[i] - A[i, i + 1:] @ x[i + 1:]) / A[i, i]
    return x
