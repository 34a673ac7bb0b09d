"""Forward-mode dual numbers over numpy arrays (oracle test infrastructure).

A ``Dual`` carries a value array ``v`` of shape (n,) and a derivative array
``d`` of shape (n, k): d[i, j] is the derivative of v[i] with respect to the
j-th independent variable of item i.  Every rule below is the textbook
derivative of the operation, so Jacobians built from it are exact up to
rounding and independent of any hand-derived formula.
"""

import numpy as np


class Dual:
    __slots__ = ("v", "d")
    __array_ufunc__ = None  # make numpy defer to the reflected Dual operators

    def __init__(self, v, d):
        self.v = np.asarray(v, dtype=np.float64)
        self.d = np.asarray(d, dtype=np.float64)

    @staticmethod
    def variable(v, k, j):
        """Independent variable number j (of k) with values v."""
        v = np.asarray(v, dtype=np.float64)
        d = np.zeros((v.shape[0], k))
        d[:, j] = 1.0
        return Dual(v, d)

    @staticmethod
    def const(v, k):
        v = np.asarray(v, dtype=np.float64)
        return Dual(v, np.zeros((v.shape[0], k)))

    @property
    def k(self):
        return self.d.shape[1]

    def take(self, idx):
        return Dual(self.v[idx], self.d[idx])

    def embed(self, k, offset):
        """Same values, derivative columns moved to [offset, offset + self.k) of k."""
        d = np.zeros((self.v.shape[0], k))
        d[:, offset:offset + self.k] = self.d
        return Dual(self.v, d)

    # arithmetic ---------------------------------------------------------
    def __add__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v + o.v, self.d + o.d)
        return Dual(self.v + o, self.d)

    __radd__ = __add__

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __sub__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v - o.v, self.d - o.d)
        return Dual(self.v - o, self.d)

    def __rsub__(self, o):
        return Dual(o - self.v, -self.d)

    def __mul__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v * o.v, self.d * o.v[:, None] + o.d * self.v[:, None])
        o = np.asarray(o, dtype=np.float64)
        return Dual(self.v * o, self.d * (o[:, None] if o.ndim else o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, Dual):
            q = self.v / o.v
            return Dual(q, (self.d - o.d * q[:, None]) / o.v[:, None])
        o = np.asarray(o, dtype=np.float64)
        return Dual(self.v / o, self.d / (o[:, None] if o.ndim else o))

    def __rtruediv__(self, o):
        q = o / self.v
        return Dual(q, -self.d * (q / self.v)[:, None])

    def __pow__(self, p):
        """Power with a constant real exponent p."""
        p = float(p)
        if p == 0.0:
            return Dual(np.ones_like(self.v), np.zeros_like(self.d))
        if p == 1.0:
            return Dual(self.v.copy(), self.d.copy())
        with np.errstate(divide="ignore", invalid="ignore"):
            dv = p * np.power(self.v, p - 1.0)
        dv = np.where(self.v == 0.0, 0.0 if p > 1.0 else dv, dv)
        return Dual(np.power(self.v, p), self.d * dv[:, None])


def exp(a):
    e = np.exp(a.v)
    return Dual(e, a.d * e[:, None])


def log(a):
    return Dual(np.log(a.v), a.d / a.v[:, None])


def where(cond, a, b):
    """Elementwise select: a where cond else b (value and derivative)."""
    cond = np.asarray(cond, dtype=bool)
    k = a.k if isinstance(a, Dual) else b.k
    n = cond.shape[0]
    if not isinstance(a, Dual):
        a = Dual(np.broadcast_to(np.asarray(a, dtype=np.float64), (n,)), np.zeros((n, k)))
    if not isinstance(b, Dual):
        b = Dual(np.broadcast_to(np.asarray(b, dtype=np.float64), (n,)), np.zeros((n, k)))
    return Dual(np.where(cond, a.v, b.v), np.where(cond[:, None], a.d, b.d))
