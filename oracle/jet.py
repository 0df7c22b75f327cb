"""Second-order forward-mode numbers ("jets") for the FP64 oracle.

TEST INFRASTRUCTURE ONLY: the oracle may be used by tests/, the smoke check and the
CPU-baseline leg of the benchmark, never by the product path.

A Jet carries, for every element of a numpy array of points, the value v, the
gradient g (last axis: k seed directions) and the Hessian h (last two axes: k x k).
The oracle uses it to evaluate the QP matrices of Eq. 4 (first derivatives of the
dynamics), the mixed derivatives d/dtheta (dF/dz) needed by dF/dtheta in Eq. 3, and
the dynamics curvature used by the exact-Hessian check (Sec. 3.4, "Exact SQP vs iLQR").

Rules implemented (chain rule to second order):
  unary  y = phi(a):  y.g = phi'(a) a.g,  y.h = phi'(a) a.h + phi''(a) a.g a.g^T
  product y = a b:    y.g = a b.g + b a.g,
                      y.h = a b.h + b a.h + a.g b.g^T + b.g a.g^T
Functions below accept either Jets or plain numpy arrays, so the same model code
evaluates plain values (line search, rollouts) and derivatives.
"""
import numpy as np


class Jet:
    __array_priority__ = 1000
    __array_ufunc__ = None  # make numpy defer to the reflected Jet operators
    __slots__ = ("v", "g", "h")

    def __init__(self, v, g, h):
        self.v = np.asarray(v, dtype=np.float64)
        self.g = g
        self.h = h

    @property
    def k(self):
        return self.g.shape[-1]

    # ---- construction -------------------------------------------------
    @staticmethod
    def seed(v, index, k):
        """Independent variable: value v (array), derivative 1 along seed `index`."""
        v = np.asarray(v, dtype=np.float64)
        g = np.zeros(v.shape + (k,))
        g[..., index] = 1.0
        h = np.zeros(v.shape + (k, k))
        return Jet(v, g, h)

    @staticmethod
    def seed_dir(v, direction, k):
        """Variable whose gradient is a given array `direction` of shape v.shape+(k,)."""
        v = np.asarray(v, dtype=np.float64)
        g = np.broadcast_to(np.asarray(direction, dtype=np.float64), v.shape + (k,)).copy()
        return Jet(v, g, np.zeros(v.shape + (k, k)))

    def _lift(self, c):
        c = np.asarray(c, dtype=np.float64)
        shape = np.broadcast_shapes(self.v.shape, c.shape)
        return Jet(np.broadcast_to(c, shape), np.zeros(shape + (self.k,)),
                   np.zeros(shape + (self.k, self.k)))

    # ---- arithmetic ---------------------------------------------------
    def __add__(self, o):
        if isinstance(o, Jet):
            return Jet(self.v + o.v, self.g + o.g, self.h + o.h)
        o = np.asarray(o, dtype=np.float64)
        return Jet(self.v + o, self.g + np.zeros(o.shape + (1,)), self.h + np.zeros(o.shape + (1, 1)))

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, -self.g, -self.h)

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if isinstance(o, Jet):
            a, b = self, o
            v = a.v * b.v
            g = a.v[..., None] * b.g + b.v[..., None] * a.g
            h = (a.v[..., None, None] * b.h + b.v[..., None, None] * a.h
                 + a.g[..., :, None] * b.g[..., None, :] + b.g[..., :, None] * a.g[..., None, :])
            return Jet(v, g, h)
        o = np.asarray(o, dtype=np.float64)
        return Jet(self.v * o, self.g * o[..., None], self.h * o[..., None, None])

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, Jet):
            return self * reciprocal(o)
        return self * (1.0 / np.asarray(o, dtype=np.float64))

    def __rtruediv__(self, o):
        return reciprocal(self) * o

    def __pow__(self, n):
        if not isinstance(n, int) or n < 0:
            raise ValueError("only non-negative integer powers")
        out = 1.0
        for _ in range(n):
            out = self * out
        return out


def _unary(a, f, d1, d2):
    """Apply phi with phi'=d1, phi''=d2 (all evaluated at a.v) to a Jet."""
    v = f
    g = d1[..., None] * a.g
    h = d1[..., None, None] * a.h + d2[..., None, None] * (a.g[..., :, None] * a.g[..., None, :])
    return Jet(v, g, h)


def reciprocal(a):
    if isinstance(a, Jet):
        x = a.v
        return _unary(a, 1.0 / x, -1.0 / x**2, 2.0 / x**3)
    return 1.0 / a


def sin(a):
    if isinstance(a, Jet):
        return _unary(a, np.sin(a.v), np.cos(a.v), -np.sin(a.v))
    return np.sin(a)


def cos(a):
    if isinstance(a, Jet):
        return _unary(a, np.cos(a.v), -np.sin(a.v), -np.cos(a.v))
    return np.cos(a)


def tan(a):
    if isinstance(a, Jet):
        t = np.tan(a.v)
        s2 = 1.0 + t * t
        return _unary(a, t, s2, 2.0 * t * s2)
    return np.tan(a)


def atan(a):
    if isinstance(a, Jet):
        x = a.v
        d = 1.0 / (1.0 + x * x)
        return _unary(a, np.arctan(x), d, -2.0 * x * d * d)
    return np.arctan(a)


def sqrt(a):
    if isinstance(a, Jet):
        s = np.sqrt(a.v)
        return _unary(a, s, 0.5 / s, -0.25 / (s * a.v))
    return np.sqrt(a)


def exp(a):
    if isinstance(a, Jet):
        e = np.exp(a.v)
        return _unary(a, e, e, e)
    return np.exp(a)


def tanh(a):
    if isinstance(a, Jet):
        t = np.tanh(a.v)
        d = 1.0 - t * t
        return _unary(a, t, d, -2.0 * t * d)
    return np.tanh(a)


def absval(a):
    """|a|; derivative sign(a) (0 at 0), zero curvature (kinks are avoided by callers)."""
    if isinstance(a, Jet):
        s = np.sign(a.v)
        return _unary(a, np.abs(a.v), s, np.zeros_like(s))
    return np.abs(a)


def value(a):
    return a.v if isinstance(a, Jet) else np.asarray(a, dtype=np.float64)


def where(cond, a, b):
    """Elementwise select between two (Jet or array) branches by a boolean array."""
    if not isinstance(a, Jet) and not isinstance(b, Jet):
        return np.where(cond, a, b)
    if not isinstance(a, Jet):
        a = b._lift(a)
    if not isinstance(b, Jet):
        b = a._lift(b)
    c = np.asarray(cond)
    return Jet(np.where(c, a.v, b.v), np.where(c[..., None], a.g, b.g),
               np.where(c[..., None, None], a.h, b.h))


def sign_of(a):
    return np.sign(value(a))
