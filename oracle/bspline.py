"""B-spline bases for the inhomogeneous direction (paper Appendix C, Eq. disc_f_inhomo).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings of points the paper leaves open:
* order p B-splines (degree p-1, maximum continuity C^{p-2}) for every field
  except m2; order p+1 B-splines on the SAME breakpoints for m2 (Appendix C:
  d/dx2 of the m2 space must span the space of the other fields);
* clamped knot vectors (end knots repeated `order` times) with uniform
  breakpoints on [y0, y1]; the number of intervals is Ny - p + 1, so the
  order-p space has dimension Ny and the order-(p+1) space Ny + 1;
* collocation / physical points are the Greville abscissae.

The evaluation is the plain Cox-de Boor recursion, one basis function and one
point at a time, so that it can be checked against the textbook definition.
"""
import numpy as np


def clamped_uniform_knots(order, n, y0=-1.0, y1=1.0):
    """Knot vector of `n` order-`order` B-splines on [y0, y1], clamped, uniform breakpoints."""
    nint = n - order + 1
    if nint < 1:
        raise ValueError("need n >= order")
    brk = y0 + (y1 - y0) * np.arange(nint + 1, dtype=np.float64) / nint
    brk[-1] = y1
    return np.concatenate([np.full(order - 1, y0), brk, np.full(order - 1, y1)])


def greville(t, order):
    """Greville abscissae g_j = (t_{j+1} + ... + t_{j+order-1}) / (order - 1)."""
    n = len(t) - order
    return np.array([np.mean(t[j + 1:j + order]) for j in range(n)])


def _basis(t, j, k, d, x):
    """d-th derivative of the j-th B-spline of order k on knots t, at x (Cox-de Boor).

    Order-1 splines are indicator functions of [t_j, t_{j+1}); at the right end of
    the domain the last non-empty interval is closed so that x = y1 is covered.
    """
    if k == 1:
        if d > 0:
            return 0.0
        left, right = t[j], t[j + 1]
        if left == right:
            return 0.0
        if left <= x < right:
            return 1.0
        # right end of the domain: x equals the last knot and [left, right] is the last non-empty interval
        if x == t[-1] and right == t[-1]:
            return 1.0
        return 0.0
    den1 = t[j + k - 1] - t[j]
    den2 = t[j + k] - t[j + 1]
    if d == 0:
        out = 0.0
        if den1 > 0:
            out += (x - t[j]) / den1 * _basis(t, j, k - 1, 0, x)
        if den2 > 0:
            out += (t[j + k] - x) / den2 * _basis(t, j + 1, k - 1, 0, x)
        return out
    # derivative recursion: B'_{j,k} = (k-1) [B_{j,k-1}/den1 - B_{j+1,k-1}/den2]
    out = 0.0
    if den1 > 0:
        out += (k - 1) / den1 * _basis(t, j, k - 1, d - 1, x)
    if den2 > 0:
        out -= (k - 1) / den2 * _basis(t, j + 1, k - 1, d - 1, x)
    return out


def collocation(t, order, pts, deriv=0):
    """Matrix M[i, j] = d^deriv B_j / dy^deriv (pts[i])."""
    n = len(t) - order
    M = np.zeros((len(pts), n))
    for i, x in enumerate(pts):
        for j in range(n):
            if t[j] <= x <= t[j + order]:  # outside its support a B-spline and its derivatives vanish
                M[i, j] = _basis(t, j, order, deriv, float(x))
    return M


def dstar(ts, order_s):
    """Exact derivative map D*: coefficients in the order-(p+1) space -> order-p space.

    d/dy sum_j c_j B*_j = sum_i (D* c)_i B_i with
    (D* c)_i = (order_s - 1) (c_{i+1} - c_i) / (t*_{i+order_s} - t*_{i+1}),
    where the order-p knot vector is t* with its first and last knot removed.
    """
    n_s = len(ts) - order_s
    D = np.zeros((n_s - 1, n_s))
    for i in range(n_s - 1):
        h = ts[i + order_s] - ts[i + 1]
        D[i, i] = -(order_s - 1) / h
        D[i, i + 1] = (order_s - 1) / h
    return D


class Basis:
    """All y-operators used by the substage, as dense matrices (small Ny only)."""

    def __init__(self, ny, p, y0=-1.0, y1=1.0):
        self.ny, self.p = ny, p
        self.t = clamped_uniform_knots(p, ny, y0, y1)          # order p, Ny functions
        self.ts = clamped_uniform_knots(p + 1, ny + 1, y0, y1)  # order p+1, Ny+1 functions
        self.g = greville(self.t, p)                            # Ny physical / collocation points
        self.gs = greville(self.ts, p + 1)                      # Ny+1 collocation points of the m2 space
        t, ts, g, gs = self.t, self.ts, self.g, self.gs
        self.Bg = [collocation(t, p, g, d) for d in range(3)]          # B, B', B'' at g
        self.Bs = [collocation(t, p, gs, d) for d in range(4)]         # B..B''' at g*
        self.Sg = [collocation(ts, p + 1, g, d) for d in range(1)]     # B* at g
        self.Ss = [collocation(ts, p + 1, gs, d) for d in range(3)]    # B*, B*', B*'' at g*
        self.D = dstar(ts, p + 1)
