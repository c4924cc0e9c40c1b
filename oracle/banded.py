"""Banded linear solves for the per-mode y-systems (paper Sec. 4.1-4.2, Appendix C).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The solve itself is LAPACK's banded Gaussian elimination with partial pivoting
(scipy.linalg.solve_banded), used as a library primitive. Matrices that depend
on the wavenumber magnitude k^2 are formed as A(k^2) = A2 - k^2 A0 and solved
once per distinct k^2 with all modes sharing it as right-hand sides. The
potential-matching rows of Eq. bc_both, multiplied through by k, add a term
linear in k: A(k) = A2 - k^2 A0 + k A1.
"""
import numpy as np
from scipy.linalg import solve_banded


def bandwidths(A):
    """(kl, ku): number of non-zero sub- and super-diagonals of dense A."""
    rows, cols = np.nonzero(A)
    if rows.size == 0:
        return 0, 0
    return int(max(0, np.max(rows - cols))), int(max(0, np.max(cols - rows)))


def to_band(A, kl, ku):
    """LAPACK band storage: ab[ku + i - j, j] = A[i, j]."""
    n = A.shape[0]
    ab = np.zeros((kl + ku + 1, n))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            ab[ku + i - j, j] = A[i, j]
    return ab


def solve(A, rhs):
    """Solve A x = rhs for one dense banded A and rhs of shape (n, ...)."""
    kl, ku = bandwidths(A)
    shape = rhs.shape
    x = solve_banded((kl, ku), to_band(A, kl, ku), rhs.reshape(shape[0], -1))
    return x.reshape(shape)


def solve_k2(A2, A0, k2, rhs, A1=None):
    """Solve (A2 - k2[m] A0 + sqrt(k2[m]) A1) x[:, m] = rhs[:, m] for every column m.

    A2, A0, A1: dense (n, n) (A1 = None: zero); k2: (M,) wavenumber magnitudes squared;
    rhs: (n, M). Columns that share the same k2 share one LAPACK factorisation.
    """
    if A1 is None:
        A1 = np.zeros_like(A2)
    kl = max(bandwidths(A2)[0], bandwidths(A0)[0], bandwidths(A1)[0])
    ku = max(bandwidths(A2)[1], bandwidths(A0)[1], bandwidths(A1)[1])
    ab2, ab0, ab1 = to_band(A2, kl, ku), to_band(A0, kl, ku), to_band(A1, kl, ku)
    out = np.zeros_like(rhs)
    uniq, inv = np.unique(k2, return_inverse=True)
    for u, val in enumerate(uniq):
        cols = np.nonzero(inv == u)[0]
        out[:, cols] = solve_banded((kl, ku), ab2 - val * ab0 + np.sqrt(val) * ab1, rhs[:, cols])
    return out
