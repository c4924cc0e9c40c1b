"""Pins for oracle/banded.py: against dense numpy solves."""
import numpy as np

from oracle import banded


def _banded(rng, n, kl, ku):
    A = rng.normal(size=(n, n))
    for i in range(n):
        for j in range(n):
            if j < i - kl or j > i + ku:
                A[i, j] = 0
    return A


def test_solve_matches_dense():
    rng = np.random.default_rng(0)
    A = _banded(rng, 40, 3, 2)
    b = rng.normal(size=(40, 5)) + 1j * rng.normal(size=(40, 5))
    x = banded.solve(A, b)
    assert np.abs(A @ x - b).max() < 1e-10
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-10 * np.abs(x).max()
    assert banded.bandwidths(A) == (3, 2)


def test_solve_k2_matches_dense_per_column():
    rng = np.random.default_rng(1)
    n = 30
    A2, A0 = _banded(rng, n, 3, 3), _banded(rng, n, 2, 2)
    k2 = np.array([0.5, 1.0, 4.0, 1.0, 9.0, 0.5])
    b = rng.normal(size=(n, 6)) + 1j * rng.normal(size=(n, 6))
    x = banded.solve_k2(A2, A0, k2, b)
    for m in range(6):
        ref = np.linalg.solve(A2 - k2[m] * A0, b[:, m])
        assert np.abs(x[:, m] - ref).max() < 1e-10 * np.abs(ref).max()
