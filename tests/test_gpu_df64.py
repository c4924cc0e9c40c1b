"""GPU: the conversions at the spectral ends of the double-float transforms (precision 1), run through
lmvd_df64_convert on the device code itself and checked against exact arithmetic.

Split x -> (hi, lo): the pair is normalised (|lo| <= ulp(hi) / 2) and hi + lo, exact in binary64 here
(its bits are a subset of x's), is within 2^-48 |x| of x for 2^-102 <= |x| < 2^128; below that the
absolute error stays below 2^-126; the special values keep their meaning.
Rounding (hi, lo) -> double: the exact sum hi + lo (fractions.Fraction) when it is a double, within one
unit of the last place of the correctly rounded sum otherwise; inf, nan and signed zeros are kept.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available()
    from paper_2206_09878_gb300 import lmvd
    return lmvd


def _run(L, x, pair_hi, pair_lo):
    dev = torch.device("cuda")
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(dev)
    ph = torch.from_numpy(np.ascontiguousarray(pair_hi, dtype=np.float32)).to(dev)
    pl = torch.from_numpy(np.ascontiguousarray(pair_lo, dtype=np.float32)).to(dev)
    hi = torch.empty(len(x), dtype=torch.float32, device=dev)
    lo = torch.empty_like(hi)
    s = torch.empty(len(x), dtype=torch.float64, device=dev)
    L.lmvd_df64_convert(xt, hi, lo, ph, pl, s)
    torch.cuda.synchronize()
    return hi.cpu().numpy(), lo.cpu().numpy(), s.cpu().numpy()


def _random_doubles(n, lo_exp, hi_exp, seed):
    rng = np.random.default_rng(seed)
    m = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    return np.ldexp(m, rng.integers(lo_exp, hi_exp, n))


def test_split_is_normalised_and_within_2_pow_minus_48(L):
    x = np.concatenate([_random_doubles(20000, -102, 127, 1),
                        [1.0, -1.0, 1 - 2.0 ** -53, 1 + 2.0 ** -52, 0.1, -1.0 / 3.0, 2.0 ** -102, 3.4e38]])
    n = len(x)
    hi, lo, _ = _run(L, x, np.zeros(n), np.zeros(n))
    total = hi.astype(np.float64) + lo.astype(np.float64)   # exact: the pair's bits are x's
    rel = np.abs(total - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -48, rel.max()
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    assert np.all(np.abs(lo.astype(np.float64)) <= ulp / 2)
    assert np.all(np.signbit(hi) == np.signbit(x))


def test_split_special_values(L):
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 2.0 ** 128, -1e300, 1e-300, -2.0 ** -127, 2.0 ** -110])
    n = len(x)
    hi, lo, _ = _run(L, x, np.zeros(n), np.zeros(n))
    assert hi[0] == 0 and not np.signbit(hi[0]) and lo[0] == 0
    assert hi[1] == 0 and np.signbit(hi[1]) and lo[1] == 0
    assert hi[2] == np.inf and hi[3] == -np.inf and np.isnan(hi[4])
    assert hi[5] == np.inf and hi[6] == -np.inf
    assert hi[7] == 0 and hi[8] == 0 and np.signbit(hi[8])                 # below 2^-126: signed zero
    total = float(hi[9]) + float(lo[9])                                    # 2^-126 <= |x| < 2^-102
    assert abs(total - x[9]) <= 2.0 ** -126


def test_pair_rounding_against_exact_sum(L):
    rng = np.random.default_rng(7)
    n = 20000
    hi = _random_doubles(n, -100, 100, 2).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    # lo: normalised (|lo| <= ulp(hi) / 2) with a random exponent gap below ulp(hi), either sign; most
    # gaps put bits of lo below the double's last place of hi (then the result is rounded)
    gap = rng.integers(1, 60, n)
    lo = (rng.uniform(-0.5, 0.5, n) * ulp * np.ldexp(1.0, -gap + 1)).astype(np.float32)
    lo = np.where(np.abs(lo.astype(np.float64)) <= ulp / 2, lo, np.float32(0))
    _, _, got = _run(L, np.zeros(n), hi, lo)
    exact_hits = 0
    for h, l, g in zip(hi, lo, got):
        exact = Fraction(float(h)) + Fraction(float(l))
        nearest = float(exact)                      # correctly rounded
        if Fraction(nearest) == exact:
            assert g == nearest, (h, l, g, nearest)
            exact_hits += 1
        else:
            assert abs(Fraction(g) - exact) <= Fraction(math.ulp(nearest)), (h, l, g, nearest)
    # hi + lo is a double when lo's last bit is not below the double's last place of hi: exponent gaps of
    # up to about 6 bits below ulp(hi) (lo carries 24 bits of its own), about a tenth of the draws
    assert exact_hits > n // 20


def test_pair_rounding_special_values(L):
    hi = np.array([np.inf, -np.inf, np.nan, 0.0, -0.0, 1e-40, -3e-45], dtype=np.float32)
    lo = np.zeros(len(hi), dtype=np.float32)
    _, _, got = _run(L, np.zeros(len(hi)), hi, lo)
    assert got[0] == np.inf and got[1] == -np.inf and np.isnan(got[2])
    assert got[3] == 0 and not np.signbit(got[3]) and got[4] == 0 and np.signbit(got[4])
    assert got[5] == float(hi[5]) and got[6] == float(hi[6])               # denormal hi: exact
