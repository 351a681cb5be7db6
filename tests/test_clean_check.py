"""The Clean-mask validity check (tests/clean_check.py) on the CPU: it accepts
the oracle's own mask, accepts a flip of a pixel whose rule sits within
float32 rounding of its threshold, and rejects a planted mistake in the
oracle's mask anywhere else."""
import numpy as np

from oracle import oracle as O
from tests import clean_check as CC


def _residuals(p, seed):
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(p).astype(np.float32)
    m = np.cumsum(rng.standard_normal(p) * 0.3).astype(np.float32)
    r[40:43] = np.array([30.0, 12.0, 6.0], np.float32)
    return r, m, np.ones(p, np.uint8)


def test_accepts_identical_masks_at_both_shifts():
    for fshift in (0.5, 0.2):
        r, m, used = _residuals(500, 1)
        keep, k = O.clean_mask(r, m, used, fshift)
        ok, nb, why = CC.check(r, m, used, fshift, keep, k, keep, k)
        assert ok and nb == 0, why


def test_rejects_a_planted_mistake_far_from_any_threshold():
    r, m, used = _residuals(500, 2)
    keep, k = O.clean_mask(r, m, used, 0.5)
    q = CC.quantities(r, m, used, 0.5)
    # a kept pixel far below every threshold, away from the flagged run
    j = int(np.argmin(np.abs(q["lhs"][200:300]))) + 200
    assert keep[j] == 1
    bad = keep.copy()
    bad[j] = 0
    ok, _, why = CC.check(r, m, used, 0.5, bad, k, keep, k)
    assert not ok and str(j) in why


def test_accepts_a_flip_at_the_b_threshold():
    p = 400
    rng = np.random.default_rng(3)
    r = rng.standard_normal(p).astype(np.float32)
    m = np.zeros(p, np.float32)
    j = 200
    r[j - 1] = r[j + 1] = np.float32(0.1)
    # put |r_j| on 3 sigma (sigma includes r_j): bisection in double, then the
    # nearest float32; the double-precision comparison is then decided by
    # less than float32 rounding
    lo, hi = 2.0, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        rr = r.astype(np.float64)
        rr[j] = mid
        if mid > 3 * rr.std():
            hi = mid
        else:
            lo = mid
    r[j] = np.float32(hi)
    used = np.ones(p, np.uint8)
    keep, k = O.clean_mask(r, m, used, 0.5)
    q = CC.quantities(r, m, used, 0.5)
    assert abs(q["lhs"][j] - k * q["sigma"]) <= q["tol"][j] + k * q["sigma"] * 8 * CC.EPS32
    flip = keep.copy()
    flip[j] = 1 - flip[j]
    ok, nb, why = CC.check(r, m, used, 0.5, flip, k, keep, k)
    assert ok and nb >= 1, why
