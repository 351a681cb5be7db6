"""Validity check of a Clean mask (stage 6, Eq. 8) taken in float32 against
the oracle's mask taken in double precision.

The kernel decides each rule on float32 quantities: G_j and |r_j| - f G_j
are rounded, sigma and sigma' are rounded to float32 after double sums.  The
oracle decides the same rules in double precision on the same inputs.  The
two masks may therefore differ only where a comparison of the oracle lies
within float32 rounding of its threshold, and where such a flip propagates:
C and D act on the neighbours of flagged pixels, so a flip spreads only along
a run of pixels flagged in one of the masks, and a flip of B or C membership
moves sigma' slightly.  `check` accepts exactly those differences and
reports the borderline pixels it used.
"""
from __future__ import annotations

import numpy as np

EPS32 = 2.0 ** -24
KS = (3.0, 4.0, 5.0, 7.0)


def _std(r, sel):
    n = int(sel.sum())
    if n == 0:
        return 0.0
    s1 = r[sel].sum()
    s2 = (r[sel] * r[sel]).sum()
    mean = s1 / n
    var = s2 / n - mean * mean
    return float(np.sqrt(var if var > 0 else 0.0))


def quantities(r, m, used, fshift):
    """G, lhs = |r| - f G, sigma, the per-k B counts and the B, C sets of the
    double-precision reading, with the rounding bound of each lhs."""
    r = np.asarray(r, np.float64)
    m = np.asarray(m, np.float64)
    used = np.asarray(used, bool)
    p = len(r)
    G = np.zeros(p)
    G[1:] = np.abs(m[1:] - m[:-1])
    G[:-1] = np.maximum(G[:-1], np.abs(m[:-1] - m[1:]))
    lhs = np.abs(r) - fshift * G
    sigma = _std(r, used)
    # |r| + f G bounds the size of every rounded term of lhs; 8 units of float32
    # rounding cover G, f G, the subtraction and float32 f
    tol = 8 * EPS32 * (np.abs(r) + fshift * G)
    return dict(r=r, G=G, lhs=lhs, sigma=sigma, used=used, tol=tol)


def check(r, m, used, fshift, keep_gpu, k_gpu, keep_ref, k_ref):
    """Returns (ok, n_borderline, why).  ok is True when every pixel where the
    two masks differ is explained by comparisons within float32 rounding."""
    q = quantities(r, m, used, fshift)
    lhs, sigma, used_b, tol, rr = q["lhs"], q["sigma"], q["used"], q["tol"], q["r"]
    keep_gpu = np.asarray(keep_gpu, bool)
    keep_ref = np.asarray(keep_ref, bool)
    if k_gpu != k_ref:
        # the k choice flips only if a count of B outliers can cross 3% of the
        # used pixels by borderline pixels alone
        n_used = used_b.sum()
        for k in KS[:3]:
            thr = k * sigma
            t_k = tol + thr * 8 * EPS32
            sure = np.sum(used_b & (lhs > thr + t_k))
            maybe = np.sum(used_b & (np.abs(lhs - thr) <= t_k))
            if sure <= 0.03 * n_used < sure + maybe:
                return True, int(maybe), f"k {k_ref} vs {k_gpu}: borderline count at k = {k}"
        return False, 0, f"k {k_gpu} (kernel) vs {k_ref} (oracle) with no borderline count"
    diff = np.where(keep_gpu != keep_ref)[0]
    if len(diff) == 0:
        return True, 0, ""
    kb = k_ref * sigma
    t_b = tol + kb * 8 * EPS32
    t_c = tol + 2 * sigma * 8 * EPS32
    B = used_b & (lhs > kb)
    border = used_b & (np.abs(lhs - kb) <= t_b)
    nbB = np.zeros_like(B)
    nbB[1:] |= B[:-1]
    nbB[:-1] |= B[1:]
    C = used_b & ~B & nbB & (lhs > 2 * sigma)
    border |= used_b & nbB & (np.abs(lhs - 2 * sigma) <= t_c)
    # sigma' over used pixels in neither B nor C, and how far toggling the
    # borderline B/C pixels can move it
    sel = used_b & ~(B | C)
    sigp = _std(rr, sel)
    dsig = 0.0
    for j in np.where(border)[0]:
        s2 = sel.copy()
        s2[j] = ~s2[j]
        dsig = max(dsig, abs(_std(rr, s2) - sigp))
    t_d = tol + (sigp * 8 * EPS32 + dsig)
    border |= used_b & (np.abs(lhs - sigp) <= t_d)
    # a flip spreads only through runs flagged in one of the masks: every
    # differing pixel must share such a run with a borderline pixel
    flagged = used_b & ~(keep_gpu & keep_ref)
    p = len(rr)
    run_id = np.full(p, -1)
    rid = 0
    j = 0
    while j < p:
        if flagged[j] or border[j]:
            e = j
            while e + 1 < p and (flagged[e + 1] or border[e + 1]):
                e += 1
            run_id[j:e + 1] = rid
            rid += 1
            j = e + 1
        else:
            j += 1
    runs_with_border = set(run_id[border & (run_id >= 0)])
    bad = [int(j) for j in diff if run_id[j] < 0 or run_id[j] not in runs_with_border]
    if bad:
        return False, int(border.sum()), f"pixels {bad[:8]} differ with no borderline comparison"
    return True, int(border[diff].sum() if len(diff) else 0), f"{len(diff)} pixels differ at borderline"
