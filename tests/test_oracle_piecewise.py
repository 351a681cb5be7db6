"""Pins of the oracle's piecewise emulator (Eq. 1 with the Teff regimes f1..f5
of section 2.2 stage 2 and the cold/warm/hot models of section 3.1).

Each pin checks the regime logic against something other than itself: the
single-regime oracle built from one regime's table alone (pure ranges), the
linear blend written out by hand (blend ranges), a partition of unity,
continuity across the bounds, finite differences, and recovery of the truth
from noise-free spectra."""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import DEG, TOL, observed, piecewise_model, pw_tables

G = S.SMALL
ROWS = np.cumsum([0] + [len(e) for e in S.PW_EXPS])


def single_regime(r, tables=None):
    tables = pw_tables(G.name) if tables is None else tables
    return O.Model(tables[r], S.PW_EXPS[r], G.dln, G.pad, G.n_pix, DEG, S.PW_BASIS_LO[r],
                   S.PW_BASIS_HI[r], S.PW_BOX_LO, S.PW_BOX_HI)


def th(teff, logg=3.3, feh=-0.4):
    return np.array([teff, logg, feh, 12.0, 80.0])


@pytest.mark.parametrize("teff,r", [(3300.0, 0), (4000.0, 0), (4550.01, 1), (5800.0, 1),
                                     (7000.0, 1), (9000.01, 2), (11800.0, 2)])
def test_pure_range_is_the_single_regime_model(teff, r):
    M = piecewise_model(G)
    phi, dphi = O.basis(M, th(teff))
    phr, dphr = O.basis(single_regime(r), th(teff))
    sl = slice(ROWS[r], ROWS[r + 1])
    np.testing.assert_allclose(phi[sl], phr, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(dphi[sl], dphr, rtol=1e-13, atol=1e-18)
    mask = np.ones(len(phi), bool)
    mask[sl] = False
    assert np.all(phi[mask] == 0.0) and np.all(dphi[mask] == 0.0)


@pytest.mark.parametrize("teff,r,lo,hi", [(4000.5, 0, 4000.0, 4550.0), (4300.0, 0, 4000.0, 4550.0),
                                          (4550.0, 0, 4000.0, 4550.0), (7600.0, 1, 7000.0, 9000.0),
                                          (8999.0, 1, 7000.0, 9000.0)])
def test_blend_is_linear_in_teff(teff, r, lo, hi):
    """F' = (1 - t) F'_r + t F'_{r+1}, t = (Teff - lo) / (hi - lo): the
    weights by hand, each regime's terms from its single-regime model."""
    M = piecewise_model(G)
    phi, dphi = O.basis(M, th(teff))
    t = (teff - lo) / (hi - lo)
    pa, da = O.basis(single_regime(r), th(teff))
    pb, db = O.basis(single_regime(r + 1), th(teff))
    a, b = slice(ROWS[r], ROWS[r + 1]), slice(ROWS[r + 1], ROWS[r + 2])
    np.testing.assert_allclose(phi[a], (1 - t) * pa, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(phi[b], t * pb, rtol=1e-12, atol=1e-15)
    # d/dTeff picks up the weights' slopes -1/(hi-lo) and +1/(hi-lo)
    np.testing.assert_allclose(dphi[a, 0], (1 - t) * da[:, 0] - pa / (hi - lo), rtol=1e-11, atol=1e-16)
    np.testing.assert_allclose(dphi[b, 0], t * db[:, 0] + pb / (hi - lo), rtol=1e-11, atol=1e-16)
    np.testing.assert_allclose(dphi[a, 1:], (1 - t) * da[:, 1:], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(dphi[b, 1:], t * db[:, 1:], rtol=1e-12, atol=1e-16)


def test_weights_are_a_partition_of_unity():
    """Tables whose only non-zero row is each regime's constant term (= 1):
    F' = sum of the weights = 1 and dF'/dTeff = 0 at every Teff."""
    tabs = [np.zeros_like(t) for t in pw_tables(G.name)]
    for t in tabs:
        t[0] = 1.0
    assert all(tuple(e[0]) == (0, 0, 0) for e in S.PW_EXPS)
    M = piecewise_model(G, tables=tabs)
    C = np.concatenate(tabs).astype(np.float64)
    for teff in np.concatenate([np.linspace(3200, 12000, 89), np.array(S.TEFF_BLEND)]):
        phi, dphi = O.basis(M, th(teff))
        Fp = phi @ C
        np.testing.assert_allclose(Fp, 1.0, rtol=0, atol=1e-14)
        np.testing.assert_allclose(dphi[:, 0] @ C, 0.0, atol=1e-15)


@pytest.mark.parametrize("tb", S.TEFF_BLEND)
def test_continuous_across_bounds_with_a_slope_jump(tb):
    M = piecewise_model(G)
    C = np.concatenate(pw_tables(G.name)).astype(np.float64)
    F = lambda teff: O.basis(M, th(teff))[0] @ C
    f0 = F(tb)
    for eps in (1e-3, 1e-5):
        assert np.max(np.abs(F(tb + eps) - f0)) < 50 * eps * np.max(np.abs(f0)) / 100.0
    # one-sided slopes: right FD vs the analytic slope just above, left FD vs
    # the analytic slope at the bound (intervals are closed above)
    h = 1e-4
    right = (F(tb + 2 * h) - F(tb + h)) / h
    left = (F(tb) - F(tb - h)) / h
    dr = O.basis(M, th(tb + 1.5 * h))[1][:, 0] @ C
    dl = O.basis(M, th(tb - 0.5 * h))[1][:, 0] @ C
    np.testing.assert_allclose(right, dr, rtol=1e-4, atol=1e-9)
    np.testing.assert_allclose(left, dl, rtol=1e-4, atol=1e-9)
    assert np.max(np.abs(dr - dl)) > 1e-6          # the kink the paper points to


@pytest.mark.parametrize("teff", [3500.0, 4200.0, 6000.0, 8100.0, 10500.0])
def test_basis_derivative_matches_finite_differences(teff):
    M = piecewise_model(G)
    x = th(teff)
    _, dphi = O.basis(M, x)
    for c, step in ((0, 0.05), (1, 1e-5), (2, 1e-5)):
        xp, xm = x.copy(), x.copy()
        xp[c] += step
        xm[c] -= step
        fd = (O.basis(M, xp)[0] - O.basis(M, xm)[0]) / (2 * step)
        np.testing.assert_allclose(dphi[:, c], fd, rtol=2e-5, atol=1e-10)


def test_noise_free_recovery_across_regimes():
    """Truths in all five Teff ranges, started 100-300 K away: the curvature-
    aware fit and Adam both return the truth."""
    M = piecewise_model(G)
    _, d = observed(G, 10, 31, M=M, noise=False, mask_frac=0.0, teff=(3300.0, 11500.0),
                    box=(S.PW_BOX_LO, S.PW_BOX_HI))
    d["truth"][:5, 0] = [3600.0, 4300.0, 5600.0, 8000.0, 10500.0]
    model = O.model_batch(M, d["truth"], d["b_true"])
    flux, ivar = S.finish_obs(model, d)
    th0 = d["truth"] + np.array([150.0, 0.1, 0.05, 5.0, 5.0]) * np.where(np.arange(10) % 2, 1, -1)[:, None]
    lm = O.fit_lm(M, flux, ivar, d["good"], th0, max_iter=200, rtol=1e-14)
    err = np.abs(lm["theta"] - d["truth"])[:, :4]
    assert np.all(err <= TOL * 0.05), err
    ad = O.fit(M, flux, ivar, d["good"], th0, lr=1e-3, max_steps=20000, tol=1e-10)
    err = np.abs(ad["theta"] - d["truth"])[:, :4]
    assert np.all(err <= TOL), err
