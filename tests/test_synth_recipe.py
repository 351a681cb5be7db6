"""The seeded input generator follows the recipe the design notes state for
the synthetic stand-ins of LAMOST-like and DESI-like spectra (CPU only):
grids, parameter ranges, continua, signal-to-noise, masks, initial values and
the observed flux and inverse variance."""
import math

import numpy as np

import lasp_synth as S


def test_grids():
    lam = S.LAMOST.wavelengths()
    assert S.LAMOST.n_pix == 3909 and abs(lam[0] - 3700.0) < 1e-9 and abs(lam[-1] - 9000.0) < 1e-6
    lam = S.DESI.wavelengths()
    assert S.DESI.n_pix == 7781 and abs(lam[0] - 3600.0) < 1e-9 and abs(lam[-1] - 9824.0) < 1e-6
    assert S.SMALL.n_pix == 1024 and S.SMALL.lam0 == 4200.0 and S.SMALL.dln == S.LAMOST.dln
    assert abs(S.LAMOST.kms_per_px - 68.19) < 0.01 and abs(S.DESI.kms_per_px - 38.68) < 0.01
    # the margin covers the widest kernel of the box: ceil(max|RV|/v_px + 5 max sigma/v_px)
    for g in (S.LAMOST, S.DESI, S.SMALL):
        v = g.kms_per_px
        assert g.pad == math.ceil(300.0 / v + 5.0 * 200.0 / v)
    assert (S.LAMOST.pad, S.DESI.pad) == (20, 34)


def test_draws_follow_the_recipe():
    g, n = S.LAMOST, 3000
    d = S.draw_batch(g, n, 77)
    t = d["truth"]
    for k, (lo, hi) in enumerate([(4000, 7000), (1, 5), (-2, 0.5), (-200, 200), (50, 150)]):
        assert t[:, k].min() >= lo and t[:, k].max() <= hi
    # continuum scale log-uniform on [0.1, 100]
    ls = np.log(d["b_true"][:, 0])
    assert ls.min() >= math.log(0.1) - 1e-12 and ls.max() <= math.log(100.0) + 1e-12
    assert abs(ls.mean() - 0.5 * (math.log(0.1) + math.log(100.0))) < 0.05 * math.log(1000.0)
    # sum |beta| <= 0.8, so the continuum stays >= 0.2 of its scale over the grid
    beta = d["b_true"][:, 1:] / d["b_true"][:, :1]
    assert np.abs(beta).sum(axis=1).max() <= 0.8 + 1e-12
    x = np.linspace(-1.0, 1.0, 201)
    P = np.polynomial.legendre.legvander(x, 6)
    cont = (P @ d["b_true"].T).T / d["b_true"][:, :1]
    assert cont.min() >= 0.2 - 1e-12
    # SNR log-uniform on [5, 100]
    lsnr = np.log(d["snr"])
    assert lsnr.min() >= math.log(5.0) - 1e-12 and lsnr.max() <= math.log(100.0) + 1e-12
    assert abs(lsnr.mean() - 0.5 * (math.log(5.0) + math.log(100.0))) < 0.05 * math.log(20.0)
    # 5% masked in runs (every masked run at least 3 pixels), Na D 5885-5900 A always masked
    masked = 1.0 - d["good"].mean(axis=1)
    assert masked.min() >= 0.05 - 0.5 / g.n_pix and masked.max() <= 0.05 + 13.0 / g.n_pix
    nad = (g.wavelengths() >= 5885.0) & (g.wavelengths() <= 5900.0)
    assert nad.sum() >= 3 and np.all(d["good"][:, nad] == 0)
    for row in d["good"][:50]:
        edges = np.flatnonzero(np.diff(np.r_[1, row, 1].astype(int)))
        runs = edges[1::2] - edges[0::2]
        assert runs.min() >= 3
    # initial values: truth + N(0, (200 K, 0.3, 0.2, 15 km/s, 20 km/s)), clipped to the box
    dt = d["theta0"] - t
    inside = (d["theta0"] > S.BOX_LO) & (d["theta0"] < S.BOX_HI)
    for k, sd in enumerate((200.0, 0.3, 0.2, 15.0, 20.0)):
        assert abs(dt[inside[:, k], k].std() / sd - 1.0) < 0.1, k
    assert np.all(d["theta0"] >= S.BOX_LO) and np.all(d["theta0"] <= S.BOX_HI)


def test_observations_from_a_model():
    g, n = S.SMALL, 40
    d = S.draw_batch(g, n, 78, mask_frac=0.05)
    rng = np.random.default_rng(3)
    model = 1.0 + 0.2 * rng.random((n, g.n_pix))
    flux, ivar = S.finish_obs(model, d)
    bad = d["good"] == 0
    med = np.median(model, axis=1, keepdims=True)
    assert np.all(ivar[bad] == 0.0)
    np.testing.assert_allclose(flux[bad], np.broadcast_to(50.0 * med, bad.shape)[bad], rtol=1e-6)
    # photon-like noise: sigma = (median / SNR) sqrt(max(model, 0.05 median) / median)
    sigma = (med / d["snr"][:, None]) * np.sqrt(np.maximum(model, 0.05 * med) / med)
    np.testing.assert_allclose(ivar[~bad], (1.0 / sigma ** 2)[~bad], rtol=1e-6)
    np.testing.assert_allclose(flux[~bad], (model + sigma * d["z"])[~bad], rtol=1e-6)
    d0 = S.draw_batch(g, n, 78, mask_frac=0.05, noise=False)
    flux0, _ = S.finish_obs(model, d0)
    ok0 = d0["good"] == 1
    np.testing.assert_array_equal(flux0[ok0], model.astype(np.float32)[ok0])


def test_seeded_and_deterministic():
    a = S.draw_batch(S.SMALL, 8, 5)
    b = S.draw_batch(S.SMALL, 8, 5)
    c = S.draw_batch(S.SMALL, 8, 6)
    for k in ("truth", "b_true", "theta0", "snr", "z", "good"):
        np.testing.assert_array_equal(a[k], b[k])
    assert not np.array_equal(a["truth"], c["truth"])
    C1, C2 = S.make_table(S.SMALL), S.make_table(S.SMALL)
    assert C1.dtype == np.float32 and C1.shape == (26, S.SMALL.n_model)
    np.testing.assert_array_equal(C1, C2)
    assert np.all(np.isfinite(C1))
