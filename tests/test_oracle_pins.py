"""Pins of the FP64 oracle to facts fixed outside it (CPU only).

Each test checks one part of the oracle against a closed form, an invariant,
a library routine the oracle does not use, or brute force, chosen so that a
dropped term, a wrong sign or index or a transposed operand fails a test.
The paper prints no worked example, so no value here is quoted from it.
"""
import math

import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import DEG, observed, oracle_model

G = S.SMALL


def _model(C=None):
    return oracle_model(G, C)


# ---------------------------------------------------------------- basis (Eq. 1)

def test_basis_box_corners_closed_form():
    M = _model()
    lo = np.array([3500.0, 0.5, -2.5, 0.0, 100.0])
    hi = np.array([7500.0, 5.5, 1.0, 0.0, 100.0])
    phi_lo, _ = O.basis(M, lo)
    phi_hi, _ = O.basis(M, hi)
    deg = S.EXPS.sum(axis=1)
    np.testing.assert_allclose(phi_lo, (-1.0) ** deg, atol=1e-13)
    np.testing.assert_allclose(phi_hi, np.ones(S.K_TERMS), atol=1e-13)
    mid = np.array([10 ** ((math.log10(3500) + math.log10(7500)) / 2), 3.0, -0.75, 0, 100])
    phi_mid, _ = O.basis(M, mid)
    expect = np.where(deg == 0, 1.0, 0.0)            # every u = 0 at the box centre
    np.testing.assert_allclose(phi_mid, expect, atol=1e-13)


def test_single_term_table_reproduces_basis():
    """A table whose only non-zero row k is all ones gives F' = phi_k."""
    rng = np.random.default_rng(1)
    th = np.array([5321.0, 2.7, -0.9, 0.0, 100.0])
    for k in rng.choice(S.K_TERMS, 6, replace=False):
        C = np.zeros((S.K_TERMS, G.n_model))
        C[k] = 1.0
        out = O.model_flux(_model(C), th, np.r_[1.0, np.zeros(DEG)])
        phi, _ = O.basis(_model(C), th)
        np.testing.assert_allclose(out["Fp"], phi[k], rtol=0, atol=1e-14)


def test_basis_derivative_fd():
    M = _model()
    th = np.array([4810.0, 3.9, -1.3, 0.0, 100.0])
    phi, dphi = O.basis(M, th)
    for i, h in enumerate([1e-3, 1e-6, 1e-6]):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (O.basis(M, tp)[0] - O.basis(M, tm)[0]) / (2 * h)
        np.testing.assert_allclose(dphi[:, i], fd, rtol=1e-6, atol=1e-9)


# ------------------------------------------------------------ kernel (Eq. 5)

@pytest.mark.parametrize("mu,sig", [(0.0, 0.8), (1.37, 1.1), (-2.9, 2.2), (4.4, 2.93), (0.3, 0.5)])
def test_kernel_unit_sum_support_and_mirror(mu, sig):
    H = 20
    g, dm, ds, h = O.kernel(mu, sig, H)
    assert h == math.ceil(abs(mu) + 5 * sig)
    assert abs(g.sum() - 1.0) < 1e-15
    s = np.arange(-H, H + 1)
    assert np.all(g[np.abs(s) > h] == 0.0)
    assert np.all(g[np.abs(s) <= h] > 0.0)
    gm, _, _, _ = O.kernel(-mu, sig, H)
    np.testing.assert_allclose(g, gm[::-1], atol=1e-16)
    # derivatives of a unit-sum kernel sum to zero
    assert abs(dm.sum()) < 1e-13 and abs(ds.sum()) < 1e-13


def test_kernel_derivative_fd():
    H = 20
    for mu, sig in [(1.3, 1.7), (-0.6, 0.9)]:
        g, dm, ds, _ = O.kernel(mu, sig, H)
        e = 1e-6
        fdm = (O.kernel(mu + e, sig, H)[0] - O.kernel(mu - e, sig, H)[0]) / (2 * e)
        fds = (O.kernel(mu, sig + e, H)[0] - O.kernel(mu, sig - e, H)[0]) / (2 * e)
        np.testing.assert_allclose(dm, fdm, atol=1e-9)
        np.testing.assert_allclose(ds, fds, atol=1e-9)


def _kms(px):
    return px * G.kms_per_px


def test_broadening_equals_numpy_convolution():
    """Eq. 5 as a convolution: F'' = np.convolve(F', G, 'valid')."""
    M = _model()
    th = np.array([5100.0, 2.2, -0.4, 47.0, 91.0])
    out = O.model_flux(M, th, np.r_[1.0, np.zeros(DEG)])
    g, _, _, _ = O.kernel(th[3] / G.kms_per_px, th[4] / G.kms_per_px, G.pad)
    np.testing.assert_allclose(out["Fpp"], np.convolve(out["Fp"], g, mode="valid"), atol=1e-13)


def test_broadening_identity_and_integer_shift():
    M = _model()
    b = np.r_[1.0, np.zeros(DEG)]
    base = np.array([5600.0, 4.1, -0.2, 0.0, 0.0])
    for shift in (0, 3, -5):
        th = base.copy()
        th[3] = _kms(shift)
        th[4] = _kms(1e-4)                            # sigma -> 0: a unit spike at s = shift
        out = O.model_flux(M, th, b)
        H = G.pad
        np.testing.assert_allclose(out["Fpp"], out["Fp"][H - shift:H - shift + G.n_pix],
                                   rtol=0, atol=1e-12)


def test_broadening_constant_in_constant_out():
    C = np.zeros((S.K_TERMS, G.n_model))
    C[0] = 2.5
    out = O.model_flux(_model(C), np.array([6000.0, 3, 0, 120.0, 140.0]), np.r_[1.0, np.zeros(DEG)])
    np.testing.assert_allclose(out["Fpp"], 2.5, atol=1e-14)


def test_broadening_moments_add():
    """Mean and variance of an isolated line add under convolution; a positive
    RV moves the line to higher pixel index by the kernel mean (~ mu)."""
    C = np.zeros((S.K_TERMS, G.n_model))
    m = np.arange(G.n_model)
    C[0] = np.exp(-0.5 * ((m - 500.3) / 1.7) ** 2)
    M = _model(C)
    th = np.array([6000.0, 3, 0, _kms(2.6), _kms(1.3)])
    out = O.model_flux(M, th, np.r_[1.0, np.zeros(DEG)])
    g, _, _, _ = O.kernel(th[3] / G.kms_per_px, th[4] / G.kms_per_px, G.pad)
    s = np.arange(-G.pad, G.pad + 1)
    j = np.arange(G.n_pix)
    Fp, Fpp = out["Fp"], out["Fpp"]
    mean_in = (m * Fp).sum() / Fp.sum() - G.pad          # in observed-pixel units
    var_in = ((m - G.pad - mean_in) ** 2 * Fp).sum() / Fp.sum()
    mean_out = (j * Fpp).sum() / Fpp.sum()
    var_out = ((j - mean_out) ** 2 * Fpp).sum() / Fpp.sum()
    gmean = (s * g).sum()
    gvar = ((s - gmean) ** 2 * g).sum()
    assert abs(mean_out - (mean_in + gmean)) < 1e-9
    assert abs(var_out - (var_in + gvar)) < 1e-8
    assert abs(gmean - 2.6) < 1e-6 and mean_out > mean_in


# --------------------------------------------------------- continuum (Eq. 6)

@pytest.mark.parametrize("D", [2, 4, 6, 8])
def test_legendre_matches_numpy(D):
    p = 1024
    x = -1.0 + 2.0 * np.arange(p) / p
    np.testing.assert_allclose(O.legendre(p, D), np.polynomial.legendre.legvander(x, D),
                               atol=1e-13)


@pytest.mark.parametrize("DEG", [2, 4, 6, 8])
def test_wls_matches_lstsq_and_envelope(DEG):
    """Every continuum degree the CUDA path supports (degree 8 fills the
    oracle's largest normal-equation buffers)."""
    M, d = observed(G, 3, 11, noise=True, snr=(20, 20), mask_frac=0.05)
    M = oracle_model(G, deg=DEG)
    for i in range(3):
        y, W, w, _ = O.prep(d["flux"][i], d["ivar"][i], d["good"][i])
        x = O.x_from_phys(M, d["theta0"][i])
        r = O.evaluate(M, y, W, x)
        th = O.phys_from_x(M, x)
        Fpp = O.model_flux(M, th, np.r_[1.0, np.zeros(DEG)])["Fpp"]
        X = np.polynomial.legendre.legvander(-1.0 + 2.0 * np.arange(G.n_pix) / G.n_pix, DEG)
        X = X * Fpp[:, None]
        sw = np.sqrt(W)
        b_ls = np.linalg.lstsq(X * sw[:, None], y * sw, rcond=None)[0]
        np.testing.assert_allclose(r["b"], b_ls, rtol=1e-9, atol=1e-12)
        # dS/db = 0 at b*: S(b) = sum W (y - (P b) F'')^2
        def S_of(b):
            return float((W * (y - O.model_flux(M, th, b)["model"]) ** 2).sum())
        S0 = S_of(r["b"])
        for k in range(DEG + 1):
            e = np.zeros(DEG + 1)
            e[k] = 1e-4 * max(1.0, abs(r["b"][0]))
            dS = (S_of(r["b"] + e) - S_of(r["b"] - e)) / (2 * e[k])
            assert abs(dS) < 1e-6 * max(S0, 1e-12) / e[k] + 1e-9


def test_loss_is_rms_of_weighted_residual():
    M, d = observed(G, 1, 12, noise=True, snr=(30, 30), mask_frac=0.05)
    y, W, w, n_obj = O.prep(d["flux"][0], d["ivar"][0], d["good"][0])
    r = O.evaluate(M, y, W, O.x_from_phys(M, d["theta0"][0]))
    assert abs(r["loss"] - math.sqrt((W * r["eps"] ** 2).sum() / G.n_pix)) < 1e-14
    # masked pixels carry weight 0 and their spike values never reach the loss
    assert np.all(W[d["good"][0] == 0] == 0)


# ------------------------------------------------------------ prep (sec. 3.3)

def test_prep_quantile_and_weights():
    M, d = observed(G, 1, 13, noise=True, snr=(15, 15), mask_frac=0.1)
    f, iv, gd = d["flux"][0], d["ivar"][0], d["good"][0]
    used = (gd == 1) & (iv > 0)
    for q in (0.5, 0.75):
        y, W, w, n_obj = O.prep(f, iv, gd, quantile=q)
        assert abs(w - np.quantile(f[used].astype(np.float64), q)) < 1e-12 * abs(w)
        assert n_obj == used.sum()
        assert abs(W[used].mean() - 1.0) < 1e-12
        np.testing.assert_allclose(y[used], f[used].astype(np.float64) / w, rtol=1e-15)
    y, W, w, n_obj = O.prep(f, iv, gd, edge_px=7)
    assert np.all(W[:7] == 0) and np.all(W[-7:] == 0) and n_obj == used[7:-7].sum()


# --------------------------------------------------------- loss and gradient

def test_zero_loss_at_truth_noise_free():
    M, d = observed(G, 4, 14, noise=False, mask_frac=0.0)
    for i in range(4):
        y, W, w, _ = O.prep(d["flux"][i], d["ivar"][i], d["good"][i])
        r = O.evaluate(M, y, W, O.x_from_phys(M, d["truth"][i]))
        assert r["loss"] < 2e-7          # float32 storage of the flux is the floor
        # the continuum recovers the true one up to the scale fixed by w
        np.testing.assert_allclose(r["b"] * w, d["b_true"][i], rtol=2e-6, atol=2e-6 * w)


def test_flux_scale_invariance():
    M, d = observed(G, 1, 15, noise=True, snr=(25, 25), mask_frac=0.05)
    y1, W1, _, _ = O.prep(d["flux"][0], d["ivar"][0], d["good"][0])
    y2, W2, _, _ = O.prep(d["flux"][0] * np.float32(8.0), d["ivar"][0] / np.float32(64.0),
                          d["good"][0])
    x = O.x_from_phys(M, d["theta0"][0])
    r1, r2 = O.evaluate(M, y1, W1, x), O.evaluate(M, y2, W2, x)
    assert abs(r1["loss"] - r2["loss"]) < 1e-13
    np.testing.assert_allclose(r1["grad"], r2["grad"], rtol=1e-10, atol=1e-14)


def _richardson(fun, x, k, h):
    def cd(hh):
        xp, xm = x.copy(), x.copy()
        xp[k] += hh
        xm[k] -= hh
        return (fun(xp) - fun(xm)) / (2 * hh)
    return (4 * cd(h / 2) - cd(h)) / 3


def test_gradient_matches_finite_differences():
    M, d = observed(G, 3, 16, noise=True, snr=(40, 40), mask_frac=0.05)
    for i in range(3):
        y, W, _, _ = O.prep(d["flux"][i], d["ivar"][i], d["good"][i])
        x = O.x_from_phys(M, d["theta0"][i])
        r = O.evaluate(M, y, W, x)
        fd = np.array([_richardson(lambda z: O.evaluate(M, y, W, z)["loss"], x, k, 1e-4)
                       for k in range(5)])
        np.testing.assert_allclose(r["grad"], fd, rtol=1e-7, atol=1e-10 * np.abs(fd).max())


def test_model_vjp_matches_finite_differences():
    """Adjoint of model = (P b) * (G (x) phi C) w.r.t. theta and b."""
    M = _model()
    rng = np.random.default_rng(3)
    th = np.array([5480.0, 3.3, -0.7, 63.0, 88.0])
    b = np.r_[1.3, rng.normal(0, 0.05, DEG)]
    gm = rng.normal(0, 1, G.n_pix)
    gth, gb = O.model_vjp(M, th, b, gm)
    f = lambda t, bb: float(gm @ O.model_flux(M, t, bb)["model"])
    steps = [0.5, 1e-4, 1e-4, 0.01, 0.01]
    fd_th = np.array([_richardson(lambda t: f(t, b), th, k, steps[k]) for k in range(5)])
    fd_b = np.array([_richardson(lambda bb: f(th, bb), b, k, 1e-3) for k in range(DEG + 1)])
    np.testing.assert_allclose(gth, fd_th, rtol=1e-7)
    np.testing.assert_allclose(gb, fd_b, rtol=1e-9)


# ------------------------------------------------------------- Adam (stage 8)

def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x0 = rng.uniform(-0.5, 0.5, 5)
    grads = rng.normal(0, 1, (30, 5)) * np.array([1e-3, 1, 10, 1e-2, 5])
    p = torch.nn.Parameter(torch.tensor(x0, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=0.1)
    x, m, v = x0.copy(), np.zeros(5), np.zeros(5)
    for t, g in enumerate(grads, start=1):
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        x, m, v = O.adam_update(x, m, v, g, t, clamp=False)
        np.testing.assert_allclose(x, p.detach().numpy(), rtol=0, atol=1e-12)


def test_adam_box_projection():
    x, m, v = O.adam_update(np.array([0.99, -0.99, 0, 0, 0]), np.zeros(5), np.zeros(5),
                            np.array([-1.0, 1.0, 0, 0, 0]), 1)
    assert x[0] == 1.0 and x[1] == -1.0


def test_stop_rules():
    W = 50
    flat = np.r_[np.linspace(1.0, 0.5, 10), np.full(200, 0.5)]
    # first t >= 50 with |l_t - l_{t-50}| < tol: l_{t-50} on the flat part, t - 50 >= 9
    stops = [t for t in range(len(flat)) if O.stop_rule(flat, t, W, 1e-5, 5000)]
    assert stops[0] == 59 and O.stop_rule(flat, 59, W, 1e-5, 5000) == O.ST_CONV_TOL
    rising = 1.0 + 1e-3 * np.arange(120)
    assert O.stop_rule(rising, 49, W, 1e-5, 5000) == 0
    assert O.stop_rule(rising, 50, W, 1e-5, 5000) == O.ST_CONV_RISE
    one_flat = rising.copy()
    one_flat[30] = one_flat[29]               # a tie breaks the run of rises
    assert O.stop_rule(one_flat, 79, W, 1e-5, 5000) == 0
    assert O.stop_rule(one_flat, 80, W, 1e-5, 5000) == O.ST_CONV_RISE
    falling = 1.0 - 1e-4 * np.arange(300)     # changes by 5e-3 per window: never tol
    assert all(O.stop_rule(falling, t, W, 1e-5, 250) == 0 for t in range(250))
    assert O.stop_rule(falling, 250, W, 1e-5, 250) == O.ST_MAXSTEPS
    tie = np.r_[np.zeros(50), 1e-5]           # |delta| == tol does not stop (strict <)
    assert O.stop_rule(tie, 50, W, 1e-5, 5000) == 0


# -------------------------------------------------------------- end to end

def test_noise_free_recovery_of_truth():
    M, d = observed(G, 8, 17, noise=False, mask_frac=0.0)
    res = O.fit(M, d["flux"], d["ivar"], d["good"], d["theta0"], lr=1e-3, tol=1e-10,
                max_steps=20000)
    err = np.abs(res["theta"] - d["truth"])
    assert np.all(err[:, :4] <= np.array([1.0, 0.005, 0.005, 0.1])), err
    assert np.all(res["loss"] < 1e-4)


def test_fit_step_accounting_and_status():
    M, d = observed(G, 4, 18, noise=True, snr=(20, 60), mask_frac=0.05)
    res = O.fit(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_steps=40)
    assert np.all(res["steps"] == 40) and np.all(res["status"] & O.ST_MAXSTEPS)
    xs, ls = O.trajectory(M, d["flux"][0], d["ivar"][0], d["good"][0], d["theta0"][0], 40)
    np.testing.assert_allclose(O.x_from_phys(M, res["theta"][0]), xs[40], atol=1e-12)
    assert abs(res["loss"][0] - ls[40]) < 1e-15
    bad = d["good"].copy()
    bad[1] = 0
    res2 = O.fit(M, d["flux"], d["ivar"], bad, d["theta0"], max_steps=40)
    assert res2["status"][1] == O.ST_NODATA and res2["steps"][1] == 0


# ----------------------------------------------------------- errors (stage 9)

def test_errors_jacobian_consistent_with_gradient():
    """J^T r / (p l) equals the analytic gradient of l (envelope theorem)."""
    M, d = observed(G, 2, 19, noise=True, snr=(30, 30), mask_frac=0.05)
    for i in range(2):
        th = d["theta0"][i]
        e = O.errors(M, d["flux"][i], d["ivar"][i], d["good"][i], th, with_jac=True)
        y, W, _, n_obj = O.prep(d["flux"][i], d["ivar"][i], d["good"][i])
        r = O.evaluate(M, y, W, O.x_from_phys(M, th))
        resid = np.sqrt(W) * r["eps"]
        gphys = r["grad"] / (0.5 * (S.BOX_HI - S.BOX_LO))
        np.testing.assert_allclose(e["jac"].T @ resid / (G.n_pix * r["loss"]), gphys,
                                   rtol=2e-5, atol=1e-6 * np.abs(gphys).max())
        s2 = (resid ** 2).sum() / (n_obj - 5)
        np.testing.assert_allclose(e["cov"], s2 * np.linalg.inv(e["jac"].T @ e["jac"]),
                                   rtol=1e-9)
        np.testing.assert_allclose(e["sigma"], np.sqrt(np.diag(e["cov"])), rtol=1e-12)


def test_errors_jacobian_is_the_schur_complement_of_the_full_problem():
    """Stage 9 differentiates sqrt(W) eps with the continuum re-solved at each
    point (variable projection).  Where the residual is zero (noise-free data
    at the truth) that Jacobian's normal matrix equals the Schur complement of
    the normal matrix of the full problem in (theta, b), A_tt - A_tb A_bb^-1
    A_bt (Golub and Pereyra), so its inverse is the theta block of the full
    inverse.  The full Jacobian is taken here by central differences of the
    forward model alone, b held at the oracle's solve.  Agreement is 1e-10 on
    these spectra; the fixed-continuum matrix A_tt misses it by a factor of
    10 or more, so a Jacobian that dropped the re-solve fails."""
    half = 0.5 * (S.BOX_HI - S.BOX_LO)
    for seed in (23, 24):
        M, d = observed(G, 1, seed, noise=False, mask_frac=0.05)
        th = d["truth"][0]
        flux, ivar, good = d["flux"][0], d["ivar"][0], d["good"][0]
        J = O.errors(M, flux, ivar, good, th, with_jac=True)["jac"]
        y, W, _, _ = O.prep(flux, ivar, good)
        b = O.evaluate(M, y, W, O.x_from_phys(M, th))["b"]
        res = lambda t, c: np.sqrt(W) * (y - O.model_flux(M, t, c)["model"])
        cols = []
        for k in range(5):
            step = np.zeros(5)
            step[k] = 1e-4 * half[k]
            cols.append((res(th + step, b) - res(th - step, b)) / (2 * step[k]))
        for k in range(len(b)):
            step = np.zeros(len(b))
            step[k] = 1e-4 * max(abs(b[k]), 1e-3)
            cols.append((res(th, b + step) - res(th, b - step)) / (2 * step[k]))
        A = np.column_stack(cols).T @ np.column_stack(cols)
        schur = A[:5, :5] - A[:5, 5:] @ np.linalg.solve(A[5:, 5:], A[5:, :5])
        scale = np.sqrt(np.outer(np.diag(schur), np.diag(schur)))
        assert np.max(np.abs(J.T @ J - schur) / scale) < 1e-7
        assert np.max(np.abs(A[:5, :5] - schur) / scale) > 1.0
        full_inv = np.linalg.inv(A)[:5, :5]
        iscale = np.sqrt(np.outer(np.diag(full_inv), np.diag(full_inv)))
        assert np.max(np.abs(np.linalg.inv(J.T @ J) - full_inv) / iscale) < 1e-6


def test_errors_vanish_without_noise():
    M, d = observed(G, 1, 20, noise=False, mask_frac=0.0)
    e = O.errors(M, d["flux"][0], d["ivar"][0], d["good"][0], d["truth"][0])
    assert np.all(e["sigma"] < np.array([0.05, 1e-4, 1e-4, 5e-3, 5e-3]))


def test_errors_match_monte_carlo_scatter():
    """Sample scatter of the fitted parameters over noise realisations agrees
    with the median reported sigma (linear error propagation, stage 9)."""
    n = 96
    M = oracle_model(G)
    d = S.draw_batch(G, n, 21, noise=True, snr=(40, 40), mask_frac=0.0)
    for k in ("truth", "b_true", "theta0", "snr"):
        d[k] = np.repeat(d[k][:1], n, axis=0)
    d["good"] = np.repeat(d["good"][:1], n, axis=0)
    model = O.model_batch(M, d["truth"][:1], d["b_true"][:1])
    flux, ivar = S.finish_obs(np.repeat(model, n, axis=0), d)
    res = O.fit(M, flux, ivar, d["good"], d["truth"], lr=3e-3, tol=1e-10, max_steps=3000)
    sig = np.array([O.errors(M, flux[i], ivar[i], d["good"][i], res["theta"][i])["sigma"]
                    for i in range(0, n, 8)])
    ratio = res["theta"].std(axis=0, ddof=1) / np.median(sig, axis=0)
    assert np.all((ratio > 0.7) & (ratio < 1.3)), ratio


# ------------------------------------------- resampling (stage 3, Eqs. 2-4)

def _bins(n_out, ln0, dln):
    return np.exp(ln0 + (np.arange(n_out + 1) - 0.5) * dln)


def _brute_resample(F, lam1, dlam, edges, sub=200):
    """Average of the piecewise-constant model over each target bin by direct
    numerical integration on a fine subgrid (independent of Eqs. 2-4)."""
    out = np.zeros(len(edges) - 1)
    for i in range(len(edges) - 1):
        xs = np.linspace(edges[i], edges[i + 1], sub + 1)
        mid = 0.5 * (xs[1:] + xs[:-1])
        k = np.floor((mid - (lam1 - 0.5 * dlam)) / dlam).astype(int)
        val = np.where((k >= 0) & (k < len(F)), F[np.clip(k, 0, len(F) - 1)], 0.0)
        out[i] = val.mean()
    return out


def test_resample_conserves_flux_and_constants():
    rng = np.random.default_rng(9)
    lam1, dlam, q = 4100.0, 0.4, 5000               # linear model grid 4100-6100 A
    F = 1.0 + 0.3 * rng.standard_normal(q)
    ln0, dln = np.log(4300.0), 2.274544e-4           # LAMOST step, inside the model range
    n_out = int(np.log(5900.0 / 4300.0) / dln)
    out = O.resample(F, lam1, dlam, n_out, ln0, dln)
    e = _bins(n_out, ln0, dln)
    # integral over the covered range equals the model's integral there (telescoping)
    k0 = (e[0] - (lam1 - 0.5 * dlam)) / dlam
    k1 = (e[-1] - (lam1 - 0.5 * dlam)) / dlam
    cum = np.concatenate([[0.0], np.cumsum(F * dlam)])
    exact = np.interp(k1, np.arange(q + 1), cum) - np.interp(k0, np.arange(q + 1), cum)
    assert abs((out * np.diff(e)).sum() - exact) < 1e-9 * abs(exact)
    const = O.resample(np.full(q, 2.5), lam1, dlam, n_out, ln0, dln)
    np.testing.assert_allclose(const, 2.5, rtol=1e-12)


def test_resample_matches_brute_force_bin_averages():
    rng = np.random.default_rng(10)
    lam1, dlam, q = 5000.0, 0.7, 60
    F = rng.uniform(0.2, 1.5, q)
    ln0, dln = np.log(5003.0), 1.3e-4
    n_out = 40
    out = O.resample(F, lam1, dlam, n_out, ln0, dln)
    ref = _brute_resample(F, lam1, dlam, _bins(n_out, ln0, dln), sub=4000)
    np.testing.assert_allclose(out, ref, rtol=2e-3, atol=1e-3)


# ------------------------------------------------ Clean masking (stage 6, Eq. 8)

def _base_noise(p):
    # deterministic residual with mean 0 and population std 1: +-1 alternating
    return np.where(np.arange(p) % 2 == 0, 1.0, -1.0).astype(np.float32)


def test_clean_primary_adjacent_and_neighbourhood_masks():
    p = 200
    r = _base_noise(p)
    m = np.zeros(p, np.float32)                      # flat model: G = 0
    r[100] = 60.0                                    # B (primary outlier)
    r[101] = 8.0                                     # C: next to B, > 2 sigma
    r[102] = 6.0                                     # D: same sign, smaller, > sigma'
    r[103] = 5.0                                     # D (second pass)
    r[104] = -4.0                                    # opposite sign: kept
    r[99] = 1.5                                      # below 2 sigma, same sign, > sigma' -> D
    used = np.ones(p, np.uint8)
    keep, k = O.clean_mask(r, m, used, 0.5)
    # sigma of r over the used pixels, the B rule at k = 3
    sig = r.astype(np.float64).std()
    assert k == 3 and 60.0 > 3 * sig and 8.0 < 3 * sig
    flagged = set(np.where(keep == 0)[0])
    assert flagged == {99, 100, 101, 102, 103}, flagged


def test_clean_flux_gradient_protects_sharp_model_features():
    p = 200
    r = _base_noise(p)
    m = np.zeros(p, np.float32)
    r[50] = 12.0
    m[51] = 30.0                                     # steep model gradient at 50
    keep, _ = O.clean_mask(r, m, np.ones(p, np.uint8), 0.5)
    assert keep[50] == 1                             # |r| - 0.5 G = 12 - 15 < 3 sigma
    keep2, _ = O.clean_mask(r, np.zeros(p, np.float32), np.ones(p, np.uint8), 0.5)
    assert keep2[50] == 0


def test_clean_threshold_relaxes_when_many_outliers():
    p = 300
    r = _base_noise(p)
    idx = np.arange(5, 300, 25)                      # 12 outliers = 4% of the pixels
    r[idx] = np.where(np.arange(len(idx)) % 2 == 0, 5.5, -5.5).astype(np.float32)
    sig = r.astype(np.float64).std()
    assert 5.5 > 3 * sig and 5.5 < 4 * sig
    keep, k = O.clean_mask(r, np.zeros(p, np.float32), np.ones(p, np.uint8), 0.5)
    assert k == 4 and np.all(keep[idx] == 1)         # at k = 4 none of them is primary


def test_clean_ignores_unused_pixels_and_fit_with_outliers():
    p = 100
    r = _base_noise(p)
    r[10] = 90.0
    used = np.ones(p, np.uint8)
    used[10] = 0                                     # already masked: not in sigma, stays masked
    keep, _ = O.clean_mask(r, np.zeros(p, np.float32), used, 0.5)
    assert keep[10] == 0 and keep.sum() == p - 1
    # a fit with cosmic-ray spikes: Clean brings the parameters back near the clean-data fit
    M, d = observed(G, 4, 22, noise=True, snr=(60, 60), mask_frac=0.0)
    ref = O.fit(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_steps=400)
    spiky = d["flux"].copy()
    rng = np.random.default_rng(1)
    for i in range(4):
        js = rng.choice(G.n_pix, 12, replace=False)
        spiky[i, js] += 25.0 * np.median(d["flux"][i])
    bad = O.fit(M, spiky, d["ivar"], d["good"], d["theta0"], max_steps=400)
    cln = O.fit(M, spiky, d["ivar"], d["good"], d["theta0"], max_steps=400, clean=1)
    e_bad = np.abs(bad["theta"] - ref["theta"])[:, 0]
    e_cln = np.abs(cln["theta"] - ref["theta"])[:, 0]
    assert np.median(e_cln) < 0.5 * np.median(e_bad), (e_cln, e_bad)


# ------------------------------------------ curvature-aware step (sec. 4.5 outlook)

def test_lm_recovers_truth_and_reaches_a_stationary_point():
    M, d = observed(G, 6, 23, noise=False, mask_frac=0.0)
    res = O.fit_lm(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_iter=60, rtol=1e-12)
    err = np.abs(res["theta"] - d["truth"])[:, :4]
    assert np.all(err <= np.array([0.05, 5e-4, 5e-4, 5e-3])), err
    assert np.all(res["steps"] < 60)
    # noisy: the LM point is stationary (analytic gradient ~ 0) and no worse than Adam's
    M, d = observed(G, 4, 24, noise=True, snr=(30, 30), mask_frac=0.05)
    lm = O.fit_lm(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_iter=60, rtol=1e-12)
    ad = O.fit(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_steps=2000)
    for i in range(4):
        y, W, _, _ = O.prep(d["flux"][i], d["ivar"][i], d["good"][i])
        r = O.evaluate(M, y, W, O.x_from_phys(M, lm["theta"][i]))
        x = O.x_from_phys(M, lm["theta"][i])
        inner = np.abs(x) < 0.999                     # components not on the box edge
        assert np.all(np.abs(r["grad"][inner]) < 1e-5 * max(r["loss"], 1e-12) * 1e3)
        assert lm["loss"][i] <= ad["loss"][i] * (1 + 1e-9)


def test_lm_stops_at_a_kkt_point_of_the_box():
    """Low signal-to-noise fits that end on the box edge: interior components
    are stationary, edge components have a gradient pointing out of the box
    (the first-order conditions of a bound-constrained minimum)."""
    M, d = observed(G, 16, 25, noise=True, snr=(3, 6), mask_frac=0.05)
    lm = O.fit_lm(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_iter=200, rtol=1e-12)
    assert np.all(lm["status"] == 1)
    on_edge = 0
    for i in range(16):
        y, W, _, _ = O.prep(d["flux"][i], d["ivar"][i], d["good"][i])
        x = O.x_from_phys(M, lm["theta"][i])
        g = O.evaluate(M, y, W, x)["grad"]
        lo, hi = x <= -1 + 1e-12, x >= 1 - 1e-12
        on_edge += int(np.any(lo | hi))
        scale = 1e-2 * lm["loss"][i]
        assert np.all(np.abs(g[~(lo | hi)]) < scale), (i, g, x)
        assert np.all(g[lo] > -scale) and np.all(g[hi] < scale), (i, g, x)
    assert on_edge >= 1


# ---------------------------------------------------------------- joint loss (PAPER_JOINT)

def test_joint_gradient_is_the_derivative_of_the_group_rms():
    """The joint step direction (l_i / (N L)) dl_i/dx_i, written out, against
    central differences of L = sqrt(sum_i p l_i^2 / (N p)) itself."""
    M, d = observed(G, 3, 26, snr=(20, 40), mask_frac=0.05)
    ys = [O.prep(d["flux"][i], d["ivar"][i], d["good"][i])[:2] for i in range(3)]
    xs = [np.clip(O.x_from_phys(M, d["theta0"][i]), -1, 1) for i in range(3)]

    def L(xx):
        ls = [O.evaluate(M, ys[i][0], ys[i][1], xx[i])["loss"] for i in range(3)]
        return math.sqrt(sum(M.n_pix * l * l for l in ls) / (3 * M.n_pix)), ls

    L0, ls = L(xs)
    for i in range(3):
        gi = O.evaluate(M, ys[i][0], ys[i][1], xs[i])["grad"]
        joint = ls[i] / (3 * L0) * gi
        for k in range(5):
            h = 1e-6
            xp = [x.copy() for x in xs]
            xm = [x.copy() for x in xs]
            xp[i][k] += h
            xm[i][k] -= h
            fd = (L(xp)[0] - L(xm)[0]) / (2 * h)
            assert abs(fd - joint[k]) <= 1e-6 * max(1e-3, abs(joint[k])), (i, k, fd, joint[k])


def test_joint_fit_of_one_spectrum_is_the_separable_fit_and_groups_stop_together():
    M, d = observed(G, 5, 27, snr=(10, 60), mask_frac=0.05)
    sep = O.fit(M, d["flux"][:1], d["ivar"][:1], d["good"][:1], d["theta0"][:1], max_steps=300)
    one = O.fit_joint(M, d["flux"][:1], d["ivar"][:1], d["good"][:1], d["theta0"][:1], max_steps=300)
    assert one["steps"][0] == sep["steps"][0] and one["status"][0] == sep["status"][0]
    np.testing.assert_allclose(one["theta"], sep["theta"], rtol=0, atol=1e-9 * np.abs(sep["theta"]).max())
    # a group: one step count and status, L is the RMS of the members' losses
    d["good"][3] = 0                                   # no data: leaves the group at once
    grp = O.fit_joint(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_steps=300)
    assert grp["status"][3] == 64
    members = [0, 1, 2, 4]
    assert len(set(grp["steps"][members])) == 1 and len(set(grp["status"][members] & 7)) == 1
    L = math.sqrt(np.mean(grp["loss"][members] ** 2))
    assert abs(L - grp["loss_group"]) <= 1e-12 * L
