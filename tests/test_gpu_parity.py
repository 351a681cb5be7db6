"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Inputs are seeded synthetic spectra whose observed flux the oracle makes;
every expected value comes from the oracle.  Tolerances: model flux 1e-5 of
the spectrum's maximum (FP32); fitted parameters Teff 1 K, log g 0.005 dex,
[Fe/H] 0.005 dex, RV 0.1 km/s; gradients and errors as stated per test.
"""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import DEG, GRAD_RTOL_THETA, GRAD_TOL_LEG, TOL, observed, oracle_model, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def lasp():
    from paper_2512_24840_gb300 import lasp as L
    L.load(build=True)
    return L


_interps = {}


def interp(lasp, grid):
    if grid.name not in _interps:
        _interps[grid.name] = lasp.Interp.from_grid(grid, table(grid.name), S.EXPS, S.BASIS_LO,
                                                    S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    return _interps[grid.name]


def q32(a):
    """Round to float32 and back: the oracle sees exactly what the GPU gets."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def T(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)


def H(t):
    return t.detach().double().cpu().numpy()


def _flux_rel_err(got, ref):
    return (np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)).max()


# ------------------------------------------------------------ Eq. 1 alone

@pytest.mark.parametrize("grid", [S.SMALL, S.LAMOST, S.DESI], ids=lambda g: g.name)
def test_interp_fp32_matches_oracle(lasp, grid):
    M, d = observed(grid, 5, 31, noise=False, mask_frac=0.0)
    d["truth"] = q32(d["truth"])
    ip = interp(lasp, grid)
    Fp = H(ip.interp_eval(T(d["truth"]), "fp32"))
    ref = np.stack([O.model_flux(M, d["truth"][i], d["b_true"][i])["Fp"] for i in range(5)])
    assert _flux_rel_err(Fp, ref) < 1e-6


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-5), ("tf32", 4e-3), ("bf16", 3e-2)])
@pytest.mark.parametrize("grid", [S.SMALL, S.LAMOST], ids=lambda g: g.name)
def test_interp_tensor_core_matches_oracle(lasp, grid, prec, tol):
    """tcgen05 contraction; N = 300 spectra spans three 128-spectrum blocks and
    a ragged tail, and the pixel tiles a ragged last tile."""
    M, d = observed(grid, 300, 34, noise=False, mask_frac=0.0)
    d["truth"] = q32(d["truth"])
    ip = interp(lasp, grid)
    Fp = H(ip.interp_eval(T(d["truth"]), prec))
    ref = np.stack([O.model_flux(M, d["truth"][i], d["b_true"][i])["Fp"] for i in range(300)])
    err = _flux_rel_err(Fp, ref)
    print(f"{grid.name} {prec}: max rel err {err:.3e}")
    assert err < tol


# ------------------------------------------------ forward model (Eqs. 1, 5, 6)

@pytest.mark.parametrize("grid", [S.SMALL, S.LAMOST, S.DESI], ids=lambda g: g.name)
def test_forward_matches_oracle(lasp, grid):
    M, d = observed(grid, 7, 32, noise=False, mask_frac=0.0)
    d["truth"] = q32(d["truth"])
    b = q32(d["b_true"] / d["b_true"][:, :1])
    ip = interp(lasp, grid)
    got = H(ip.forward(T(d["truth"]), T(b)))
    ref = O.model_batch(M, d["truth"], b)
    assert _flux_rel_err(got, ref) < 1e-5


def test_forward_kernel_edge_cases(lasp):
    grid = S.SMALL
    M = oracle_model(grid)
    ip = interp(lasp, grid)
    th = np.array([[3500.0, 0.5, -2.5, -300.0, 30.0],      # box corners: widest shift,
                   [7500.0, 5.5, 1.0, 300.0, 200.0],       # widest kernel (h = H)
                   [5000.0, 3.0, -0.5, 0.0, 30.0]])
    b = np.tile(np.r_[1.0, np.zeros(DEG)], (3, 1))
    got = H(ip.forward(T(th), T(b)))
    ref = O.model_batch(M, th, b)
    assert _flux_rel_err(got, ref) < 1e-5
    assert ip.forward(T(np.zeros((0, 5))), T(np.zeros((0, DEG + 1)))).shape == (0, grid.n_pix)


# ------------------------------------------------ hand-written adjoint

@pytest.mark.parametrize("grid", [S.SMALL, S.LAMOST], ids=lambda g: g.name)
def test_backward_matches_oracle_vjp(lasp, grid):
    M, d = observed(grid, 6, 33, noise=False, mask_frac=0.0)
    rng = np.random.default_rng(5)
    b = q32(d["b_true"] / d["b_true"][:, :1])
    d["theta0"] = q32(d["theta0"])
    gm = q32(rng.normal(0, 1, (6, grid.n_pix)))
    ip = interp(lasp, grid)
    gth, gb = ip.backward(T(d["theta0"]), T(b), T(gm))
    gth, gb = H(gth), H(gb)
    worst = 0.0
    for i in range(6):
        rth, rb = O.model_vjp(M, d["theta0"][i], b[i], gm[i])
        scale_th = np.abs(rth) + 1e-3 * np.abs(rth).max()
        worst = max(worst, float(np.max(np.abs(gth[i] - rth) / scale_th)))
        assert np.all(np.abs(gth[i] - rth) <= GRAD_RTOL_THETA * scale_th), (gth[i], rth)
        np.testing.assert_allclose(gb[i], rb, rtol=GRAD_TOL_LEG, atol=GRAD_TOL_LEG * np.abs(rb).max())
    print(f"{grid.name} adjoint vs oracle VJP: theta {worst:.2e} (bound {GRAD_RTOL_THETA:g})")


# ------------------------------------------------ fits (stage 8)

def _fit_both(lasp, grid, M, d, n=None, **opts):
    d["theta0"] = q32(d["theta0"])
    ip = interp(lasp, grid)
    out = ip.fit(T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(d["theta0"]), **opts)
    torch.cuda.synchronize()
    ref = O.fit(M, d["flux"], d["ivar"], d["good"], d["theta0"], **opts)
    return out, ref


@pytest.mark.parametrize("lr,nsteps", [(0.1, 12), (0.01, 30)])
def test_fixed_step_trajectory_parity_small(lasp, lr, nsteps):
    """16 x 1024 noise-free, stop rules off, a fixed number of Adam steps.

    Noise-free fits end in an oscillation about the optimum where the path is
    chaotic.  Calibrated on the oracle itself with the flux perturbed by
    1e-5 relative (about the FP32 rounding of the GPU path, whose continuum
    solve is good to ~1e-5): at lr 0.1 the path leaves the tolerance after
    step 21 (within 0.31 of it at step 10); at lr 0.01 after step 42 (within
    0.45 of it at step 40).  Fixed-step parity is checked inside those
    well-conditioned stretches."""
    M, d = observed(S.SMALL, 16, S.SPECTRA_SEED, noise=False, mask_frac=0.0)
    out, ref = _fit_both(lasp, S.SMALL, M, d, max_steps=nsteps, tol=0.0, lr=lr)
    assert np.all(H(out["steps"]) == ref["steps"])
    err = np.abs(H(out["theta"]) - ref["theta"])[:, :4]
    assert np.all(err <= TOL), err.max(axis=0)


@pytest.mark.parametrize("deg", [2, 4, 8])
def test_fit_other_continuum_degrees(lasp, deg):
    """Legendre continua of degree 2, 4 and 8 (the FP32 path's other degrees):
    fixed-step parity with the oracle's fit of the same degree on a batch of
    seven (fewer spectra than two CTAs of the batch fit carry), and the served
    form (one spectrum per CTA, resumed every 7 steps) bitwise equal to it."""
    M, d = observed(S.SMALL, 7, 46, noise=False, mask_frac=0.0)
    d["theta0"] = q32(d["theta0"])
    ip = interp(lasp, S.SMALL)
    args = (T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(d["theta0"]))
    out = ip.fit(*args, max_steps=12, tol=0.0, legendre_deg=deg)
    torch.cuda.synchronize()
    ref = O.fit(oracle_model(S.SMALL, deg=deg), d["flux"], d["ivar"], d["good"], d["theta0"],
                max_steps=12, tol=0.0)
    assert np.all(H(out["steps"]) == ref["steps"])
    err = np.abs(H(out["theta"]) - ref["theta"])[:, :4]
    assert np.all(err <= TOL), err.max(axis=0)
    from paper_2512_24840_gb300.server import DevicePool, Server
    one = ip.fit(*args, max_steps=60, legendre_deg=deg)
    srv = Server({"s": DevicePool(ip, 3, max_steps=60, legendre_deg=deg)}, chunk=7)
    ids = [srv.submit("s", d["flux"][i], d["ivar"][i], d["good"][i], d["theta0"][i]) for i in range(7)]
    res = {r.rid: r for r in srv.run_until_idle()}
    srv.close()
    for k, rid in enumerate(ids):
        assert np.array_equal(res[rid].theta, H(one["theta"])[k]), k
        assert res[rid].steps == int(H(one["steps"])[k])


def test_noise_free_recovery_small(lasp):
    """Small steps to convergence: the GPU fit recovers the truth (config-1
    data).  lr 3e-4 keeps Adam's end-of-fit jitter (about lr x half box
    width = 0.6 K in Teff) inside the tolerance."""
    M, d = observed(S.SMALL, 16, S.SPECTRA_SEED, noise=False, mask_frac=0.0)
    ip = interp(lasp, S.SMALL)
    out = ip.fit(T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(q32(d["theta0"])),
                 lr=3e-4, tol=1e-11, max_steps=40000)
    err = np.abs(H(out["theta"]) - d["truth"])[:, :4]
    assert np.all(err <= TOL), err.max(axis=0)


def test_fit_early_stop_parity_lamost(lasp):
    """Paper defaults (lr 0.1, tol 1e-5, window 50) on noisy LAMOST-like spectra."""
    M, d = observed(S.LAMOST, 96, 41, snr=(5, 100), mask_frac=0.05)
    out, ref = _fit_both(lasp, S.LAMOST, M, d, max_steps=500)
    err = np.abs(H(out["theta"]) - ref["theta"])[:, :4]
    ok = np.all(err <= TOL, axis=1)
    same_steps = H(out["steps"]) == ref["steps"]
    print(f"LAMOST early-stop parity {ok.mean():.3f}, same steps {same_steps.mean():.3f}")
    assert ok.mean() >= 0.95, (ok.mean(), err.max(axis=0))
    assert same_steps.mean() >= 0.9
    assert np.all((H(out["status"]).astype(np.int64) & 7) != 0)


def test_fit_mixed_grid_desi_parity(lasp):
    M, d = observed(S.DESI, 24, 42, snr=(10, 100), mask_frac=0.0, mask_frac_max=0.2)
    out, ref = _fit_both(lasp, S.DESI, M, d, max_steps=300)
    err = np.abs(H(out["theta"]) - ref["theta"])[:, :4]
    ok = np.all(err <= TOL, axis=1)
    print(f"DESI mixed-grid parity {ok.mean():.3f}")
    assert ok.mean() >= 0.9, err.max(axis=0)


def test_fit_edge_cases(lasp):
    grid = S.SMALL
    M, d = observed(grid, 6, 43, snr=(20, 50), mask_frac=0.05)
    d["good"][1] = 0                                 # all masked -> NODATA
    d["flux"][2, 100:110] = np.nan                   # non-finite pixels are not used
    d["good"][3, :1020] = 0                          # too few pixels -> NODATA
    out, ref = _fit_both(lasp, grid, M, d, max_steps=60, tol=0.0)
    st = H(out["status"]).astype(np.int64)
    assert st[1] == lasp.ST_NODATA and st[3] == lasp.ST_NODATA
    assert np.all(st == ref["status"])
    use = [0, 2, 4, 5]
    err = np.abs(H(out["theta"]) - ref["theta"])[use, :4]
    assert np.all(err <= TOL)
    # max_steps = 0: one evaluation, no update
    out0, ref0 = _fit_both(lasp, grid, M, d, max_steps=0)
    assert np.all(H(out0["steps"]) == 0)
    np.testing.assert_allclose(H(out0["loss"])[use], ref0["loss"][use], rtol=1e-5)
    # empty batch
    ip = interp(lasp, grid)
    e = ip.fit(T(np.zeros((0, grid.n_pix))), T(np.zeros((0, grid.n_pix))),
               T(np.zeros((0, grid.n_pix)), torch.uint8), T(np.zeros((0, 5))))
    assert e["theta"].shape == (0, 5)


def test_fit_loss_and_weight_outputs(lasp):
    grid = S.SMALL
    M, d = observed(grid, 8, 44, snr=(20, 50), mask_frac=0.05)
    out, ref = _fit_both(lasp, grid, M, d, max_steps=40, tol=0.0)
    np.testing.assert_allclose(H(out["loss"]), ref["loss"], rtol=1e-4)
    for i in range(8):
        _, _, w, _ = O.prep(d["flux"][i], d["ivar"][i], d["good"][i])
        assert abs(H(out["weight"])[i] - w) <= 1e-6 * abs(w)
    np.testing.assert_allclose(H(out["cont"]), ref["b"], rtol=1e-3, atol=1e-4)


@pytest.mark.parametrize("q", [0.0, 0.25, 0.5, 0.9, 1.0])
def test_weight_quantile_exact(lasp, q):
    """w, the flux quantile that scales Eq. 9's data, interpolates between two
    order statistics of the used pixels.  The kernels select those two values
    (radix select) where the oracle sorts, so w is float32 of the oracle's w
    exactly, including ties, negative values, zeros of both signs, spectra of
    one repeated value and masked or zero-ivar pixels.  Spectra whose w is not
    positive stop with LASP_ST_NODATA and still report w."""
    grid = S.SMALL
    n, p = 7, grid.n_pix
    rng = np.random.default_rng(77)
    flux = rng.normal(1.0, 0.3, (n, p)).astype(np.float32)
    flux[1] = np.round(flux[1] * 4.0) / 4.0          # heavy ties
    flux[2] -= 1.0                                   # about half negative
    flux[3, 0::3] = 0.0
    flux[3, 1::3] = -0.0                             # zeros of both signs
    flux[4] = 2.5                                    # one repeated value
    flux[5] = rng.lognormal(0.0, 2.0, p)             # a wide range of exponents
    ivar = np.ones((n, p), np.float32)
    good = np.ones((n, p), np.uint8)
    good[6, : p // 2] = 0
    ivar[6, p // 2: p // 2 + 17] = 0.0               # masked and zero-ivar pixels
    theta0 = np.asarray(S.draw_batch(grid, n, 78)["theta0"], np.float32)
    ip = interp(lasp, grid)
    out = ip.fit(T(flux), T(ivar), T(good, torch.uint8), T(theta0), max_steps=0, quantile=q)
    got = H(out["weight"])
    for i in range(n):
        # the options carry the quantile as float32: the oracle gets that value
        _, _, w, _ = O.prep(flux[i], ivar[i], good[i], quantile=float(np.float32(q)))
        assert got[i] == np.float32(w), (i, got[i], w)


def test_batch_invariance_bitwise(lasp):
    """A spectrum's result does not depend on the batch it is fitted in."""
    grid = S.LAMOST
    M, d = observed(grid, 64, 45, snr=(5, 100), mask_frac=0.05)
    ip = interp(lasp, grid)
    args = [T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(d["theta0"])]
    full = ip.fit(*args, max_steps=300)
    for i in (0, 17, 63):
        one = ip.fit(*[a[i:i + 1].contiguous() for a in args], max_steps=300)
        assert torch.equal(one["theta"][0], full["theta"][i])
        assert int(one["steps"][0]) == int(full["steps"][i])


# ------------------------------------------------ errors (stage 9)

@pytest.mark.parametrize("grid", [S.SMALL, S.LAMOST], ids=lambda g: g.name)
@pytest.mark.parametrize("ne", [1, 2], ids=["float-float", "fp64"])
def test_errors_match_oracle(lasp, grid, ne):
    M, d = observed(grid, 12, 46, snr=(10, 100), mask_frac=0.05)
    d["theta0"] = q32(d["theta0"])
    ip = interp(lasp, grid)
    e = ip.errors(T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(d["theta0"]), fp64_normal_eq=ne)
    sig = H(e["sigma"])
    ref = np.stack([O.errors(M, d["flux"][i], d["ivar"][i], d["good"][i], d["theta0"][i])["sigma"]
                    for i in range(12)])
    rel = np.abs(sig - ref) / ref
    print(f"stage-9 sigma ({'FP64' if ne == 2 else 'float-float'} sums): median rel. error "
          f"{np.median(rel):.2e} vs the oracle's central differences")
    assert np.median(rel) < 1e-3 and np.mean(rel < 1e-2) >= 0.95, rel.max(axis=0)
    assert np.all(H(e["status"]) == 0)
    # the covariance is symmetric positive definite and its diagonal gives sigma
    cov = e["cov"].cpu().numpy()
    assert np.allclose(cov, np.transpose(cov, (0, 2, 1)), rtol=1e-12, atol=0)
    assert np.all(np.linalg.eigvalsh(cov) > 0)
    np.testing.assert_allclose(np.sqrt(np.diagonal(cov, axis1=1, axis2=2)), sig, rtol=1e-6)


def test_empty_batches_on_every_entry_point(lasp):
    """N = 0 is a valid call everywhere: every compute entry point returns
    LASP_OK with empty outputs and enqueues nothing."""
    grid = S.SMALL
    ip = interp(lasp, grid)
    z = lambda *shape, dt=torch.float32: torch.zeros(shape, dtype=dt, device=DEV)
    args = [z(0, grid.n_pix), z(0, grid.n_pix), z(0, grid.n_pix, dt=torch.uint8), z(0, 5)]
    for opts in (dict(precision="tf32x3", fp64_normal_eq=1), dict(optimizer="lm"), dict(clean=1)):
        out = ip.fit(*args, **opts)
        assert out["theta"].shape == (0, 5) and lasp.load().lasp_last_launches() == 0, opts
    e = ip.errors(*args[:3], z(0, 5))
    assert e["sigma"].shape == (0, 5) and e["cov"].shape == (0, 5, 5)
    assert ip.forward(z(0, 5), z(0, 7)).shape == (0, grid.n_pix)
    gt, gb = ip.backward(z(0, 5), z(0, 7), z(0, grid.n_pix))
    assert gt.shape == (0, 5) and gb.shape == (0, 7)
    for prec in ("fp32", "tf32", "bf16", "tf32x3"):
        assert ip.interp_eval(z(0, 5), prec).shape == (0, grid.n_model)
        assert lasp.load().lasp_last_launches() == 0


def test_launch_counts(lasp):
    """lasp_last_launches counts the kernels a call enqueued: the FP32 batch
    fit is its preprocessing kernel and the fused fit, the errors one kernel."""
    grid = S.SMALL
    ip = interp(lasp, grid)
    M, d = observed(grid, 8, 45, snr=(20, 50), mask_frac=0.05)
    args = [T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(np.asarray(d["theta0"], np.float32))]
    out = ip.fit(*args, max_steps=50)
    assert lasp.last_launches() == 2
    ip.errors(*args[:3], out["theta"], with_cov=False)
    assert lasp.last_launches() == 1
