"""Piecewise Teff-regime emulator (Eq. 1 with the ranges f1..f5; cold, warm
and hot models of section 3.1) on the GPU, through the C-ABI, against the FP64
oracle.  Parameters span all five Teff ranges and sit exactly on the blend
bounds (4000, 4550, 7000, 9000 K are exact in float32, and both sides treat
the intervals as closed above)."""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import DEG, GRAD_RTOL_THETA, GRAD_TOL_LEG, TOL, observed, piecewise_model, pw_tables, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PW_DRAW = dict(teff=(3300.0, 11500.0), box=(S.PW_BOX_LO, S.PW_BOX_HI))


@pytest.fixture(scope="module")
def lasp():
    from paper_2512_24840_gb300 import lasp as L
    L.load(build=True)
    return L


_ips = {}


def pw_interp(lasp, grid):
    if grid.name not in _ips:
        _ips[grid.name] = lasp.Interp.piecewise(pw_tables(grid.name), S.PW_EXPS, grid.n_pix, grid.pad,
                                                grid.dln, S.PW_BASIS_LO, S.PW_BASIS_HI, S.TEFF_BLEND,
                                                S.PW_BOX_LO, S.PW_BOX_HI)
    return _ips[grid.name]


def q32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def T(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)


def H(t):
    return t.detach().double().cpu().numpy()


def rel_err(got, ref):
    return (np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)).max()


def spread_thetas(n, seed):
    """Teff over the whole box, on every bound and just either side of it."""
    rng = np.random.default_rng(seed)
    teff = np.concatenate([rng.uniform(3200.0, 12000.0, n), np.array(S.TEFF_BLEND),
                           np.array(S.TEFF_BLEND) - 0.5, np.array(S.TEFF_BLEND) + 0.5, [3200.0, 12000.0]])
    m = len(teff)
    th = np.stack([teff, rng.uniform(0.5, 5.5, m), rng.uniform(-2.5, 1.0, m), rng.uniform(-300, 300, m),
                   rng.uniform(30, 200, m)], axis=1)
    return q32(th)


@pytest.mark.parametrize("grid", [S.SMALL, S.LAMOST], ids=lambda g: g.name)
def test_interp_all_ranges(lasp, grid):
    M = piecewise_model(grid)
    th = spread_thetas(20, 61)
    Fp = H(pw_interp(lasp, grid).interp_eval(T(th), "fp32"))
    b = np.tile(np.r_[1.0, np.zeros(DEG)], (len(th), 1))
    ref = np.stack([O.model_flux(M, th[i], b[i])["Fp"] for i in range(len(th))])
    assert rel_err(Fp, ref) < 2e-6


def test_forward_and_backward_all_ranges(lasp):
    grid = S.LAMOST
    M = piecewise_model(grid)
    th = spread_thetas(12, 62)
    n = len(th)
    rng = np.random.default_rng(7)
    b = q32(np.c_[np.ones(n), rng.normal(0, 0.05, (n, DEG))])
    ip = pw_interp(lasp, grid)
    got = H(ip.forward(T(th), T(b)))
    ref = O.model_batch(M, th, b)
    assert rel_err(got, ref) < 1e-5
    gm = q32(rng.normal(0, 1, (n, grid.n_pix)))
    gth, gb = ip.backward(T(th), T(b), T(gm))
    gth, gb = H(gth), H(gb)
    worst = 0.0
    for i in range(n):
        rth, rb = O.model_vjp(M, th[i], b[i], gm[i])
        scale = np.abs(rth) + 1e-3 * np.abs(rth).max()
        worst = max(worst, float(np.max(np.abs(gth[i] - rth) / scale)))
        assert np.all(np.abs(gth[i] - rth) <= GRAD_RTOL_THETA * scale), (i, th[i, 0], gth[i], rth)
        np.testing.assert_allclose(gb[i], rb, rtol=GRAD_TOL_LEG, atol=GRAD_TOL_LEG * np.abs(rb).max())
    print(f"piecewise adjoint vs oracle VJP, all Teff ranges: theta {worst:.2e} (bound {GRAD_RTOL_THETA:g})")


def _inputs(grid, n, seed, **kw):
    M = piecewise_model(grid)
    _, d = observed(grid, n, seed, M=M, **PW_DRAW, **kw)
    d["theta0"] = q32(d["theta0"])
    return M, d


def _gpu(lasp, grid, d, what="fit", **opts):
    ip = pw_interp(lasp, grid)
    args = [T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(d["theta0"])]
    out = getattr(ip, what)(*args, **opts)
    torch.cuda.synchronize()
    return {k: H(v) for k, v in out.items()}


def test_adam_fit_parity(lasp):
    M, d = _inputs(S.LAMOST, 96, 63, snr=(5, 100), mask_frac=0.05)
    out = _gpu(lasp, S.LAMOST, d, max_steps=500)
    ref = O.fit(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_steps=500)
    err = np.abs(out["theta"] - ref["theta"])[:, :4]
    ok = np.all(err <= TOL, axis=1)
    print(f"piecewise Adam parity {ok.mean():.3f}, same steps {(out['steps'] == ref['steps']).mean():.3f}")
    assert ok.mean() >= 0.9
    assert np.all((out["status"].astype(np.int64) & 7) != 0)


def test_noise_free_recovery_all_ranges(lasp):
    M, d = _inputs(S.SMALL, 10, 64, noise=False, mask_frac=0.0)
    out = _gpu(lasp, S.SMALL, d, max_steps=100, tol=1e-10, optimizer="lm")
    err = np.abs(out["theta"] - d["truth"])[:, :4]
    assert np.all(err <= TOL), err


def test_lm_parity(lasp):
    M, d = _inputs(S.LAMOST, 64, 65, snr=(5, 100), mask_frac=0.05)
    out = _gpu(lasp, S.LAMOST, d, max_steps=100, tol=1e-10, optimizer="lm")
    ref = O.fit_lm(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_iter=100, rtol=1e-10)
    ok = np.all(np.abs(out["theta"] - ref["theta"])[:, :4] <= TOL, axis=1)
    print(f"piecewise LM parity {ok.mean():.3f}")
    assert ok.mean() >= 0.95


def test_errors_parity(lasp):
    M, d = _inputs(S.LAMOST, 12, 66, snr=(10, 100), mask_frac=0.05)
    e = _gpu(lasp, S.LAMOST, d, what="errors")
    ref = np.stack([O.errors(M, d["flux"][i], d["ivar"][i], d["good"][i], d["theta0"][i])["sigma"]
                    for i in range(12)])
    rel = np.abs(e["sigma"] - ref) / ref
    assert np.median(rel) < 1e-3 and np.mean(rel < 1e-2) >= 0.9, rel.max(axis=0)


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-5), ("tf32", 4e-3), ("bf16", 3e-2)])
def test_tensor_core_interp_all_ranges(lasp, prec, tol):
    """Eq. 1 with the Teff regimes on tcgen05: the stacked rows of the three
    regimes in three K blocks of 32 terms, the rows of inactive regimes
    weighted zero (a masked grouped contraction)."""
    grid = S.LAMOST
    M = piecewise_model(grid)
    th = spread_thetas(150, 67)
    Fp = H(pw_interp(lasp, grid).interp_eval(T(th), prec))
    b = np.tile(np.r_[1.0, np.zeros(DEG)], (len(th), 1))
    ref = np.stack([O.model_flux(M, th[i], b[i])["Fp"] for i in range(len(th))])
    err = rel_err(Fp, ref)
    print(f"piecewise {prec} contraction: max rel err {err:.3e}")
    assert err < tol


def test_tensor_core_adam_fit_parity(lasp):
    """The grouped tensor-core fit (split TF32, float-float normal equations)
    on the piecewise emulator against the oracle, all five Teff ranges."""
    M, d = _inputs(S.LAMOST, 96, 63, snr=(5, 100), mask_frac=0.05)
    out = _gpu(lasp, S.LAMOST, d, max_steps=500, precision="tf32x3", fp64_normal_eq=1)
    ref = O.fit(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_steps=500)
    err = np.abs(out["theta"] - ref["theta"])[:, :4]
    ok = np.all(err <= TOL, axis=1)
    print(f"piecewise tf32x3 Adam parity {ok.mean():.3f}, same steps {(out['steps'] == ref['steps']).mean():.3f}")
    assert ok.mean() >= 0.9
    assert np.all((out["status"].astype(np.int64) & 7) != 0)
    # and against the FP32 fit of the same spectra
    fp = _gpu(lasp, S.LAMOST, d, max_steps=500)
    same = np.all(np.abs(out["theta"] - fp["theta"])[:, :4] <= TOL, axis=1)
    print(f"piecewise tf32x3 vs FP32 fit: {same.mean():.3f} within tolerance")
    assert same.mean() >= 0.9


def test_one_regime_piecewise_handle_equals_plain_handle(lasp):
    """The one-regime form of the piecewise entry point is the plain
    interpolator: bitwise-equal fits."""
    grid = S.LAMOST
    plain = lasp.Interp.from_grid(grid, table(grid.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO,
                                  S.BOX_HI)
    one = lasp.Interp.piecewise([table(grid.name)], [S.EXPS], grid.n_pix, grid.pad, grid.dln,
                                [S.BASIS_LO], [S.BASIS_HI], [], S.BOX_LO, S.BOX_HI)
    _, d = observed(grid, 32, 69, snr=(5, 100), mask_frac=0.05)
    args = [T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(q32(d["theta0"]))]
    a = plain.fit(*args, max_steps=300)
    b = one.fit(*args, max_steps=300)
    assert torch.equal(a["theta"], b["theta"]) and torch.equal(a["steps"], b["steps"])


def test_fit_results_do_not_depend_on_batch_order(lasp):
    """The batch fit takes a piecewise batch's spectra grouped by the Teff
    range of their starting parameters; each spectrum's result is bitwise the
    same whatever the order of the batch (here reversed and shuffled)."""
    M, d = _inputs(S.LAMOST, 200, 64, snr=(5, 100), mask_frac=0.05)
    base = _gpu(lasp, S.LAMOST, d, max_steps=300)
    for perm in (np.arange(200)[::-1], np.random.default_rng(5).permutation(200)):
        dp = {k: (v[perm] if isinstance(v, np.ndarray) and v.shape[:1] == (200,) else v) for k, v in d.items()}
        out = _gpu(lasp, S.LAMOST, dp, max_steps=300)
        for k in ("theta", "loss", "steps", "status", "cont"):
            assert np.array_equal(out[k], base[k][perm], equal_nan=True), k
    assert lasp.last_launches() == 5        # the regime order, the preprocessing and the fit
