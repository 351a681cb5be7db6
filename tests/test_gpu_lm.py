"""Curvature-aware fit (Levenberg-Marquardt, the paper's outlook) on the GPU
against the FP64 oracle's LM: both converge to the same least-squares
minimum, so parity is checked at the converged point."""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import TOL, observed, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _gpu_lm(grid, d, **opts):
    from paper_2512_24840_gb300 import lasp
    lasp.load(build=True)
    ip = lasp.Interp.from_grid(grid, table(grid.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    T = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)
    out = ip.fit(T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(d["theta0"]),
                 optimizer="lm", **opts)
    torch.cuda.synchronize()
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def test_lm_noise_free_recovery():
    M, d = observed(S.SMALL, 16, S.SPECTRA_SEED, noise=False, mask_frac=0.0)
    d["theta0"] = np.asarray(d["theta0"], np.float32).astype(np.float64)
    out = _gpu_lm(S.SMALL, d, max_steps=100, tol=1e-10)
    err = np.abs(out["theta"] - d["truth"])[:, :4]
    assert np.all(err <= TOL), err.max(axis=0)
    assert np.all(out["steps"] < 100)


@pytest.mark.parametrize("grid,n", [(S.LAMOST, 96), (S.DESI, 24)], ids=["lamost", "desi"])
def test_lm_matches_oracle_lm(grid, n):
    M, d = observed(grid, n, 101, snr=(5, 100), mask_frac=0.05)
    d["theta0"] = np.asarray(d["theta0"], np.float32).astype(np.float64)
    ref = O.fit_lm(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_iter=100, rtol=1e-10)
    out = _gpu_lm(grid, d, max_steps=100, tol=1e-10)
    err = np.abs(out["theta"] - ref["theta"])[:, :4]
    ok = np.all(err <= TOL, axis=1)
    print(f"{grid.name} LM parity {ok.mean():.3f}; median iterations GPU {np.median(out['steps'])}, "
          f"oracle {np.median(ref['steps'])}")
    assert ok.mean() >= 0.95
    np.testing.assert_allclose(out["loss"], ref["loss"], rtol=1e-4)
    # the continuum coefficients returned are those of the result: the
    # oracle's weighted least squares (Eq. 6) at the GPU's own parameters
    for i in range(0, n, max(1, n // 8)):
        y, W, _, _ = O.prep(d["flux"][i], d["ivar"][i], d["good"][i])
        b = O.evaluate(M, y, W, O.x_from_phys(M, out["theta"][i]))["b"]
        np.testing.assert_allclose(out["cont"][i], b, rtol=2e-3, atol=2e-4)
