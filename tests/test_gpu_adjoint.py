"""The hand-written adjoint behind the autograd Function (adjoint check on
1024 LAMOST-like spectra x 3909 pixels, FP32): gradients w.r.t. theta (Teff,
log g, [Fe/H], RV, sigma) and the Legendre coefficients against the FP64
oracle's vector-Jacobian product and against central finite differences."""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import DEG, GRAD_RTOL_THETA, GRAD_TOL_LEG, oracle_model, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2512_24840_gb300 import lasp
    from paper_2512_24840_gb300.autograd import spectrum_model
    lasp.load(build=True)
    g = S.LAMOST
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    d = S.draw_batch(g, 1024, S.SPECTRA_SEED + 2, noise=False, mask_frac=0.0)
    th = np.asarray(d["truth"] + np.array([30.0, 0.05, 0.03, 2.0, 4.0]), np.float32).astype(np.float64)
    b = np.asarray(d["b_true"] / d["b_true"][:, :1], np.float32).astype(np.float64)
    rng = np.random.default_rng(7)
    gm = rng.normal(0, 1, (1024, g.n_pix)).astype(np.float32).astype(np.float64)
    return lasp, spectrum_model, ip, g, th, b, gm


def test_autograd_matches_oracle_vjp_full_size(setup):
    lasp, spectrum_model, ip, g, th, b, gm = setup
    dev = "cuda:0"
    theta = torch.tensor(th, dtype=torch.float32, device=dev, requires_grad=True)
    bb = torch.tensor(b, dtype=torch.float32, device=dev, requires_grad=True)
    model = spectrum_model(ip, theta, bb)
    (model * torch.tensor(gm, dtype=torch.float32, device=dev)).sum().backward()
    gth, gb = theta.grad.double().cpu().numpy(), bb.grad.double().cpu().numpy()
    M = oracle_model(g)
    worst_th = worst_b = 0.0
    for i in np.random.default_rng(8).choice(1024, 24, replace=False):
        rth, rb = O.model_vjp(M, th[i], b[i], gm[i])
        scale = np.abs(rth) + 1e-3 * np.abs(rth).max()
        worst_th = max(worst_th, float(np.max(np.abs(gth[i] - rth) / scale)))
        worst_b = max(worst_b, float(np.max(np.abs(gb[i] - rb)) / np.abs(rb).max()))
        assert np.all(np.abs(gth[i] - rth) <= GRAD_RTOL_THETA * scale), (i, gth[i], rth)
        np.testing.assert_allclose(gb[i], rb, rtol=GRAD_TOL_LEG, atol=GRAD_TOL_LEG * np.abs(rb).max())
    print(f"adjoint vs oracle VJP (24 of 1024): theta {worst_th:.2e} (bound {GRAD_RTOL_THETA:g}), "
          f"Legendre {worst_b:.2e} of max (bound {GRAD_TOL_LEG:g})")


def test_autograd_matches_central_differences(setup):
    """Central differences with h = 1e-4 relative, taken in FP64 on the
    oracle's forward model, against the GPU adjoint (GRAD_RTOL_THETA, GRAD_TOL_LEG;
    the differences' own truncation and rounding errors are below 1e-7); and central
    differences of the GPU's own FP32 forward with a step large enough for
    FP32 (3e-3 relative; median agreement 5e-2), so forward and adjoint of
    the CUDA path are consistent with each other."""
    lasp, spectrum_model, ip, g, th, b, gm = setup
    dev = "cuda:0"
    M = oracle_model(g)
    idx = np.arange(0, 1024, 128)
    theta = torch.tensor(th[idx], dtype=torch.float32, device=dev)
    bb = torch.tensor(b[idx], dtype=torch.float32, device=dev)
    gmt = torch.tensor(gm[idx], dtype=torch.float32, device=dev)
    gth, gb = ip.backward(theta, bb, gmt)
    gth, gb = gth.double().cpu().numpy(), gb.double().cpu().numpy()
    worst_th = worst_b = 0.0
    for n, i in enumerate(idx):
        f = lambda t, c: float(gm[i] @ O.model_flux(M, t, c)["model"])
        for k in range(5):
            h = 1e-4 * max(abs(th[i, k]), 1.0)
            tp, tm = th[i].copy(), th[i].copy()
            tp[k] += h
            tm[k] -= h
            fd = (f(tp, b[i]) - f(tm, b[i])) / (2 * h)
            worst_th = max(worst_th, abs(fd - gth[n, k]) / (abs(fd) + 1e-3 * np.abs(gth[n]).max()))
            assert abs(fd - gth[n, k]) <= GRAD_RTOL_THETA * (abs(fd) + 1e-3 * np.abs(gth[n]).max()), (i, k, fd, gth[n, k])
        for k in range(DEG + 1):
            bp, bm = b[i].copy(), b[i].copy()
            bp[k] += 1e-4
            bm[k] -= 1e-4
            fd = (f(th[i], bp) - f(th[i], bm)) / 2e-4
            worst_b = max(worst_b, abs(fd - gb[n, k]) / np.abs(gb[n]).max())
            assert abs(fd - gb[n, k]) <= GRAD_TOL_LEG * np.abs(gb[n]).max()
    print(f"adjoint vs FP64 central differences: theta {worst_th:.2e} (bound {GRAD_RTOL_THETA:g}), "
          f"Legendre {worst_b:.2e} of max (bound {GRAD_TOL_LEG:g})")
    # FD of the FP32 forward itself
    fg = lambda t, c: (ip.forward(t, c).double() * gmt.double()).sum(dim=1)
    for k in range(5):
        h = 3e-3 * torch.clamp(theta[:, k].abs(), min=1.0)
        tp, tm = theta.clone(), theta.clone()
        tp[:, k] += h
        tm[:, k] -= h
        fd = ((fg(tp, bb) - fg(tm, bb)) / (tp[:, k] - tm[:, k]).double()).cpu().numpy()
        rel = np.abs(fd - gth[:, k]) / (np.abs(gth[:, k]) + 1e-30)
        print(f"FP32 forward differences, parameter {k}: median rel {np.median(rel):.2e} (bound 5e-2)")
        assert np.median(rel) < 5e-2, (k, rel)
