"""Flux-conserving resampling (stage 3, Eqs. 2-4) on the GPU against the FP64
oracle: table rows on a linear grid resampled onto the LAMOST-like ln grid,
and a forward model built from the resampled table."""
import math

import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import DEG, oracle_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _linear_table(lam1, dlam, q, K, seed=5):
    rng = np.random.default_rng(seed)
    lam = lam1 + dlam * np.arange(q)
    t = (lam - lam.mean()) / (lam.max() - lam.min())
    C = np.zeros((K, q))
    C[0] = 1.0 + 0.1 * t
    for k in range(1, K):
        C[k] = 0.02 / k * np.cos(3.0 * k * t)
    for c, d, s in zip(rng.uniform(lam[0], lam[-1], 400), rng.uniform(0.05, 0.5, 400),
                       rng.uniform(0.3, 0.8, 400)):
        C[0] -= d * np.exp(-0.5 * ((lam - c) / s) ** 2)
        C[1:] -= 0.1 * d * np.exp(-0.5 * ((lam - c) / s) ** 2)[None, :] * rng.normal(0, 1, (K - 1, 1))
    return C.astype(np.float32)


def test_resample_matches_oracle_and_forward():
    from paper_2512_24840_gb300 import lasp
    lasp.load(build=True)
    g = S.LAMOST
    lam1, dlam = 3600.0, 0.25
    q = int((9200.0 - lam1) / dlam)                 # covers the padded LAMOST-like grid
    K = S.K_TERMS
    Cl = _linear_table(lam1, dlam, q, K)
    ln0 = math.log(g.lam0) - g.pad * g.dln
    got = lasp.resample_linear(torch.tensor(Cl, device="cuda:0"), lam1, dlam, g.n_model, ln0, g.dln)
    got = got.double().cpu().numpy()
    ref = np.stack([O.resample(Cl[k].astype(np.float64), lam1, dlam, g.n_model, ln0, g.dln)
                    for k in range(K)])
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert (np.abs(got - ref) / scale).max() < 2e-6
    # an interpolator built from the linear table through the GPU resampling
    ip = lasp.Interp.from_linear(g.n_pix, g.pad, g.lam0, g.dln, Cl, lam1, dlam, S.EXPS,
                                 S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    M = oracle_model(g, C=ref.astype(np.float32))
    d = S.draw_batch(g, 6, 81, noise=False, mask_frac=0.0)
    th = np.asarray(d["truth"], np.float32).astype(np.float64)
    b = np.tile(np.r_[1.0, np.zeros(DEG)], (6, 1))
    model = ip.forward(torch.tensor(th, dtype=torch.float32, device="cuda:0"),
                       torch.tensor(b, dtype=torch.float32, device="cuda:0")).double().cpu().numpy()
    refm = O.model_batch(M, th, b)
    assert (np.abs(model - refm).max(axis=1) / np.abs(refm).max(axis=1)).max() < 1e-5
