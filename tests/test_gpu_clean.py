"""Clean outlier masking (stage 6, Eq. 8) on the GPU against the FP64
oracle: the mask itself on identical float32 inputs (the kernel decides in
float32, the oracle in double precision; differences only at borderline
comparisons), and Clean fits of spectra with cosmic-ray spikes and sky-like
residual runs."""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests import clean_check as CC
from tests.helpers import TOL, observed, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _residuals(N, p, seed):
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((N, p)).astype(np.float32)
    m = np.cumsum(rng.standard_normal((N, p)) * 0.3, axis=1).astype(np.float32)
    used = (rng.random((N, p)) > 0.03).astype(np.uint8)
    for i in range(N):
        n_spk = 0 if i % 3 == 0 else 6 + i % 10
        for c in rng.choice(p - 10, n_spk, replace=False):          # spikes with decaying tails
            sgn = 1.0 if rng.random() < 0.5 else -1.0
            amp = rng.uniform(4.0, 40.0)
            for d in range(int(rng.integers(1, 6))):
                r[i, c + d] = sgn * amp * 0.6 ** d
        if i % 3 == 0:                                                # many outliers: k relaxes
            idx = rng.choice(p, p // 20, replace=False)
            r[i, idx] = np.where(rng.random(len(idx)) < 0.5, 6.0, -6.0)
        m[i, rng.choice(p, 10)] += 50.0                              # sharp model features
    return r, m, used


@pytest.mark.parametrize("p", [1024, 3909, 7781])
@pytest.mark.parametrize("fshift", [0.5, 0.2])
def test_clean_mask_matches_oracle(p, fshift):
    """The kernel takes every Clean decision in float32, the oracle in double
    precision.  Where the masks differ, every differing pixel must be
    explained by a comparison within float32 rounding of its threshold (and
    the spread of such a flip along a flagged run); any other difference
    fails.  The borderline count is printed."""
    from paper_2512_24840_gb300 import lasp
    lasp.load(build=True)
    N = 24
    r, m, used = _residuals(N, p, 90 + p)
    keep, k = lasp.clean_mask(torch.tensor(r, device=DEV), torch.tensor(m, device=DEV),
                              torch.tensor(used, device=DEV), fshift)
    keep, k = keep.cpu().numpy(), k.cpu().numpy()
    n_diff = n_border = 0
    for i in range(N):
        ref, kr = O.clean_mask(r[i], m[i], used[i], fshift)
        ok, nb, why = CC.check(r[i], m[i], used[i], fshift, keep[i], int(k[i]), ref, kr)
        assert ok, (i, why)
        if k[i] != kr or not np.array_equal(keep[i], ref):
            n_diff += 1
            n_border += nb
    print(f"clean mask p={p} f_shift={fshift}: {n_diff} of {N} spectra differ from the FP64 "
          f"oracle, {n_border} borderline pixels")
    assert np.any(k == 4) or np.any(k == 5) or np.any(k == 7)


def test_clean_fit_parity_with_spikes():
    from paper_2512_24840_gb300 import lasp
    lasp.load(build=True)
    g = S.SMALL
    M, d = observed(g, 48, 91, snr=(30, 100), mask_frac=0.0)
    rng = np.random.default_rng(2)
    flux = d["flux"].copy()
    for i in range(48):
        med = np.median(flux[i])
        for c in rng.choice(g.n_pix - 8, 8, replace=False):
            flux[i, c:c + 3] += med * rng.uniform(0.5, 3.0) * np.array([1.0, 0.5, 0.2], np.float32)
    th0 = np.asarray(d["theta0"], np.float32).astype(np.float64)
    ref = O.fit(M, flux, d["ivar"], d["good"], th0, max_steps=400, clean=1)
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    T = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)
    out = ip.fit(T(flux), T(d["ivar"]), T(d["good"], torch.uint8), T(th0), max_steps=400, clean=1)
    th = out["theta"].double().cpu().numpy()
    ok = np.all(np.abs(th - ref["theta"])[:, :4] <= TOL, axis=1)
    print(f"clean fit parity: {ok.mean():.3f} within tolerance")
    assert ok.mean() >= 0.9
    # Clean helps: compared with No Clean on the same spiky data
    noc = ip.fit(T(flux), T(d["ivar"]), T(d["good"], torch.uint8), T(th0), max_steps=400)
    clean_ref = O.fit(M, d["flux"], d["ivar"], d["good"], th0, max_steps=400)
    e_c = np.abs(th - clean_ref["theta"])[:, 0]
    e_n = np.abs(noc["theta"].double().cpu().numpy() - clean_ref["theta"])[:, 0]
    assert np.median(e_c) < np.median(e_n)


def test_clean_rejected_where_unsupported():
    """Clean runs in Adam fits with the separable loss; the curvature-aware
    fit and the joint loss reject it."""
    from paper_2512_24840_gb300 import lasp
    lasp.load(build=True)
    g = S.SMALL
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    z = torch.zeros((2, g.n_pix), device=DEV)
    one = torch.ones((2, g.n_pix), dtype=torch.uint8, device=DEV)
    for extra in (dict(optimizer="lm"), dict(precision="tf32x3", loss_mode="joint")):
        with pytest.raises(lasp.LaspError):
            ip.fit(z, z, one, torch.zeros((2, 5), device=DEV), clean=1, **extra)


def _spiky(g, n, seed):
    M, d = observed(g, n, seed, snr=(30, 100), mask_frac=0.0)
    rng = np.random.default_rng(seed + 1)
    flux = d["flux"].copy()
    for i in range(n):
        med = np.median(flux[i])
        for c in rng.choice(g.n_pix - 8, 8, replace=False):
            flux[i, c:c + 3] += med * rng.uniform(0.5, 3.0) * np.array([1.0, 0.5, 0.2], np.float32)
    return M, d, flux


def test_clean_tensor_core_fit_parity():
    """Clean on the grouped tensor-core pipeline (split TF32 contractions,
    float-float normal equations; the Clean pass runs between K3 and K4 of a
    step): fits of spiky spectra against the oracle's Clean fits.  The
    contractions differ from FP32 in the last bits, so a mask decision on a
    borderline pixel may differ; most fits still agree within the tolerances,
    and Clean still beats no Clean."""
    from paper_2512_24840_gb300 import lasp
    lasp.load(build=True)
    g = S.SMALL
    M, d, flux = _spiky(g, 48, 95)
    th0 = np.asarray(d["theta0"], np.float32).astype(np.float64)
    ref = O.fit(M, flux, d["ivar"], d["good"], th0, max_steps=400, clean=1)
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    T = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)
    mo = dict(precision="tf32x3", fp64_normal_eq=1, max_steps=400)
    out = ip.fit(T(flux), T(d["ivar"]), T(d["good"], torch.uint8), T(th0), clean=1, **mo)
    th = out["theta"].double().cpu().numpy()
    ok = np.all(np.abs(th - ref["theta"])[:, :4] <= TOL, axis=1)
    print(f"tensor-core clean fit parity: {ok.mean():.3f} within tolerance")
    assert ok.mean() >= 0.85
    noc = ip.fit(T(flux), T(d["ivar"]), T(d["good"], torch.uint8), T(th0), **mo)
    clean_ref = O.fit(M, d["flux"], d["ivar"], d["good"], th0, max_steps=400)
    e_c = np.abs(th - clean_ref["theta"])[:, 0]
    e_n = np.abs(noc["theta"].double().cpu().numpy() - clean_ref["theta"])[:, 0]
    assert np.median(e_c) < np.median(e_n)


def test_served_tensor_core_clean_equals_one_shot():
    """Clean in tensor-core slot pools: each slot's mask stays in its W row
    between chunks, so a served fit is bitwise the one-shot fit at the same
    precision."""
    from paper_2512_24840_gb300 import lasp
    from paper_2512_24840_gb300.server import NativeServer
    lasp.load(build=True)
    g = S.SMALL
    M, d, flux = _spiky(g, 12, 97)
    th0 = np.asarray(d["theta0"], np.float32)
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    T = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)
    mo = dict(precision="tf32x3", fp64_normal_eq=1, max_steps=400, clean=1)
    one = ip.fit(T(flux), T(d["ivar"]), T(d["good"], torch.uint8), T(th0), **mo)
    srv = NativeServer({"s": ip}, {"s": 5}, chunk=7, **mo)
    ids = [srv.submit("s", flux[i], d["ivar"][i], d["good"][i], th0[i]) for i in range(12)]
    res = {r.rid: r for r in srv.run_until_idle()}
    srv.close()
    for k, rid in enumerate(ids):
        assert np.array_equal(res[rid].theta, one["theta"][k].cpu().numpy()), k
        assert res[rid].steps == int(one["steps"][k]) and res[rid].status == int(one["status"][k])


@pytest.mark.parametrize("chunk", [7, 31])
def test_served_clean_equals_one_shot(chunk):
    """Clean in served fits: each slot keeps its mask between chunks; with
    chunk 31 a chunk ends exactly on the first mask update (step 30), which
    still has to be applied before the slot is suspended."""
    from paper_2512_24840_gb300 import lasp
    from paper_2512_24840_gb300.server import NativeServer
    lasp.load(build=True)
    g = S.SMALL
    M, d = observed(g, 12, 92, snr=(30, 100), mask_frac=0.0)
    rng = np.random.default_rng(3)
    flux = d["flux"].copy()
    for i in range(12):
        med = np.median(flux[i])
        for c in rng.choice(g.n_pix - 8, 8, replace=False):
            flux[i, c:c + 3] += med * rng.uniform(0.5, 3.0) * np.array([1.0, 0.5, 0.2], np.float32)
    th0 = np.asarray(d["theta0"], np.float32)
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    T = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)
    one = ip.fit(T(flux), T(d["ivar"]), T(d["good"], torch.uint8), T(th0), max_steps=400, clean=1)
    srv = NativeServer({"s": ip}, {"s": 5}, chunk=chunk, max_steps=400, clean=1)
    ids = [srv.submit("s", flux[i], d["ivar"][i], d["good"][i], th0[i]) for i in range(12)]
    res = {r.rid: r for r in srv.run_until_idle()}
    srv.close()
    for k, rid in enumerate(ids):
        assert np.array_equal(res[rid].theta, one["theta"][k].cpu().numpy()), k
        assert res[rid].steps == int(one["steps"][k]) and res[rid].status == int(one["status"][k])
