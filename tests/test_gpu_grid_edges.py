"""Grids at the size limits of the library.  Each thread of a fit kernel owns
16 model pixels, so the block size follows the model grid n_model = n_pix +
2 pad: 256 threads up to 4096 model pixels, 512 up to 8192, the largest the
library takes.  Three grids:

- 16 observed pixels, the fewest accepted (LAMOST-like step, 56 model
  pixels: one partial 128-pixel tile on the tensor-core path);
- 4090 observed pixels on the LAMOST-like step (margin 20): 4130 model
  pixels, just past 256 threads' reach while the observed pixels alone
  would still fit it;
- 8124 observed pixels on the DESI-like step (margin 34): exactly 8192 model
  pixels.

On each: forward model and hand-written adjoint against the oracle; on the
two large grids also fixed-step batch fits in FP32 and at split TF32 against
the oracle, the served form (resumable slots) bitwise equal to the batch fit,
and the stage-9 errors against the oracle."""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import GRAD_RTOL_THETA, TOL, observed, oracle_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GRIDS = [S.Grid("min16", 16, 4200.0, S.LAMOST.dln),
         S.Grid("edge4090", 4090, 3700.0, S.LAMOST.dln),
         S.Grid("max8124", 8124, 3600.0, S.DESI.dln)]
# fixed Adam steps of the parity fits (the two large grids; on 16 pixels the
# 12 unknowns, 5 parameters and 7 continuum terms, leave the path so poorly
# conditioned that FP32 rounding moves Teff by about 1 K within 4 steps:
# measured 0.87 K in FP32 and 1.26 K at split TF32, so no trajectory parity
# is asserted there)
NSTEPS = {"edge4090": 12, "max8124": 12}


def q32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def T(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)


def H(t):
    return t.detach().double().cpu().numpy()


_cache = {}


def setup(grid):
    from paper_2512_24840_gb300 import lasp
    lasp.load(build=True)
    if grid.name not in _cache:
        C = S.make_table(grid)
        ip = lasp.Interp.from_grid(grid, C, S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
        _cache[grid.name] = (ip, oracle_model(grid, C=C))
    return _cache[grid.name]


def test_grid_sizes():
    assert GRIDS[0].n_model == 56
    assert GRIDS[1].n_model == 4130 and GRIDS[1].n_pix <= 16 * 256 < GRIDS[1].n_model
    assert GRIDS[2].n_model == 8192


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: g.name)
def test_forward_and_adjoint_at_block_edges(grid):
    ip, M = setup(grid)
    th = q32([[3500.0, 0.5, -2.5, -300.0, 30.0],        # box corners: widest shift and
              [7500.0, 5.5, 1.0, 300.0, 200.0],         # the widest kernel (h = H)
              [5200.0, 3.1, -0.4, 41.0, 95.0]])
    rng = np.random.default_rng(17)
    b = q32(np.c_[np.ones(3), rng.normal(0, 0.05, (3, 6))])
    got = H(ip.forward(T(th), T(b)))
    ref = O.model_batch(M, th, b)
    err = (np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)).max()
    print(f"{grid.name} forward: max rel err {err:.2e} (bound 1e-5)")
    assert err < 1e-5
    gm = q32(rng.normal(0, 1, (3, grid.n_pix)))
    gth, gb = ip.backward(T(th), T(b), T(gm))
    gth, gb = H(gth), H(gb)
    for i in range(3):
        rth, rb = O.model_vjp(M, th[i], b[i], gm[i])
        scale = np.abs(rth) + 1e-3 * np.abs(rth).max()
        assert np.all(np.abs(gth[i] - rth) <= GRAD_RTOL_THETA * scale), (i, gth[i], rth)
        np.testing.assert_allclose(gb[i], rb, rtol=1e-4, atol=1e-4 * np.abs(rb).max())


@pytest.mark.parametrize("grid", GRIDS[1:], ids=lambda g: g.name)
def test_fit_at_block_edges(grid):
    """Nine spectra (two CTAs of the batch fit and a ragged third), a fixed
    number of Adam steps with the stop rules off, in FP32 and on the split-TF32
    tensor-core pipeline: same step counts as the oracle and every spectrum
    within the parameter tolerances; then the served form."""
    ip, M = setup(grid)
    _, d = observed(grid, 9, 801, M=M, snr=(30, 100), mask_frac=0.05)
    d["theta0"] = q32(d["theta0"])
    args = (T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(d["theta0"]))
    n = NSTEPS[grid.name]
    ref = O.fit(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_steps=n, tol=0.0)
    for prec, ne in (("fp32", 0), ("tf32x3", 1)):
        out = ip.fit(*args, max_steps=n, tol=0.0, precision=prec, fp64_normal_eq=ne)
        torch.cuda.synchronize()
        assert np.all(H(out["steps"]) == ref["steps"]), prec
        err = np.abs(H(out["theta"]) - ref["theta"])[:, :4]
        print(f"{grid.name} {prec} fixed-step fit ({n} steps): max |dtheta| {err.max(axis=0)} (bounds {TOL})")
        assert np.all(err <= TOL), (prec, err.max(axis=0))

    from paper_2512_24840_gb300.server import DevicePool, Server
    one = ip.fit(*args, max_steps=40)
    srv = Server({"s": DevicePool(ip, 4, max_steps=40)}, chunk=9)
    ids = [srv.submit("s", d["flux"][i], d["ivar"][i], d["good"][i], d["theta0"][i]) for i in range(9)]
    res = {r.rid: r for r in srv.run_until_idle()}
    srv.close()
    for k, rid in enumerate(ids):
        assert np.array_equal(res[rid].theta, H(one["theta"])[k]), k
        assert res[rid].steps == int(H(one["steps"])[k])


@pytest.mark.parametrize("grid", GRIDS[1:], ids=lambda g: g.name)
def test_errors_at_grid_edges(grid):
    """Stage 9 on the two large grids.  (On 16 pixels the 5 parameters and 7
    continuum terms leave J^T J nearly singular, sigma(Teff) of order 1e6 K, so
    a comparison of FP32 sums with the oracle's differences says nothing.)"""
    ip, M = setup(grid)
    _, d = observed(grid, 6, 803, M=M, snr=(30, 100), mask_frac=0.05)
    d["theta0"] = q32(d["theta0"])
    e = ip.errors(T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(d["theta0"]))
    sig = H(e["sigma"])
    ref = np.stack([O.errors(M, d["flux"][i], d["ivar"][i], d["good"][i], d["theta0"][i])["sigma"]
                    for i in range(6)])
    rel = np.abs(sig - ref) / ref
    print(f"{grid.name} stage-9 sigma: median rel. error {np.median(rel):.2e} (bound 1e-3)")
    assert np.median(rel) < 1e-3 and np.all(H(e["status"]) == 0), rel
