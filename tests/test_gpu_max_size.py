"""Model grids at the edges of the fit kernels' thread blocks.  Each thread of
a fit kernel owns 16 model pixels, so the block size follows the model grid
n_model = n_pix + 2 pad: 256 threads up to 4096 model pixels, 512 up to
8192, the largest the library takes.  Two grids sit at those edges:

- 4090 observed pixels on the LAMOST-like step (margin 20): 4130 model
  pixels, just past 256 threads' reach while the observed pixels alone
  would still fit it;
- 8124 observed pixels on the DESI-like step (margin 34): exactly 8192 model
  pixels.

On each: forward model, hand-written adjoint, a fixed-step batch fit against
the oracle, and the served form (resumable slots) bitwise equal to the batch
fit."""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import GRAD_RTOL_THETA, TOL, observed, oracle_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GRIDS = [S.Grid("edge4090", 4090, 3700.0, S.LAMOST.dln),
         S.Grid("max8124", 8124, 3600.0, S.DESI.dln)]


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
    assert GRIDS[0].n_model == 4130 and GRIDS[0].n_pix <= 16 * 256 < GRIDS[0].n_model
    assert GRIDS[1].n_model == 8192


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


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: g.name)
def test_fit_at_block_edges(grid):
    """Nine spectra (two CTAs of the batch fit and a ragged third), 12 Adam
    steps with the stop rules off: same step counts as the oracle and every
    spectrum within the parameter tolerances; then the served form."""
    ip, M = setup(grid)
    _, d = observed(grid, 9, 801, M=M, snr=(30, 100), mask_frac=0.05)
    d["theta0"] = q32(d["theta0"])
    args = (T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(d["theta0"]))
    out = ip.fit(*args, max_steps=12, tol=0.0)
    torch.cuda.synchronize()
    ref = O.fit(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_steps=12, tol=0.0)
    assert np.all(H(out["steps"]) == ref["steps"])
    err = np.abs(H(out["theta"]) - ref["theta"])[:, :4]
    print(f"{grid.name} fixed-step fit: max |dtheta| {err.max(axis=0)} (bounds {TOL})")
    assert np.all(err <= TOL), err.max(axis=0)

    from paper_2512_24840_gb300.server import DevicePool, Server
    one = ip.fit(*args, max_steps=40)
    srv = Server({"s": DevicePool(ip, 4, max_steps=40)}, chunk=9)
    ids = [srv.submit("s", d["flux"][i], d["ivar"][i], d["good"][i], d["theta0"][i]) for i in range(9)]
    res = {r.rid: r for r in srv.run_until_idle()}
    srv.close()
    for k, rid in enumerate(ids):
        assert np.array_equal(res[rid].theta, H(one["theta"])[k]), k
        assert res[rid].steps == int(H(one["steps"])[k])
