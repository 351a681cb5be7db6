"""Bounded device waits that give up reach the caller as LASP_ETIMEOUT.

The testing hook lasp_test_wait_limit(0) makes the first table-copy wait of
every CTA of the tensor-core kernels give up at once.  That wait comes before
any MMA of the CTA; the copy it waited for is drained under the normal limit
before the CTA frees its TMEM and exits, so nothing asynchronous is left in
flight and the context stays usable: each test runs the same call again with
the normal limits and checks it against the undisturbed result.
"""
import ctypes as ct

import numpy as np
import pytest

import lasp_synth as S
from tests.helpers import observed, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def lasp():
    from paper_2512_24840_gb300 import lasp as L
    L.load(build=True)
    yield L
    L.test_wait_limit(-1)


def _interp(lasp, g):
    return lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)


def _batch(g, n, seed):
    M, d = observed(g, n, seed, snr=(30, 100), mask_frac=0.02)
    T = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)
    return [T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(np.asarray(d["theta0"], np.float32))]


def _out(N, deg=6):
    return dict(theta=torch.zeros((N, 5), device=DEV), loss=torch.zeros(N, device=DEV),
                steps=torch.zeros(N, dtype=torch.int32, device=DEV),
                status=torch.zeros(N, dtype=torch.int32, device=DEV),
                cont=torch.zeros((N, deg + 1), device=DEV), weight=torch.zeros(N, device=DEV))


def test_grouped_fit_reports_timeout_and_marks_every_fit(lasp):
    g = S.SMALL
    ip = _interp(lasp, g)
    args = _batch(g, 40, 301)
    mo = dict(precision="tf32x3", fp64_normal_eq=1, max_steps=200)
    before = ip.fit(*args, **mo)
    out = _out(40)
    lasp.test_wait_limit(0)
    try:
        with pytest.raises(lasp.LaspError) as ei:
            ip.fit(*args, out=out, **mo)
    finally:
        lasp.test_wait_limit(-1)
    assert ei.value.code == lasp.ETIMEOUT
    st = out["status"].cpu().numpy()
    assert np.all(st == lasp.ST_TIMEOUT), np.unique(st)       # no fit reported converged
    assert torch.isnan(out["loss"]).all()
    # the context is usable: the same fit with the normal limits gives the
    # undisturbed result again, bit for bit
    after = ip.fit(*args, **mo)
    assert torch.equal(after["theta"], before["theta"])
    assert torch.equal(after["status"], before["status"])
    assert not np.any(after["status"].cpu().numpy() & lasp.ST_TIMEOUT)
    ip.close()


def test_interp_eval_reports_timeout_with_nan_rows(lasp):
    g = S.LAMOST
    ip = _interp(lasp, g)
    d = S.draw_batch(g, 150, 302, noise=False, mask_frac=0.0)
    theta = torch.tensor(d["truth"], dtype=torch.float32, device=DEV)
    ref = ip.interp_eval(theta, "tf32x3")
    lasp.test_wait_limit(0)
    try:
        with pytest.raises(lasp.LaspError) as ei:
            ip.interp_eval(theta, "tf32x3")
    finally:
        lasp.test_wait_limit(-1)
    assert ei.value.code == lasp.ETIMEOUT
    again = ip.interp_eval(theta, "tf32x3")
    assert torch.equal(again, ref)
    ip.close()


def test_static_entry_point_reports_timeout_on_next_call(lasp):
    lib = lasp.load()
    lib.lasp_interp_eval_static.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p,
                                            ct.c_void_p, ct.c_int, ct.c_void_p]
    lib.lasp_interp_eval_static.restype = ct.c_int
    g = S.SMALL
    C = table(g.name)
    exps = np.ascontiguousarray(S.EXPS)
    d = lasp.InterpDesc(len(exps), g.n_pix, g.pad, g.dln, exps.ctypes.data,
                        (ct.c_double * 3)(*S.BASIS_LO), (ct.c_double * 3)(*S.BASIS_HI),
                        (ct.c_double * 5)(*S.BOX_LO), (ct.c_double * 5)(*S.BOX_HI))
    coeff = torch.tensor(C, device=DEV)
    dr = S.draw_batch(g, 130, 303, noise=False, mask_frac=0.0)
    theta = torch.tensor(dr["truth"], dtype=torch.float32, device=DEV)
    N = theta.shape[0]
    out = torch.zeros((N, g.n_model), device=DEV)
    st = ct.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        return lib.lasp_interp_eval_static(ct.byref(d), coeff.data_ptr(), N, theta.data_ptr(),
                                           out.data_ptr(), lasp.PREC["tf32x3"], st)

    assert call() == lasp.OK
    torch.cuda.synchronize()
    good = out.clone()
    lasp.test_wait_limit(0)
    try:
        assert call() == lasp.OK                 # enqueued; its waits give up on the GPU
        torch.cuda.synchronize()
    finally:
        lasp.test_wait_limit(-1)
    assert torch.isnan(out).all()                # every tile left uncomputed is NaN
    assert call() == lasp.ETIMEOUT               # reported (and cleared) by the next call
    assert call() == lasp.OK
    torch.cuda.synchronize()
    assert torch.equal(out, good)


def test_served_tensor_core_tick_reports_timeout(lasp):
    from paper_2512_24840_gb300.server import NativeServer
    g = S.SMALL
    ip = _interp(lasp, g)
    M, d = observed(g, 6, 304, snr=(30, 100), mask_frac=0.0)
    th0 = np.asarray(d["theta0"], np.float32)
    lasp.test_wait_limit(0)                      # captured into the pool's step graph
    try:
        srv = NativeServer({"s": ip}, {"s": 8}, chunk=8, precision="tf32x3", fp64_normal_eq=1,
                           max_steps=200)
    finally:
        lasp.test_wait_limit(-1)
    for i in range(6):
        srv.submit("s", d["flux"][i], d["ivar"][i], d["good"][i], th0[i])
    with pytest.raises(lasp.LaspError) as ei:
        srv.tick()
    assert ei.value.code == lasp.ETIMEOUT
    res = []
    got = ct.c_int()
    srv.lib.lasp_server_poll(srv._h, srv._buf, len(srv._buf), ct.byref(got))
    res = [int(r.status) for r in srv._buf[:got.value]]
    assert len(res) == 6 and all(s == lasp.ST_TIMEOUT for s in res)
    srv.close()
    ip.close()
