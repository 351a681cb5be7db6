"""Served fits: requests on two grids (LAMOST-like 3909 px and DESI-like
7781 px) with uneven masks are admitted into small slot pools (forcing slot
reuse) and stepped in chunks of 7 Adam steps on two streams.  Each result is
bitwise the one the same spectrum gets when fitted alone with
lasp_fit_batch -- alone and in the mix are the same."""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import oracle_model, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _observed(grid, n, seed):
    M = oracle_model(grid)
    d = S.draw_batch(grid, n, seed, snr=(5, 100), mask_frac=0.0, mask_frac_max=0.2)
    flux, ivar = S.finish_obs(O.model_batch(M, d["truth"], d["b_true"]), d)
    th0 = np.asarray(d["theta0"], np.float32)
    return flux, ivar, d["good"], th0


@pytest.mark.parametrize("kind", ["python", "native", "native_small_ring", "native_tf32x3",
                                  "python_tf32x3"])
def test_served_equals_alone(kind):
    """The Python scheduler over slot pools and the library's native scheduler
    (lasp_server_*; with a ring smaller than the arrivals its overflow path
    and LASP_EBUSY are exercised too)."""
    from paper_2512_24840_gb300 import lasp
    from paper_2512_24840_gb300.server import DevicePool, NativeServer, Server
    lasp.load(build=True)
    ips = {g.name: lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI,
                                         S.BOX_LO, S.BOX_HI) for g in (S.LAMOST, S.DESI)}
    data = {"lamost": _observed(S.LAMOST, 40, 61), "desi": _observed(S.DESI, 24, 62)}
    # served mixed precision: the grouped tensor-core pipeline runs over the slots
    fo = dict(max_steps=400)
    if kind.endswith("tf32x3"):
        fo.update(precision="tf32x3", fp64_normal_eq=1)
    if kind.startswith("python"):
        pools = {"lamost": DevicePool(ips["lamost"], 16, **fo),
                 "desi": DevicePool(ips["desi"], 8, **fo)}
        srv = Server(pools, chunk=7)
    else:
        ring = {"lamost": 3, "desi": 2} if kind == "native_small_ring" else None
        srv = NativeServer(ips, {"lamost": 16, "desi": 8}, chunk=7, ring=ring, **fo)
    rids = {}
    order = [("lamost", i) for i in range(40)] + [("desi", i) for i in range(24)]
    np.random.default_rng(3).shuffle(order)
    results = {}
    for k, (lane, i) in enumerate(order):        # arrivals interleaved with ticks
        f, iv, gd, th = data[lane]
        rids[srv.submit(lane, f[i], iv[i], gd[i], th[i])] = (lane, i)
        if k % 5 == 4:
            for r in srv.tick():
                results[r.rid] = r
    for r in srv.run_until_idle():
        results[r.rid] = r
    assert len(results) == 64
    dev = torch.device("cuda:0")
    for lane in ("lamost", "desi"):
        f, iv, gd, th = data[lane]
        for i in range(len(f)):
            one = ips[lane].fit(torch.tensor(f[i:i + 1], device=dev), torch.tensor(iv[i:i + 1], device=dev),
                                torch.tensor(gd[i:i + 1], device=dev), torch.tensor(th[i:i + 1], device=dev),
                                **fo)
            rid = [r for r, v in rids.items() if v == (lane, i)][0]
            got = results[rid]
            assert np.array_equal(got.theta, one["theta"][0].cpu().numpy()), (lane, i)
            assert got.steps == int(one["steps"][0]) and got.status == int(one["status"][0])
    assert srv.pending() == 0
    lat = np.array([r.latency for r in results.values()])
    assert np.all(lat > 0)
    srv.close()


def test_server_created_while_a_fit_runs():
    """A pool made while a one-shot fit is still running on the default
    stream: its zero fills must be done before the scheduler's non-blocking
    lane streams admit into it, or the first admitted spectra are wiped."""
    from paper_2512_24840_gb300 import lasp
    from paper_2512_24840_gb300.server import NativeServer
    lasp.load(build=True)
    g = S.LAMOST
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    f, iv, gd, th = _observed(g, 8, 63)
    dev = torch.device("cuda:0")
    big = np.repeat(f, 256, axis=0)              # 2048 spectra keep the default stream busy
    T = lambda a: torch.tensor(a, device=dev)
    busy = ip.fit(T(big), T(np.repeat(iv, 256, axis=0)), T(np.repeat(gd, 256, axis=0)),
                  T(np.repeat(th, 256, axis=0)), max_steps=400)
    srv = NativeServer({"l": ip}, {"l": 8}, chunk=7, max_steps=400)   # no host sync before this
    rids = [srv.submit("l", f[i], iv[i], gd[i], th[i]) for i in range(8)]
    res = {r.rid: r for r in srv.run_until_idle()}
    srv.close()
    for i, rid in enumerate(rids):
        assert np.array_equal(res[rid].theta, busy["theta"][256 * i].cpu().numpy()), i
        assert res[rid].status == int(busy["status"][256 * i])


@pytest.mark.parametrize("hint", ["one", "true", "too_many"])
def test_step_running_hint_only_sizes_the_launch(hint):
    """lasp_slots_step_running sizes the launch from the caller's count of
    running slots; a wrong count (1, or more than the pool holds) changes the
    schedule, never a result."""
    from paper_2512_24840_gb300 import lasp
    from paper_2512_24840_gb300.server import DevicePool, Request
    lasp.load(build=True)
    g = S.LAMOST
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    f, iv, gd, th = _observed(g, 24, 64)
    dev = torch.device("cuda:0")
    one = ip.fit(torch.tensor(f, device=dev), torch.tensor(iv, device=dev), torch.tensor(gd, device=dev),
                 torch.tensor(th, device=dev), max_steps=400)
    pool = DevicePool(ip, 40, max_steps=400)
    slots = list(range(3, 27))
    pool.admit(slots, [Request(k, "l", f[k], iv[k], gd[k], th[k]) for k in range(24)])
    n_hint = {"one": 1, "true": 24, "too_many": 1000}[hint]
    for _ in range(40):
        pool.step(11, n_hint)
        pool.fetch()
        status, theta, loss, steps = pool.wait()
        if not np.any(status[slots] == lasp.ST_RUNNING):
            break
    for k, s in enumerate(slots):
        assert np.array_equal(theta[s], one["theta"][k].cpu().numpy()), k
        assert steps[s] == int(one["steps"][k])
    pool.close()


def test_native_ticks_as_arrays_equal_the_result_objects():
    """NativeServer.tick_arrays hands back a tick's finished fits as one
    structured array (what the bench's native scheduler uses); its fields are
    those of the Result objects of tick()."""
    from paper_2512_24840_gb300 import lasp
    from paper_2512_24840_gb300.server import NativeServer
    lasp.load(build=True)
    g = S.LAMOST
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    f, iv, gd, th = _observed(g, 20, 65)
    got = {}
    for how in ("objects", "arrays"):
        srv = NativeServer({"l": ip}, {"l": 8}, chunk=9, max_steps=400)
        rids = [srv.submit("l", f[i], iv[i], gd[i], th[i]) for i in range(20)]
        if how == "objects":
            res = {r.rid: (r.theta, r.steps, r.status, r.latency) for r in srv.run_until_idle()}
        else:
            a = srv.run_until_idle_arrays()
            res = {int(r["tag"]): (r["theta"], int(r["steps"]), int(r["status"]),
                                   (int(r["t_done_ns"]) - int(r["t_submit_ns"])) * 1e-9) for r in a}
        srv.close()
        got[how] = [res[rid] for rid in rids]
    for a, b in zip(got["objects"], got["arrays"]):
        assert np.array_equal(a[0], b[0]) and a[1] == b[1] and a[2] == b[2]
        assert a[3] > 0 and b[3] > 0


@pytest.mark.parametrize("ring", [32, 5])
def test_native_submit_many_equals_single_submits(ring):
    """submit_many hands rows to lasp_server_submit_n in one call; with a ring
    smaller than the batch the rows it has no room for wait on the host and
    enter at later ticks.  Either way each request's result is bitwise the one
    of a request submitted on its own, and ids follow the row order."""
    from paper_2512_24840_gb300 import lasp
    from paper_2512_24840_gb300.server import NativeServer
    lasp.load(build=True)
    g = S.LAMOST
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    f, iv, gd, th = _observed(g, 20, 66)
    srv = NativeServer({"l": ip}, {"l": 8}, chunk=9, max_steps=400)
    rids = [srv.submit("l", f[i], iv[i], gd[i], th[i]) for i in range(20)]
    one = {int(r["tag"]): r for r in srv.run_until_idle_arrays()}
    srv.close()
    srv = NativeServer({"l": ip}, {"l": 8}, chunk=9, ring={"l": ring}, max_steps=400)
    head = srv.submit("l", f[0], iv[0], gd[0], th[0])
    fb, ivb, gdb, thb = f[1:].copy(), iv[1:].copy(), gd[1:].copy(), th[1:].copy()
    ids = srv.submit_many("l", fb, ivb, gdb, thb)
    assert ids.tolist() == list(range(head + 1, head + 20))
    fb[:] = np.nan                                  # the caller's rows may be reused on return
    many = {int(r["tag"]): r for r in srv.run_until_idle_arrays()}
    srv.close()
    assert len(many) == 20
    for k in range(20):
        a, b = one[rids[k]], many[head + k]
        assert np.array_equal(a["theta"], b["theta"]) and a["steps"] == b["steps"], k
        assert a["status"] == b["status"] and a["loss"] == b["loss"], k
    ip.close()


@pytest.mark.parametrize("ring", [32, 5])
def test_python_submit_many_equals_single_submits(ring):
    """The Python scheduler's submit_many stages a batch of rows into the
    pool's ring with one copy per array (rows without ring room keep copies
    and are staged at admission); each result is bitwise the one of a
    request submitted on its own."""
    from paper_2512_24840_gb300 import lasp
    from paper_2512_24840_gb300.server import DevicePool, Server
    lasp.load(build=True)
    g = S.LAMOST
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    f, iv, gd, th = _observed(g, 20, 67)
    srv = Server({"l": DevicePool(ip, 8, max_steps=400)}, chunk=9)
    rids = [srv.submit("l", f[i], iv[i], gd[i], th[i]) for i in range(20)]
    one = {r.rid: r for r in srv.run_until_idle()}
    srv.close()
    srv = Server({"l": DevicePool(ip, 8, ring=ring, max_steps=400)}, chunk=9)
    fb, ivb, gdb, thb = f.copy(), iv.copy(), gd.copy(), th.copy()
    ids = srv.submit_many("l", fb, ivb, gdb, thb)
    fb[:] = np.nan                                  # the caller's rows may be reused on return
    many = {r.rid: r for r in srv.run_until_idle()}
    srv.close()
    assert len(many) == 20
    for k in range(20):
        a, b = one[rids[k]], many[int(ids[k])]
        assert np.array_equal(a.theta, b.theta) and a.steps == b.steps and a.status == b.status, k
    ip.close()
