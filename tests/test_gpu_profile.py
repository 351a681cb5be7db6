"""lasp_profile: per-kernel device times, and results unchanged by it.

With profiling on, every kernel of a call is bracketed by CUDA events and
the tensor-core fit launches its steps one by one instead of replaying the
step graph; the arithmetic is the same, so every result is bitwise the one
of the unprofiled call."""
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
    L.profile(False)


def test_profile_times_each_kernel_and_changes_nothing(lasp):
    g = S.LAMOST
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    M, d = observed(g, 200, 401, snr=(10, 100), mask_frac=0.05)
    T = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)
    args = [T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(np.asarray(d["theta0"], np.float32))]
    forms = [dict(max_steps=300), dict(max_steps=300, precision="tf32x3", fp64_normal_eq=1),
             dict(max_steps=300, fp64_normal_eq=2), dict(max_steps=300, clean=1)]
    plain = [ip.fit(*args, **o) for o in forms]
    e_plain = ip.errors(*args[:3], plain[0]["theta"], with_cov=False)
    lasp.profile(True)
    try:
        lasp.profile_read()
        prof = [ip.fit(*args, **o) for o in forms]
        e_prof = ip.errors(*args[:3], prof[0]["theta"], with_cov=False)
        times = lasp.profile_read()
    finally:
        lasp.profile(False)
    for a, b in zip(plain, prof):
        assert torch.equal(a["theta"], b["theta"]) and torch.equal(a["status"], b["status"])
        assert torch.equal(a["steps"], b["steps"])
    assert torch.equal(e_plain["sigma"], e_prof["sigma"])
    for name in ("fit_prep_kernel", "fit_multi_kernel", "fit_multi_kernel<ne64>", "fit_multi_kernel<clean>",
                 "errors_kernel",
                 "k0_prep", "k1_interp", "k2_rest", "k3_back", "k4_adam"):
        assert name in times, (name, sorted(times))
        launches, ms = times[name]
        assert launches >= 1 and ms > 0.0
    steps = int(prof[1]["steps"].max())
    assert times["k1_interp"][0] >= steps + 1            # one K1 per step of the longest fit
    assert lasp.profile_read() == {}                      # read clears
    ip.close()


def test_profile_times_a_served_tick(lasp):
    """The slot calls behind a served tick are profiled too: the admission
    copies, the scatter and prep kernels, the running-slot list, the step
    kernel and the result fetch, one entry each."""
    from paper_2512_24840_gb300.server import NativeServer
    g = S.LAMOST
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    M, d = observed(g, 12, 402, snr=(30, 100), mask_frac=0.02)
    th0 = np.asarray(d["theta0"], np.float32)
    srv = NativeServer({"l": ip}, {"l": 8}, chunk=20, max_steps=300)
    for i in range(12):
        srv.submit("l", d["flux"][i], d["ivar"][i], d["good"][i], th0[i])
    lasp.profile(True)
    try:
        lasp.profile_read()
        n_ticks = 0
        while srv.pending():
            srv.tick_arrays()
            n_ticks += 1
        times = lasp.profile_read()
    finally:
        lasp.profile(False)
    srv.close()
    for name in ("slots_admit_h2d", "slots_scatter_kernel", "fit_prep_slots_kernel", "slots_running_list",
                 "fit_multi_kernel<slots>", "slots_fetch_d2h"):
        assert name in times, (name, sorted(times))
        assert times[name][1] > 0.0
    assert times["slots_fetch_d2h"][0] == n_ticks           # one result fetch a tick
    assert times["fit_multi_kernel<slots>"][0] == n_ticks   # one step launch a tick
    assert times["slots_admit_h2d"][0] >= 2                 # 8 slots for 12 requests: two admissions
    ip.close()
