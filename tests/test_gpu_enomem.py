"""A device allocation that cannot be met is reported as LASP_ENOMEM and
leaves the library usable.

A slot pool of 64 million LAMOST-like slots asks for 1 TB of flux rows
alone, beyond the device's HBM, so its first cudaMalloc fails (an ordinary
error return, nothing is allocated).  The call must return LASP_ENOMEM with
no handle, and the failed allocation must not be reported again by a later
call: a pool that fits is made afterwards and a batch fit gives the same
result as before the failure.
"""
import ctypes as ct

import numpy as np
import pytest

import lasp_synth as S
from tests.helpers import observed, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_pool_beyond_hbm_is_enomem_and_not_sticky():
    from paper_2512_24840_gb300 import lasp
    lib = lasp.load(build=True)
    g = S.LAMOST
    ip = lasp.Interp.from_grid(g, table(g.name), S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    _, d = observed(g, 8, 411, snr=(30, 100), mask_frac=0.02)
    T = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)
    args = [T(d["flux"]), T(d["ivar"]), T(d["good"], torch.uint8), T(np.asarray(d["theta0"], np.float32))]
    before = ip.fit(*args, max_steps=100)
    torch.cuda.synchronize()

    P = ct.c_void_p
    lib.lasp_slots_create.argtypes = [P, ct.c_int, P, P]
    lib.lasp_slots_create.restype = ct.c_int
    lib.lasp_slots_free.argtypes = [P]
    opts = lasp.default_opts()
    n_huge = 64 * 1024 * 1024
    assert n_huge * g.n_pix * 4 > 2 * torch.cuda.get_device_properties(0).total_memory
    h = ct.c_void_p()
    rc = lib.lasp_slots_create(ip._h, n_huge, ct.byref(opts), ct.byref(h))
    assert rc == lasp.ENOMEM and not h.value

    # the failure is not re-reported: a pool that fits, then the same fit again
    rc = lib.lasp_slots_create(ip._h, 4, ct.byref(opts), ct.byref(h))
    assert rc == lasp.OK and h.value
    lib.lasp_slots_free(h)
    after = ip.fit(*args, max_steps=100)
    torch.cuda.synchronize()
    for k in ("theta", "steps", "status"):
        assert torch.equal(before[k], after[k]), k
