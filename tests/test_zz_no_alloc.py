"""The allocation-free contraction entry point against the handle-based one.

lasp_interp_eval_static serves callers that may not allocate device memory
(a framework that owns all device memory through its own pool, a serving loop
with a fixed memory budget): it needs no handle and keeps its scratch in a
static device array.  This file is named to be collected last, so a run that
stops at the first failure has run every other test before it.  It also
passes on its own in a fresh process.
"""
import ctypes as ct

import numpy as np
import pytest

import lasp_synth as S
from tests.helpers import table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Same tolerance as the tensor-core parity tests: split TF32 to 1e-5 of the
# spectrum maximum; single-pass TF32 and BF16 as there.
TOLS = {"tf32x3": 1e-5, "tf32": 4e-3, "bf16": 3e-2}


@pytest.fixture(scope="module")
def lasp():
    from paper_2512_24840_gb300 import lasp as L
    lib = L.load(build=True)
    lib.lasp_interp_eval_static.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p,
                                            ct.c_void_p, ct.c_int, ct.c_void_p]
    lib.lasp_interp_eval_static.restype = ct.c_int
    return L


def _desc(lasp, grid, exps):
    return lasp.InterpDesc(len(exps), grid.n_pix, grid.pad, grid.dln, exps.ctypes.data,
                           (ct.c_double * 3)(*S.BASIS_LO), (ct.c_double * 3)(*S.BASIS_HI),
                           (ct.c_double * 5)(*S.BOX_LO), (ct.c_double * 5)(*S.BOX_HI))


def _rel_err(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return (np.abs(a - b).max(axis=1) / np.abs(b).max(axis=1)).max()


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16"])
@pytest.mark.parametrize("grid", [S.SMALL, S.LAMOST], ids=lambda g: g.name)
def test_static_entry_point_matches_handle_path(lasp, grid, prec):
    lib = lasp.load()
    C = table(grid.name)
    exps = np.ascontiguousarray(S.EXPS)
    ip = lasp.Interp.from_grid(grid, C, exps, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    dev = torch.device("cuda:0")
    coeff = torch.tensor(C, device=dev)
    d = _desc(lasp, grid, exps)
    stream = torch.cuda.current_stream()
    for call in range(2):                      # two calls in a row, different inputs
        draws = S.draw_batch(grid, 200 + 37 * call, 900 + call, noise=False, mask_frac=0.0)
        theta = torch.tensor(draws["truth"], dtype=torch.float32, device=dev)
        N = theta.shape[0]
        out = torch.full((N, grid.n_model), float("nan"), device=dev)
        rc = lib.lasp_interp_eval_static(ct.byref(d), coeff.data_ptr(), N, theta.data_ptr(),
                                         out.data_ptr(), lasp.PREC[prec],
                                         ct.c_void_p(stream.cuda_stream))
        assert rc == 0, lasp.strerror(rc)
        ref = ip.interp_eval(theta, prec)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel_err(out, ref) <= TOLS[prec]


def test_static_entry_point_rejects_oversize_and_bad_args(lasp):
    lib = lasp.load()
    exps = np.ascontiguousarray(S.EXPS)
    big = S.Grid("big", 9000, 3600.0, S.DESI.dln)          # n_model > 8192
    d = _desc(lasp, big, exps)
    dev = torch.device("cuda:0")
    x = torch.zeros((4, 5), device=dev)
    y = torch.zeros((4, big.n_model), device=dev)
    coeff = torch.zeros((len(exps), big.n_model), device=dev)
    assert lib.lasp_interp_eval_static(ct.byref(d), coeff.data_ptr(), 4, x.data_ptr(), y.data_ptr(),
                                       lasp.PREC["tf32"], None) == lasp.EINVAL
    d2 = _desc(lasp, S.SMALL, exps)
    assert lib.lasp_interp_eval_static(ct.byref(d2), coeff.data_ptr(), 4, x.data_ptr(), y.data_ptr(),
                                       lasp.PREC["fp32"], None) == lasp.EINVAL
