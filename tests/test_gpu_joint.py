"""Joint loss (LASP_LOSS_JOINT, Eq. 9 read literally: one RMS over the group,
group stop rules) on the grouped tensor-core pipeline against the oracle's
joint fit."""
import numpy as np
import pytest

import lasp_synth as S
from oracle import oracle as O
from tests.helpers import TOL, observed, table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ip():
    from paper_2512_24840_gb300 import lasp
    lasp.load(build=True)
    return lasp.Interp.from_grid(S.LAMOST, table(S.LAMOST.name), S.EXPS, S.BASIS_LO, S.BASIS_HI,
                                 S.BOX_LO, S.BOX_HI)


def _T(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dt)


def _fit(ip, d, **opts):
    out = ip.fit(_T(d["flux"]), _T(d["ivar"]), _T(d["good"], torch.uint8), _T(d["theta0"]), **opts)
    torch.cuda.synchronize()
    return {k: v.double().cpu().numpy() for k, v in out.items()}


def test_joint_matches_oracle_joint(ip):
    M, d = observed(S.LAMOST, 64, 81, snr=(5, 100), mask_frac=0.05)
    d["theta0"] = np.asarray(d["theta0"], np.float32).astype(np.float64)
    d["good"][7] = 0                                  # no data: outside the group
    ref = O.fit_joint(M, d["flux"], d["ivar"], d["good"], d["theta0"], max_steps=500)
    out = _fit(ip, d, max_steps=500, precision="tf32x3", fp64_normal_eq=1, loss_mode="joint")
    members = np.array([i for i in range(64) if i != 7])
    assert out["status"][7] == 64 and ref["status"][7] == 64
    steps = np.unique(out["steps"][members])
    assert len(steps) == 1 and len(np.unique(out["status"][members].astype(int) & 7)) == 1
    print(f"joint: GPU stops at step {int(steps[0])}, oracle at {int(ref['steps'][members][0])}")
    assert abs(int(steps[0]) - int(ref["steps"][members][0])) <= 3
    ok = np.all(np.abs(out["theta"][members] - ref["theta"][members])[:, :4] <= TOL, axis=1)
    print(f"joint parity {ok.mean():.3f}")
    assert ok.mean() >= 0.9


def test_joint_group_of_one_is_the_separable_fit(ip):
    M, d = observed(S.LAMOST, 1, 82, snr=(30, 60), mask_frac=0.05)
    o = dict(max_steps=400, precision="tf32x3", fp64_normal_eq=1)
    sep = _fit(ip, d, **o)
    one = _fit(ip, d, loss_mode="joint", **o)
    assert one["steps"][0] == sep["steps"][0]
    assert np.all(np.abs(one["theta"] - sep["theta"])[:, :4] <= TOL / 10)


def test_joint_needs_the_grouped_pipeline(ip):
    from paper_2512_24840_gb300 import lasp
    M, d = observed(S.LAMOST, 2, 83)
    with pytest.raises(lasp.LaspError) as e:
        _fit(ip, d, loss_mode="joint")                # FP32 fused kernel: per-spectrum only
    assert e.value.code == lasp.EINVAL
