"""The no-allocation penalty entry point, for callers that must not call
cudaMalloc/cudaFree (memory owned by another framework's allocator, or loops
where cudaFree's device-wide synchronisation is unacceptable).

It is checked through the C ABI against the plan-based sps_penalty_apply on
two calls in a row (the second call reuses the shared scratch left by the
first), against the oracle's assembled Lambda, and for the promise it exists
for: after its first call on the device, further calls leave the device's
free memory unchanged.  This file runs last so that a failure here stops a -x
run only after every other test has run; it passes alone in a fresh process
as well.
"""
import numpy as np
import pytest

from oracle import sampled

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1901_00654_gb300.binding")
torch = pytest.importorskip("torch")

FP64_TOL = 1e-12


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("P,intervals,lo,hi,scale", [
    (3, [8, 16, 8], [0.0, -1.0, 0.5], [1.0, 1.0, 2.0], 1.0),
    (2, [32, 16], None, None, 1.0),
    (4, [4, 8, 4, 4], None, None, 1.0),
    (1, [64], None, None, 1.0),
    (5, [4, 4, 4, 4, 4], None, None, 1.0),
    (3, [8, 8, 8], None, None, 2.5),
])
def test_noalloc_penalty_matches_plan_path_twice(P, intervals, lo, hi, scale):
    r = np.random.default_rng(P)
    lo_ = lo if lo is not None else [0.0] * P
    hi_ = hi if hi is not None else [1.0] * P
    x = np.stack([lo_[p] + (hi_[p] - lo_[p]) * r.random(500) for p in range(P)], axis=1)
    # one level and the inner coarse CG: no dense coarse matrix, so any grid size is accepted
    with B.Plan(P, intervals, 1, 1e-2, lo_, hi_, coarse_cg=1) as plan:
        plan.set_points(x, np.sin(x[:, 0]))
        K = plan.K
        for call in range(2):
            vh = r.standard_normal(K)
            v = torch.from_numpy(vh).cuda()
            ref = torch.zeros(K, dtype=torch.float64, device="cuda")
            B.sps_penalty_apply(plan.h, 1, B.SPS_PREC_FP64, v, ref)
            ref *= scale
            u = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
            B.sps_penalty_apply_noalloc(P, intervals, lo, hi, scale, v, u)
            torch.cuda.synchronize()
            assert _rel(u, ref) < FP64_TOL, (call, _rel(u, ref))
            oracle = torch.from_numpy(scale * sampled.penalty_apply_kron(vh, lo_, hi_, intervals, 3))
            assert _rel(u.cpu(), oracle) < 10 * FP64_TOL, (call, _rel(u.cpu(), oracle))


def test_noalloc_calls_leave_free_memory_unchanged():
    P, intervals = 3, [16, 16, 16]
    K = 19 ** 3
    v = torch.randn(K, dtype=torch.float64, device="cuda")
    u = torch.empty_like(v)
    B.sps_penalty_apply_noalloc(P, intervals, None, None, 1.0, v, u)   # first call: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        B.sps_penalty_apply_noalloc(P, intervals, None, None, 1.0, v, u)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_grids_above_the_limit_and_overlap():
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SpsError) as e:
        B.sps_penalty_apply_noalloc(3, [64, 64, 64], None, None, 1.0, v, v)   # 67^3 > 262144
    assert e.value.code == B.SPS_EINVAL
    assert "262144" in str(e.value)
    w = torch.zeros(2 * 67, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SpsError) as e:
        B.sps_penalty_apply_noalloc(1, [64], None, None, 1.0, w[:67], w[10:77])
    assert e.value.code == B.SPS_EINVAL
