"""The CUDA path at the full sizes of the workloads, in the launch
configuration bench.py times, checked on outputs the oracle can compute one
coefficient at a time and on properties that hold at any size."""
import hashlib
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import sampled, spline
from tests.gpu_util import rel_err

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1901_00654_gb300.binding")
torch = pytest.importorskip("torch")


def _device(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def scale():
    pr = W.scale()
    plan = B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi)
    plan.set_points(_device(pr.x), _device(pr.y))
    yield pr, plan
    plan.close()


def _sample_coefficients(pr, plan, count, seed):
    """Random coefficients plus the ones with the largest right-hand side
    (inside the clusters, where runs are long)."""
    b = np.zeros(plan.K)
    B.sps_rhs(plan.h, b)
    r = np.random.default_rng(seed)
    ks = np.concatenate([r.choice(plan.K, count // 2, replace=False), np.argsort(-np.abs(b))[:count // 2]])
    return np.unique(ks)


def test_scale_sort_bit_exact(scale):
    pr, plan = scale
    perm_o, key_o, _ = spline.sort_permutation(pr.x, pr.lo, pr.hi, pr.intervals)
    perm = np.zeros(pr.n, dtype=np.int64)
    key = np.zeros(pr.n, dtype=np.uint64)
    B.sps_get_sort(plan.h, perm, key)
    np.testing.assert_array_equal(perm, perm_o)
    np.testing.assert_array_equal(key, key_o[perm_o])


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_scale_apply_sampled(scale, prec, tol):
    pr, plan = scale
    v = np.random.default_rng(3).standard_normal(plan.K)
    u = np.zeros_like(v)
    B.sps_apply(plan.h, pr.levels, prec, v, u)
    ks = _sample_coefficients(pr, plan, 64, 4)
    ref = sampled.apply_rows(pr.x, v, ks, pr.lo, pr.hi, pr.intervals, 3, pr.lam)
    assert np.max(np.abs(u[ks] - ref)) <= tol * np.max(np.abs(u))


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _scale_golden(pr):
    """The oracle's solution of the scale workload (tier-2 MG-PCG to rel.res
    1e-15, written by tests/golden/make_scale_alpha.py) and its record; the
    inputs must be bit-identical to the ones it was computed from."""
    rec = json.load(open(os.path.join(GOLDEN, "scale_alpha.json")))
    sha = lambda a: hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
    assert rec["x_sha256"] == sha(pr.x) and rec["y_sha256"] == sha(pr.y), "scale inputs differ from the golden's"
    return np.load(os.path.join(GOLDEN, "scale_alpha.npy")), rec


def test_scale_fp64_coefficients_match_oracle(scale):
    """The FP64 solve of the full scale workload (P = 3, 64^3 intervals, K =
    300,763, 10^6 clustered points) at tol 1e-13 equals the oracle's converged
    coefficients to 1e-8 relative (max norm); at the benchmark tolerance 1e-8
    the remaining iteration error is reported."""
    pr, plan = scale
    ref, rec = _scale_golden(pr)
    coef = torch.zeros(plan.K, dtype=torch.float64, device="cuda")
    _, res = plan.solve(1e-13, coef)
    err = rel_err(coef.cpu().numpy(), ref)
    _, res8 = plan.solve(pr.tol, coef)
    err8 = rel_err(coef.cpu().numpy(), ref)
    print("scale FP64: tol 1e-13: %d iterations, max rel. coefficient error %.2e; tol 1e-8: %d iterations, %.2e "
          "(oracle: %d iterations to 1e-8)" % (res.iterations, err, res8.iterations, err8, rec["iterations_to_1e-8"]))
    assert res.status == B.SPS_OK and err < 1e-8
    assert err8 < 1e-3


def test_scale_mixed_coefficients_match_oracle(scale):
    """Mixed precision (FP32 V-cycle and operator in the FP64 flexible PCG) on
    the full scale workload: at tol 1e-12 within 1e-7 of the oracle's
    coefficients; the error at the benchmark tolerance is reported."""
    pr, plan = scale
    ref, _ = _scale_golden(pr)
    with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED) as pm:
        pm.set_points(_device(pr.x), _device(pr.y))
        c = torch.zeros(plan.K, dtype=torch.float64, device="cuda")
        _, res = pm.solve(1e-12, c)
        err = rel_err(c.cpu().numpy(), ref)
        _, res8 = pm.solve(pr.tol, c)
        err8 = rel_err(c.cpu().numpy(), ref)
    print("scale mixed: tol 1e-12: %d iterations, max rel. coefficient error %.2e; tol 1e-8: %d iterations, %.2e"
          % (res.iterations, err, res8.iterations, err8))
    assert res.status == B.SPS_OK and err < 1e-7
    assert err8 < 1e-3


def test_scale_solve_residual_by_oracle(scale):
    """FP64 MGCG to rel.res 1e-8; the oracle recomputes the residual matrix free."""
    pr, plan = scale
    coef = torch.zeros(plan.K, dtype=torch.float64, device="cuda")
    _, res = plan.solve(pr.tol, coef)
    assert res.status == B.SPS_OK and res.rel_res_true <= pr.tol
    alpha = coef.cpu().numpy()
    rr = sampled.residual_norm(pr.x, pr.y, alpha, pr.lo, pr.hi, pr.intervals, 3, pr.lam, chunk=50000)
    assert rr <= 1.05 * pr.tol


def test_scale_mixed_solve_matches_fp64(scale):
    pr, plan = scale
    c64 = torch.zeros(plan.K, dtype=torch.float64, device="cuda")
    plan.solve(pr.tol, c64)
    with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED) as pm:
        pm.set_points(_device(pr.x), _device(pr.y))
        c32 = torch.zeros(plan.K, dtype=torch.float64, device="cuda")
        _, res = pm.solve(pr.tol, c32)
    assert res.status == B.SPS_OK and res.rel_res_true <= pr.tol
    rr = sampled.residual_norm(pr.x, pr.y, c32.cpu().numpy(), pr.lo, pr.hi, pr.intervals, 3, pr.lam, chunk=50000)
    assert rr <= 1.05 * pr.tol


def test_scale_null_space_recovery():
    """Affine responses on the clustered points: alpha = affine Greville tensor."""
    pr = W.scale()
    c = np.array([0.5, 1.0, -2.0, 0.25])
    y = c[0] + pr.x @ c[1:]
    with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi) as pl:
        pl.set_points(_device(pr.x), _device(y))
        coef = torch.zeros(pl.K, dtype=torch.float64, device="cuda")
        pl.solve(1e-11, coef)
    grids = np.meshgrid(*[spline.greville(pr.lo[p], pr.hi[p], pr.intervals[p], 3) for p in range(3)],
                        indexing="ij")
    ref = c[0] + sum(c[p + 1] * grids[p] for p in range(3))
    # coefficients far from the clusters are fixed only by the tiny penalty,
    # so the iterate's error is kappa * tol there
    assert rel_err(coef.cpu().numpy(), ref.ravel()) < 1e-4


def test_mixed_config_apply_sampled_and_solve():
    """P = 4, 32^4 intervals, n = 4e6 FP32 points: FP32 and FP64 operators on
    sampled coefficients, then the mixed solve to rel.res 1e-10."""
    pr = W.mixed()
    with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED) as pl:
        pl.set_points(_device(pr.x), _device(pr.y))
        v = np.random.default_rng(5).standard_normal(pl.K)
        ks = np.random.default_rng(6).choice(pl.K, 24, replace=False)
        ref = sampled.apply_rows(pr.x, v, ks, pr.lo, pr.hi, pr.intervals, 3, pr.lam)
        for prec, tol in ((0, 1e-12), (1, 2e-5)):
            u = np.zeros_like(v)
            B.sps_apply(pl.h, pr.levels, prec, v, u)
            assert np.max(np.abs(u[ks] - ref)) <= tol * np.max(np.abs(u))
        coef = torch.zeros(pl.K, dtype=torch.float64, device="cuda")
        _, res = pl.solve(pr.tol, coef)
        assert res.status == B.SPS_OK and res.rel_res_true <= pr.tol
