"""sps_evaluate (Algorithm 4 at query points) against the oracle's explicit
Phi, and the closed form of a fitted spline on data from the penalty's null
space."""
import numpy as np
import pytest

from oracle import spline
from tests.gpu_util import random_problem, rel_err

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1901_00654_gb300.binding")

SHAPES = [(1, [64]), (2, [16, 32]), (3, [8, 16, 8]), (4, [4, 8, 4, 4]), (5, [2, 2, 4, 2, 2])]


def _queries(P, intervals, lo, hi, m, seed, dtype):
    r = np.random.default_rng(seed)
    x = lo + (np.asarray(hi) - lo) * r.random((m, P))
    x[0] = lo                                     # corners
    x[1] = hi
    for p in range(P):                            # every interior knot of dimension p
        k = np.arange(1, intervals[p])
        x[2:2 + len(k), p] = lo[p] + (hi[p] - lo[p]) * k / intervals[p]
    return np.ascontiguousarray(x.astype(dtype))


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "P%d" % s[0])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_evaluate_matches_oracle_phi(shape, dtype):
    P, intervals = shape
    lo, hi = [-0.5] * P, [1.5] * P
    K = int(np.prod([N + 3 for N in intervals]))
    coef = np.random.default_rng(P).standard_normal(K)
    xq = _queries(P, intervals, np.array(lo), np.array(hi), 3001, 10 + P, dtype)
    ref = spline.phi_matrix(xq.astype(np.float64), lo, hi, intervals, 3) @ coef
    with B.Plan(P, intervals, 2, 1e-3, lo, hi) as pl:     # no points needed
        got = pl.evaluate(coef, xq)
    assert rel_err(got, ref) < 1e-12


def test_evaluate_device_buffers_and_empty():
    torch = pytest.importorskip("torch")
    P, intervals = 3, [8, 16, 8]
    lo, hi = [0.0] * 3, [1.0] * 3
    K = int(np.prod([N + 3 for N in intervals]))
    coef = np.random.default_rng(1).standard_normal(K)
    xq = _queries(P, intervals, np.array(lo), np.array(hi), 777, 3, np.float64)
    ref = spline.phi_matrix(xq, lo, hi, intervals, 3) @ coef
    with B.Plan(P, intervals, 2, 1e-3, lo, hi) as pl:
        out = torch.zeros(777, dtype=torch.float64, device="cuda")
        B.sps_evaluate(pl.h, torch.from_numpy(coef).cuda(), torch.from_numpy(xq).cuda(), out)
        assert rel_err(out.cpu().numpy(), ref) < 1e-12
        B.sps_evaluate(pl.h, coef, np.zeros((0, P)), np.zeros(0))          # m = 0: nothing to do


def test_evaluate_rejects_points_outside_but_fills_the_rest():
    P, intervals = 2, [16, 16]
    with B.Plan(P, intervals, 2, 1e-3) as pl:
        coef = np.random.default_rng(2).standard_normal(pl.K)
        xq = np.array([[0.25, 0.5], [1.5, 0.5], [0.75, np.nan], [1.0, 0.0]])
        out = np.zeros(4)
        with pytest.raises(B.SpsError) as e:
            B.sps_evaluate(pl.h, coef, xq, out)
        assert e.value.code == B.SPS_EDOM
        ref = spline.phi_matrix(xq[[0, 3]], [0.0] * 2, [1.0] * 2, intervals, 3) @ coef
        assert np.all(np.isnan(out[[1, 2]]))
        assert rel_err(out[[0, 3]], ref) < 1e-12


@pytest.mark.parametrize("P,intervals,G", [(2, [32, 32], 4), (3, [16, 16, 16], 3)])
def test_fitted_spline_reproduces_affine_data(P, intervals, G):
    """y affine in x lies in the penalty's null space and is fitted exactly, so
    the fitted spline equals that affine function everywhere on the domain
    (Marsden's identity): a closed form at any query point."""
    x, _, lo, hi = random_problem(P, intervals, 20000, seed=40 + P)
    c = np.arange(1, P + 2) / 7.0
    y = c[0] + x @ c[1:]
    with B.Plan(P, intervals, G, 1e-2, lo, hi) as pl:
        pl.set_points(x, y)
        coef, res = pl.solve(1e-13)
        xq = _queries(P, intervals, np.array(lo), np.array(hi), 5000, 99, np.float64)
        got = pl.evaluate(coef, xq)
    want = c[0] + xq @ c[1:]
    assert np.max(np.abs(got - want)) < 1e-8 * np.max(np.abs(want))
