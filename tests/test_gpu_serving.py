"""The continuous-batching server: admission by memory budget, overlap of
requests, and every result equal (within the solve tolerance) alone and in
the mix."""
import numpy as np
import pytest

import workloads as W
from oracle import mgcg, spline
from tests.gpu_util import rel_err

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1901_00654_gb300.binding")
S = pytest.importorskip("paper_1901_00654_gb300.serving")

TOL = 1e-8


def _trace(count=10):
    return W.serving_trace(seed=21, count=count, rate=100.0, n_lo=2e3, n_hi=2e4, P_choices=(2, 3))


def test_mix_equals_alone():
    trace = _trace()
    srv = S.Server(slots=4, tol=TOL)
    try:
        stats = srv.run(trace)
    finally:
        srv.close()
    assert len(stats.completed) == len(trace)
    assert stats.max_in_flight >= 2          # requests really overlapped
    errs = []
    for c, req in zip(stats.completed, trace):
        pr = req.problem
        assert c.status == B.SPS_OK and c.result.rel_res_true <= TOL
        # the served (mixed-precision) result against the oracle's direct solve
        A, b, _, _ = spline.system(pr.x, pr.y, pr.lo, pr.hi, pr.intervals, 3, pr.lam)
        ref = mgcg.solve_direct(A, b)
        assert np.linalg.norm(b - A @ c.coef) <= 1.05 * TOL * np.linalg.norm(b)
        errs.append(rel_err(c.coef, ref))
        with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED) as pl:
            pl.set_points(pr.x, pr.y)
            alone, r = pl.solve(TOL)
        # both iterates satisfy |r| <= tol |b|, so ||A (c_mix - c_alone)|| <= 2 tol ||b||
        A, b, _, _ = spline.system(pr.x, pr.y, pr.lo, pr.hi, pr.intervals, 3, pr.lam)
        assert np.linalg.norm(A @ (c.coef - alone)) <= 2.05 * TOL * np.linalg.norm(b)
        assert rel_err(c.coef, alone) < 1e-4
    print("served results vs the oracle's direct solve (tol %g): max rel. coefficient error %.2e, median %.2e"
          % (TOL, max(errs), float(np.median(errs))))


def test_admission_estimate_covers_the_plan():
    """The admission estimate of a request is at least the device memory its
    plan actually holds after set_points (sps_plan_device_bytes)."""
    trace = W.serving_trace(seed=22, count=6, n_lo=1e4, n_hi=2e5, P_choices=(2, 3, 4))
    for req in trace:
        pr = req.problem
        est = S.estimate_bytes(pr.P, pr.intervals, pr.levels, pr.n, pr.x.dtype.itemsize)
        with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED) as pl:
            pl.set_points(pr.x, pr.y)
            used = B.sps_plan_device_bytes(pl.h)
        assert used <= est, (pr.P, pr.intervals, pr.n, used, est)


def test_budget_serialises_admission():
    """A budget smaller than any request admits one at a time (a request is
    always admitted when nothing else is in flight, so none waits forever)."""
    trace = _trace(4)
    srv = S.Server(slots=4, budget_bytes=1, tol=TOL)
    try:
        stats = srv.run(trace, time_scale=0.0)
    finally:
        srv.close()
    assert stats.max_in_flight == 1
    assert all(c.status == B.SPS_OK for c in stats.completed)
