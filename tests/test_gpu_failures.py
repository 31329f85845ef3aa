"""Failure paths of the C ABI that need a plan on a device: every failure is
made on the host (bad data, a tiny iteration cap, a memory limit, a singular
system) and comes back as a status code; nothing here faults or hangs a GPU.
"""
import math

import numpy as np
import pytest

from tests.gpu_util import random_problem

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1901_00654_gb300.binding")


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_non_finite_response_is_rejected(bad, dtype):
    x, y, lo, hi = random_problem(2, [8, 8], 500, seed=1, dtype=dtype)
    y[123] = bad
    with B.Plan(2, [8, 8], 2, 1e-3) as pl:
        with pytest.raises(B.SpsError) as e:
            pl.set_points(x, y)
        assert e.value.code == B.SPS_EDOM
        with pytest.raises(B.SpsError) as e:       # no points were accepted
            pl.solve(1e-8)
        assert e.value.code == B.SPS_ESTATE
        y[123] = 0.5                                # the plan stays usable
        pl.set_points(x, y)
        _, res = pl.solve(1e-8)
        assert res.status == B.SPS_OK


def test_iteration_cap_reports_no_convergence_with_result():
    x, y, lo, hi = random_problem(3, [16, 16, 16], 20000, seed=2)
    for prec in (B.SPS_PREC_FP64, B.SPS_PREC_MIXED):
        with B.Plan(3, [16, 16, 16], 4, 1e-4, precision=prec, max_iter=2) as pl:
            pl.set_points(x, y)
            coef, res = pl.solve(1e-12, check=False)
            assert res.status == B.SPS_ENOCONV
            assert res.iterations == 2
            assert math.isfinite(res.rel_res_true) and 1e-12 < res.rel_res_true < 1.0
            assert math.isfinite(res.rel_res)
            assert np.all(np.isfinite(coef)) and np.any(coef != 0.0)   # the last iterate is returned
            with pytest.raises(B.SpsError) as e:
                pl.solve(1e-12)
            assert e.value.code == B.SPS_ENOCONV


def test_device_memory_limit():
    """sps_options.max_device_bytes: allocations beyond the limit fail with
    SPS_ENOMEM before cudaMalloc, at plan creation or at set_points, and the
    plan reports the bytes it holds."""
    x, y, lo, hi = random_problem(3, [16, 16, 16], 20000, seed=3)
    with pytest.raises(B.SpsError) as e:
        B.Plan(3, [16, 16, 16], 4, 1e-3, max_device_bytes=1 << 16)
    assert e.value.code == B.SPS_ENOMEM
    with B.Plan(3, [16, 16, 16], 4, 1e-3) as free:
        created = B.sps_plan_device_bytes(free.h)
        free.set_points(x, y)
        loaded = B.sps_plan_device_bytes(free.h)
        assert 0 < created < loaded
    # room for the plan but not for the points
    with B.Plan(3, [16, 16, 16], 4, 1e-3, max_device_bytes=created + 4096) as pl:
        assert B.sps_plan_device_bytes(pl.h) == created
        with pytest.raises(B.SpsError) as e:
            pl.set_points(x, y)
        assert e.value.code == B.SPS_ENOMEM
        assert B.sps_plan_device_bytes(pl.h) <= created + 4096
    with B.Plan(3, [16, 16, 16], 4, 1e-3, max_device_bytes=loaded + (64 << 20)) as pl:
        pl.set_points(x, y)
        _, res = pl.solve(1e-8)
        assert res.status == B.SPS_OK


@pytest.mark.parametrize("prec", [B.SPS_PREC_FP64, B.SPS_PREC_MIXED])
def test_singular_system_reports_breakdown(prec):
    """lambda = 0 with every point in one corner cell: the basis functions
    without data have a zero diagonal, the damped Jacobi step divides by it,
    and the CG scalars stop being finite -- a breakdown, reported as such.  The
    mixed solve first retries with the FP64 outer operator (its answer to an
    FP32 breakdown), breaks down again and reports it."""
    r = np.random.default_rng(4)
    x = 0.1 * r.random((400, 2))                   # all in the first of 8 x 8 cells
    y = r.standard_normal(400)
    with B.Plan(2, [8, 8], 2, 0.0, omega=0.5, precision=prec) as pl:
        pl.set_points(x, y)
        coef, res = pl.solve(1e-8, check=False)
        assert res.status == B.SPS_EBREAKDOWN
        with pytest.raises(B.SpsError) as e:
            pl.solve(1e-8)
        assert e.value.code == B.SPS_EBREAKDOWN


def test_invalid_new_options_are_rejected():
    for kw in (dict(coarse_cg=2), dict(coarse_iters=0), dict(max_device_bytes=-1), dict(replace_ratio=1.5)):
        with pytest.raises(B.SpsError) as e:
            B.Plan(2, [8, 8], 2, 1e-3, **kw)
        assert e.value.code == B.SPS_EINVAL
