"""The batched persistent-kernel solve against per-problem solves and the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import spline
from tests.gpu_util import rel_err

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1901_00654_gb300.binding")


def _problems(count, seed=3, n_hi=2e4):
    return W.batched(seed=seed, count=count, n_lo=1e3, n_hi=n_hi)


@pytest.fixture(params=[1, 2, 4, 8])
def cluster(request):
    """Thread-block cluster size of the batched kernel's launch shape."""
    return request.param


def test_batch_matches_oracle_residual_and_single_solves(cluster):
    probs = _problems(24)
    tol = 1e-8
    plans = []
    try:
        for pr in probs:
            pl = B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED)
            pl.set_points(pr.x, pr.y)
            plans.append(pl)
        coefs = [np.zeros(pl.K) for pl in plans]
        res, used = B.sps_solve_batch_shape([pl.h for pl in plans], coefs, tol, cluster=cluster)
        assert used[0] == cluster
        for pr, pl, c, r in zip(probs, plans, coefs, res):
            assert r.status == B.SPS_OK and r.rel_res_true <= tol
            A, b, _, _ = spline.system(pr.x, pr.y, pr.lo, pr.hi, pr.intervals, 3, pr.lam)
            assert np.linalg.norm(b - A @ c) / np.linalg.norm(b) <= 1.05 * tol
            single, rs = pl.solve(tol)
            # same algorithm and arithmetic, one CTA instead of many kernels
            assert abs(r.iterations - rs.iterations) <= max(3, 0.1 * rs.iterations)
            assert rel_err(c, single) < 1e-4
    finally:
        for pl in plans:
            pl.close()


def test_batch_single_problem(cluster):
    # one problem: with clusters it is solved by a whole cluster, the other CTAs find the queue empty
    pr = _problems(1, seed=5)[0]
    with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED) as pl:
        pl.set_points(pr.x, pr.y)
        c = np.zeros(pl.K)
        (r,), _ = B.sps_solve_batch_shape([pl.h], [c], 1e-8, cluster=cluster)
        assert r.status == B.SPS_OK and r.rel_res_true <= 1e-8
        A, b, _, _ = spline.system(pr.x, pr.y, pr.lo, pr.hi, pr.intervals, 3, pr.lam)
        assert np.linalg.norm(b - A @ c) / np.linalg.norm(b) <= 1.05e-8


def test_batch_twice_agrees_with_device_buffers():
    torch = pytest.importorskip("torch")
    probs = _problems(8, seed=11)
    plans = []
    try:
        for pr in probs:
            pl = B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED)
            pl.set_points(pr.x, pr.y)
            plans.append(pl)
        c1 = [torch.zeros(pl.K, dtype=torch.float64, device="cuda") for pl in plans]
        c2 = [torch.zeros(pl.K, dtype=torch.float64, device="cuda") for pl in plans]
        tol = 1e-8
        B.sps_solve_batch([pl.h for pl in plans], c1, tol)
        B.sps_solve_batch([pl.h for pl in plans], c2, tol)
        # atomics make the summation order differ from run to run, so the two
        # runs stop at different iterates; both have relative residual <= tol,
        # hence ||A (c1 - c2)|| <= 2 tol ||b|| whatever the conditioning
        for pr, a, b in zip(probs, c1, c2):
            A, rhs, _, _ = spline.system(pr.x, pr.y, pr.lo, pr.hi, pr.intervals, 3, pr.lam)
            d = a.cpu().numpy() - b.cpu().numpy()
            assert np.linalg.norm(A @ d) <= 2.05 * tol * np.linalg.norm(rhs)
            assert rel_err(a.cpu().numpy(), b.cpu().numpy()) < 1e-4
    finally:
        for pl in plans:
            pl.close()


def test_batch_rejects_p4():
    x = np.random.default_rng(0).random((500, 4))
    with B.Plan(4, [4] * 4, 2, 1e-2) as pl:
        pl.set_points(x, np.sin(x[:, 0]))
        with pytest.raises(B.SpsError) as e:
            B.sps_solve_batch([pl.h], [np.zeros(pl.K)], 1e-8)
        assert e.value.code == B.SPS_EINVAL


def test_batch_autotuner_picks_a_measured_shape():
    """sps_tune_batch measures every cluster size and picks the shape with the
    shortest simulated batch time; later sps_solve_batch calls on the same
    problems use it, converge, and take no longer than the simulation said
    (within launch and timing noise)."""
    import time
    probs = _problems(48, seed=13, n_hi=5e4)
    tol = 1e-8
    plans = []
    try:
        for pr in probs:
            pl = B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED)
            pl.set_points(pr.x, pr.y)
            plans.append(pl)
        hs = [pl.h for pl in plans]
        coefs = [np.zeros(pl.K) for pl in plans]
        cluster, big, predicted = B.sps_tune_batch(hs, coefs, tol)
        assert cluster in (1, 2, 4, 8) and 0 <= big <= len(probs) and predicted > 0
        t0 = time.perf_counter()
        res = B.sps_solve_batch(hs, coefs, tol)
        wall = (time.perf_counter() - t0) * 1e3
        assert all(r.status == B.SPS_OK and r.rel_res_true <= tol for r in res)
        _, used = B.sps_solve_batch_shape(hs, coefs, tol)          # no shape given: the tuned one
        assert used == (cluster, big if cluster > 1 else 0)
        print("batch autotuner: cluster %d, %d problems on clusters, simulated %.1f ms, measured %.1f ms"
              % (cluster, big, predicted, wall))
        assert wall < 3.0 * predicted + 50.0
    finally:
        for pl in plans:
            pl.close()
