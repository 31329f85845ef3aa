"""Host logic of the serving loop that needs no GPU: the memory estimate that
drives admission by budget."""
import pytest

S = pytest.importorskip("paper_1901_00654_gb300.serving")


def test_estimate_bytes_closed_form():
    # P = 2, N = 16, 3 levels: K = 19^2 + 11^2 + 7^2 = 531; coarsest 7^2 = 49; the middle
    # level (11^2 coefficients) may be assembled with 7^2 stencil entries per coefficient
    P, n = 2, 1000
    base = n * (P * 8 + P * 4 + 8 + 16 + 8 + 12 * 3) + 531 * 8 * 30 + 49 * 49 * 32 + (64 << 20)
    assert S.estimate_bytes(P, [16, 16], 3, n) == base + 49 * 121 * 12
    # FP64 plans: FP64 stencils and the precomputed basis values of levels 2 and 3
    assert S.estimate_bytes(P, [16, 16], 3, n, precision=0) == base + 49 * 121 * 8 + 2 * n * 8 * 8


def test_estimate_bytes_grows_with_the_problem():
    base = S.estimate_bytes(3, [32] * 3, 4, 100_000)
    assert S.estimate_bytes(3, [32] * 3, 4, 200_000) > base          # more points
    assert S.estimate_bytes(3, [64] * 3, 5, 100_000) > base          # finer grid
    assert S.estimate_bytes(3, [32] * 3, 4, 100_000, itemsize=4) < base   # FP32 coordinates
    # the P = 5 serving grid (16^5 intervals, 2e6 points) stays far below the 120 GB budget
    assert S.estimate_bytes(5, [16] * 5, 4, 2_000_000) < 120e9 / 8


class _Recorder:
    """Fake executor: holds each request for a fixed time and records what
    the scheduler had in flight (requests and their estimated bytes)."""

    def __init__(self, hold_s, precision):
        import threading
        self.hold_s, self.precision = hold_s, precision
        self.lock = threading.Lock()
        self.active = {}
        self.order = []
        self.max_active = 0
        self.max_bytes = 0
        self.started = {}

    def __call__(self, problem, stream):
        import time
        est = S.estimate_bytes(problem.P, problem.intervals, problem.levels, problem.n,
                               problem.x.dtype.itemsize, self.precision)
        with self.lock:
            self.active[id(problem)] = est
            self.order.append(problem.name)
            self.started[problem.name] = time.perf_counter()
            self.max_active = max(self.max_active, len(self.active))
            self.max_bytes = max(self.max_bytes, sum(self.active.values()))
        time.sleep(self.hold_s)
        with self.lock:
            del self.active[id(problem)]
        return None, S.B.sps_result(), S.B.SPS_OK


def _trace(sizes, gap_s):
    import numpy as np
    import workloads as W
    reqs = []
    for i, n in enumerate(sizes):
        pr = W.Problem("r%d" % i, 3, 3, [32, 32, 32], 4, 1e-3, 1e-8, np.zeros((n, 3)), np.zeros(n),
                       [0.0] * 3, [1.0] * 3)
        reqs.append(W.Request(i * gap_s, pr))
    return reqs


def test_scheduler_respects_slots_budget_and_arrival_order():
    """Continuous batching without a GPU: requests are admitted in arrival
    order as slots and budget free up, never more than `slots` at once and
    never more estimated bytes than the budget (a request alone may exceed
    it), and every request completes with its latency measured from arrival."""
    sizes = [200_000, 50_000, 400_000, 100_000, 300_000, 50_000, 250_000, 120_000, 80_000, 60_000]
    est = [S.estimate_bytes(3, [32] * 3, 4, n, 8, S.B.SPS_PREC_MIXED) for n in sizes]
    budget = int(2.5 * max(est))
    rec = _Recorder(0.05, S.B.SPS_PREC_MIXED)
    srv = S.Server(slots=3, budget_bytes=budget, executor=rec, stream_factory=object)
    stats = srv.run(_trace(sizes, 0.005))
    assert len(stats.completed) == len(sizes)
    assert [c.index for c in stats.completed] == list(range(len(sizes)))
    assert rec.order == ["r%d" % i for i in range(len(sizes))]          # FIFO admission
    assert rec.max_active <= 3 and stats.max_in_flight <= 3
    assert rec.max_bytes <= budget and stats.peak_bytes <= budget
    assert rec.max_active >= 2                                         # requests overlap
    for c in stats.completed:
        assert c.t_done - c.t_arrival >= 0.05 * 0.9 and c.t_admit >= c.t_arrival - 1e-3
    summ = stats.summary()
    assert summ["requests"] == len(sizes) and summ["converged"] == len(sizes)
    assert summ["p99_ms"] >= summ["p50_ms"] >= 45.0


def test_scheduler_admits_an_oversized_request_alone():
    """A request larger than the whole budget still runs, alone."""
    sizes = [100_000, 2_000_000, 100_000]
    est = [S.estimate_bytes(3, [32] * 3, 4, n, 8, S.B.SPS_PREC_MIXED) for n in sizes]
    budget = int(1.5 * est[0])
    assert est[1] > budget
    rec = _Recorder(0.03, S.B.SPS_PREC_MIXED)
    srv = S.Server(slots=4, budget_bytes=budget, executor=rec, stream_factory=object)
    stats = srv.run(_trace(sizes, 0.0))
    assert len(stats.completed) == 3 and rec.max_active == 1


def test_executor_and_streams_go_together():
    with pytest.raises(ValueError):
        S.Server(executor=lambda p, s: None)


def test_a_failing_request_releases_its_slot():
    """A request whose execution raises is reported (SPS_EINTERNAL) and frees
    its slot and budget, so the requests behind it still run."""
    calls = []

    def flaky(problem, stream):
        calls.append(problem.name)
        if problem.name == "r1":
            raise RuntimeError("injected host-side failure")
        return None, S.B.sps_result(), S.B.SPS_OK

    srv = S.Server(slots=1, budget_bytes=1e12, executor=flaky, stream_factory=object)
    stats = srv.run(_trace([1000, 1000, 1000], 0.0))
    assert [c.status for c in stats.completed] == [S.B.SPS_OK, S.B.SPS_EINTERNAL, S.B.SPS_OK]
    assert calls == ["r0", "r1", "r2"]
