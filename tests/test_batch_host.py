"""Host logic of the batched solver's autotuner, on the CPU: the makespan
model of its persistent queues (sps_simulate_batch) against closed forms and
an event simulation written here from the queue rules."""
import heapq

import numpy as np
import pytest

from paper_1901_00654_gb300 import build


@pytest.fixture(scope="module")
def B():
    build.build_library()
    from paper_1901_00654_gb300 import binding
    return binding


def queues(order, t1, tc, C, big, grid):
    """grid CTAs as grid // C teams take the first `big` problems of `order`
    (times tc); a team that finds that queue empty becomes C single CTAs, which
    take the rest in order (times t1).  Events are (time free, team size):
    at equal times single CTAs are served before teams."""
    teams = grid // C if C > 1 else grid
    ev = [(0.0, C if C > 1 else 1) for _ in range(teams)]
    heapq.heapify(ev)
    nb, nx = 0, (big if C > 1 else 0)
    end = 0.0
    while ev:
        t, size = heapq.heappop(ev)
        if size > 1:
            if nb < big:
                f = t + tc[order[nb]]
                nb += 1
                end = max(end, f)
                heapq.heappush(ev, (f, size))
            else:
                for _ in range(size):
                    heapq.heappush(ev, (t, 1))
        elif nx < len(order):
            f = t + t1[order[nx]]
            nx += 1
            end = max(end, f)
            heapq.heappush(ev, (f, 1))
    return end


def test_closed_forms(B):
    t1 = np.array([5.0, 3.0, 2.0, 1.0])
    tc = t1 / 1.5
    order = [0, 1, 2, 3]
    # enough single CTAs: the longest problem
    assert B.sps_simulate_batch(order, t1, tc, 1, 0, 8) == pytest.approx(5.0)
    # one CTA: the sum
    assert B.sps_simulate_batch(order, t1, tc, 1, 0, 1) == pytest.approx(11.0)
    # one team of two takes every problem in turn
    assert B.sps_simulate_batch(order, t1, tc, 2, 4, 2) == pytest.approx(11.0 / 1.5)
    # no problem for the teams: they split at once, two CTAs in cost order (5 | 3 + 2 + 1)
    assert B.sps_simulate_batch(order, t1, tc, 2, 0, 2) == pytest.approx(6.0)
    # the team takes the costliest, then splits: 5/1.5 | then 3, 2, 1 on two CTAs
    assert B.sps_simulate_batch(order, t1, tc, 2, 1, 2) == pytest.approx(5.0 / 1.5 + 3.0)


@pytest.mark.parametrize("C", [1, 2, 4, 8])
def test_matches_an_event_simulation(B, C):
    rng = np.random.default_rng(C)
    for trial in range(20):
        n = int(rng.integers(1, 300))
        t1 = rng.lognormal(0.0, 1.5, n)
        tc = t1 * rng.uniform(0.2, 1.0, n)
        order = np.argsort(-t1, kind="stable")
        grid = C * int(rng.integers(1, 40))
        big = int(rng.integers(0, n + 1)) if C > 1 else 0
        got = B.sps_simulate_batch(order, t1, tc, C, big, grid)
        assert got == pytest.approx(queues(order, t1, tc, C, big, grid), rel=1e-12)
        # never below the longest single task nor the total work spread over all CTAs
        lower = max(np.max(tc[order[:big]]) if big else 0.0, np.max(t1[order[big:]]) if big < n else 0.0)
        assert got >= lower * (1 - 1e-12)
        assert got >= (np.sum(t1[order[big:]]) + C * np.sum(tc[order[:big]])) / grid * (1 - 1e-12)


def test_rejects_bad_arguments(B):
    t = np.ones(3)
    for order, C, big, grid in (([0, 1, 1], 1, 0, 4), ([0, 1, 3], 1, 0, 4), ([0, 1, 2], 3, 0, 6),
                                ([0, 1, 2], 4, 0, 2), ([0, 1, 2], 2, 4, 4)):
        with pytest.raises(B.SpsError):
            B.sps_simulate_batch(order, t, t, C, big, grid)
    with pytest.raises(B.SpsError):
        B.sps_simulate_batch([0, 1, 2], np.array([1.0, -1.0, 1.0]), t, 1, 0, 4)
