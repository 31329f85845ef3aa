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
