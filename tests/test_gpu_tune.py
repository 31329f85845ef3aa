"""Launch-shape choices of the point operator: every tile side and lane layout
computes the same operator as the oracle, and the autotuner's choice is one
of its candidates and leaves the solve's result unchanged."""
import numpy as np
import pytest

from oracle import spline
from tests.gpu_util import random_problem, rel_err

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1901_00654_gb300.binding")

FP64_TOL = 1e-12
FP32_TOL = 2e-5
TS_DEFAULT = {3: 8, 4: 4}

# (P, intervals, levels, n): several tiles per level and ragged item tails
SHAPES = [(3, [8, 16, 8], 3, 6007), (4, [4, 8, 4, 4], 2, 4001)]


def _phi_all(x, lo, hi, intervals, G):
    return {g: spline.phi_matrix(x, lo, hi, spline.level_intervals(intervals, G, g), 3) for g in range(1, G + 1)}


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "P%d" % s[0])
@pytest.mark.parametrize("lanes_r", [2, 3])
@pytest.mark.parametrize("tile_scale", [0.5, 1, 2])
@pytest.mark.parametrize("prec", [B.SPS_PREC_FP64, B.SPS_PREC_MIXED], ids=["fp64", "mixed"])
def test_lane_layouts_and_tiles_match_oracle(shape, lanes_r, tile_scale, prec):
    # FP64 plans apply matrix-free levels >= 2 from precomputed basis values (both layouts);
    # level 1 and the FP32 kernels evaluate the basis from the coordinates
    P, intervals, G, n = shape
    x, y, lo, hi = random_problem(P, intervals, n, seed=300 + P)
    tile = int(TS_DEFAULT[P] * tile_scale)
    phis = _phi_all(x, lo, hi, intervals, G)
    r = np.random.default_rng(5)
    tol = FP64_TOL if prec == B.SPS_PREC_FP64 else FP32_TOL
    with B.Plan(P, intervals, G, 1e-3, lo, hi, precision=prec, lanes_r=lanes_r, tile=tile, hybrid=0) as pl:
        pl.set_points(x, y)
        for g in range(1, G + 1):
            ts, lr = B.sps_get_tuning(pl.h, g)
            assert (ts, lr) == (tile, lanes_r)
            Phi = phis[g]
            v = r.standard_normal(Phi.shape[1])
            u = np.zeros_like(v)
            B.sps_point_apply(pl.h, g, prec, v, u)
            assert rel_err(u, Phi.T @ (Phi @ v)) < tol, (g, rel_err(u, Phi.T @ (Phi @ v)))


@pytest.mark.parametrize("prec", [B.SPS_PREC_FP64, B.SPS_PREC_MIXED])
def test_autotune_choice_and_solve(prec):
    P, intervals, G, n = 3, [16, 16, 16], 3, 40000
    x, y, lo, hi = random_problem(P, intervals, n, seed=77)
    lam, tol = 1e-3, 1e-10
    A, b, _, _ = spline.system(x, y, lo, hi, intervals, 3, lam)
    phis = _phi_all(x, lo, hi, intervals, G)
    coefs = []
    for autotune in (0, 1):
        with B.Plan(P, intervals, G, lam, lo, hi, precision=prec, autotune=autotune, hybrid=0) as pl:
            pl.set_points(x, y)
            for g in range(2, G + 1):
                ts, lr = B.sps_get_tuning(pl.h, g)
                assert ts in (4, 8, 16)
                assert lr in ((2, 3) if autotune else (0,))
                Phi = phis[g]
                v = np.random.default_rng(g).standard_normal(Phi.shape[1])
                u = np.zeros_like(v)
                B.sps_point_apply(pl.h, g, prec, v, u)
                ref = Phi.T @ (Phi @ v)
                assert rel_err(u, ref) < (FP64_TOL if prec == B.SPS_PREC_FP64 else FP32_TOL)
            c, res = pl.solve(tol)
            assert res.status == B.SPS_OK
            assert np.linalg.norm(b - A @ c) <= 1.05 * tol * np.linalg.norm(b)
            # a second set-up keeps the tuned shape
            shape1 = [B.sps_get_tuning(pl.h, g) for g in range(1, G + 1)]
            pl.set_points(x, y)
            assert [B.sps_get_tuning(pl.h, g) for g in range(1, G + 1)] == shape1
            coefs.append(c)
    # both satisfy |r| <= tol |b|
    assert np.linalg.norm(A @ (coefs[0] - coefs[1])) <= 2.1 * tol * np.linalg.norm(b)
