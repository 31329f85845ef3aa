"""P = 5 on a multi-level hierarchy whose coarsest grid has two intervals per
dimension ([4]^5 intervals, G = 2: K_1 = 3125, K_G = 16,807), and the inner
matrix-free CG coarse solver (Section 3.2, coarse grid solver), against the
oracle.

At P = 5 the damped-Jacobi V-cycle converges slowly (thousands of iterations
to 1e-12, in the oracle's MG-PCG as on the GPU): the solve test allows for
that, and a trajectory test checks that the GPU's residual history is the
oracle's.

The oracle's coarse matrix is the Galerkin product I' A_G I (Section 3.2,
grid transfer; pinned in tests/test_oracle_pins.py), equal to the
rediscretised A_1 up to rounding and far cheaper to form at P = 5.
"""
import numpy as np
import pytest

from oracle import mgcg, spline
from tests.gpu_util import random_problem, rel_err

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1901_00654_gb300.binding")

P5, N5, G5, LAM5, n5 = 5, [4] * 5, 2, 1.0, 20011


@pytest.fixture(scope="module")
def p5():
    x, y, lo, hi = random_problem(P5, N5, n5, seed=105)
    A, b, _, _ = spline.system(x, y, lo, hi, N5, 3, LAM5)
    I = spline.prolongation([2] * 5, 3)
    A1 = (I.T @ A @ I).toarray()
    ref = mgcg.solve_direct(A, b)
    return dict(x=x, y=y, lo=lo, hi=hi, A=A, b=b, A1=A1, ref=ref)


def test_p5_coarse_matrix_and_solve(p5):
    with B.Plan(P5, N5, G5, LAM5) as pl:
        pl.set_points(p5["x"], p5["y"])
        cnt = B.sps_level_matrix(pl.h, 1)
        assert cnt == 3125 * 3125
        A1 = np.zeros(cnt)
        B.sps_level_matrix(pl.h, 1, A1)
        A1 = A1.reshape(3125, 3125)
        assert np.max(np.abs(A1 - p5["A1"])) <= 1e-12 * np.max(np.abs(p5["A1"]))
        r = np.random.default_rng(8).standard_normal(3125)
        e = np.zeros_like(r)
        B.sps_coarse_solve(pl.h, r, e)
        Ao = p5["A1"]
        eta = np.max(np.abs(r - Ao @ e)) / (np.max(np.abs(Ao).sum(axis=1)) * np.max(np.abs(e)) + np.max(np.abs(r)))
        assert eta < 1e-13, eta


def test_p5_solve_matches_direct(p5):
    """The multi-level P = 5 FP64 solve at tol 1e-12 against the direct solve.
    The coefficient error of any iterate is bounded by kappa * rel.res; this
    system's effective kappa is about 1e6 (its Jacobi-scaled condition number
    is near 4e8, which also bounds the direct solve's own accuracy near 1e-8),
    so the bound here is 2e-6, and the A-norm error, which CG minimises, is
    checked at 1e-8."""
    with B.Plan(P5, N5, G5, LAM5, max_iter=80000) as pl:
        pl.set_points(p5["x"], p5["y"])
        coef, res = pl.solve(1e-12)
    assert res.status == B.SPS_OK and res.rel_res_true <= 1e-12
    A, b = p5["A"], p5["b"]
    assert np.linalg.norm(b - A @ coef) / np.linalg.norm(b) <= 2e-12
    err = rel_err(coef, p5["ref"])
    d = coef - p5["ref"]
    aerr = float(np.sqrt(d @ (A @ d)) / np.sqrt(p5["ref"] @ (A @ p5["ref"])))
    print("P=5 FP64: %d iterations, max rel. coefficient error %.2e, relative A-norm error %.2e"
          % (res.iterations, err, aerr))
    assert err < 2e-6 and aerr < 1e-8


def test_p5_trajectory_matches_oracle(p5):
    """The GPU's MG-PCG is the oracle's Algorithm 8 at P = 5: with the same
    damping, its residual after 50 and 200 iterations is the oracle's within
    rounding-driven drift (a factor 1.5)."""
    import scipy.linalg as sla
    A, b = p5["A"], p5["b"]
    I = spline.prolongation([2] * 5, 3)
    out = {}
    for m in (50, 200):
        with B.Plan(P5, N5, G5, LAM5, max_iter=m) as pl:
            pl.set_points(p5["x"], p5["y"])
            om = B.sps_get_omega(pl.h, G5)
            _, res = pl.solve(1e-14, check=False)
            out[m] = res.rel_res_true
    H = mgcg.Hierarchy()
    H.b = b
    A1 = (I.T @ A @ I).tocsr()
    for Ag, Ng, Ig, o in ((A1, [2] * 5, None, 1.0), (A, N5, I, om[1])):
        H.levels.append(mgcg.Level(Ng, Ag, 1.0 / Ag.diagonal(), o, Ig))
    H.coarse_factor = sla.cho_factor(p5["A1"])
    hist = mgcg.mgcg(H, 1e-14, max_iter=200).history
    print("P=5 residual after 50 / 200 iterations: GPU %.3e / %.3e, oracle %.3e / %.3e"
          % (out[50], out[200], hist[50], hist[200]))
    for m in (50, 200):
        assert hist[m] / 1.5 <= out[m] <= 1.5 * hist[m]


def test_p5_mixed_solve(p5):
    """Mixed precision at P = 5: FP32 V-cycle and operator inside the FP64
    flexible PCG, to tol 1e-9; error against the direct solve stated."""
    with B.Plan(P5, N5, G5, LAM5, precision=B.SPS_PREC_MIXED, max_iter=80000) as pl:
        pl.set_points(p5["x"], p5["y"])
        coef, res = pl.solve(1e-9)
    assert res.status == B.SPS_OK and res.rel_res_true <= 1e-9
    err = rel_err(coef, p5["ref"])
    A = p5["A"]
    d = coef - p5["ref"]
    aerr = float(np.sqrt(d @ (A @ d)) / np.sqrt(p5["ref"] @ (A @ p5["ref"])))
    print("P=5 mixed: %d iterations, max rel. coefficient error vs oracle %.2e, relative A-norm error %.2e"
          % (res.iterations, err, aerr))
    assert aerr < 1e-5 and err < 5e-3     # kappa_eff * tol, as for the FP64 solve


def test_mixed_with_an_indefinite_fp32_coarse_matrix():
    """P = 5 with lambda = 1e-2: the mixed plan assembles A_1 from FP32
    products, which at this conditioning (Jacobi-scaled condition number near
    5e10) is not positive definite; the factorisation is repeated with a small
    diagonal shift and the mixed solve converges."""
    x, y, lo, hi = random_problem(P5, N5, n5, seed=105)
    with B.Plan(P5, N5, G5, 1e-2, precision=B.SPS_PREC_MIXED, max_iter=20000) as pl:
        pl.set_points(x, y)
        coef, res = pl.solve(1e-6)
    with B.Plan(P5, N5, G5, 1e-2, max_iter=20000) as p64:
        p64.set_points(x, y)
        c64, r64 = p64.solve(1e-6)
    print("P=5, lambda 1e-2, tol 1e-6: mixed %d iterations, FP64 %d iterations" % (res.iterations, r64.iterations))
    assert res.status == B.SPS_OK and res.rel_res_true <= 1e-6
    assert res.iterations <= 4 * r64.iterations


# ------------------------------------------------------------------ inner coarse CG (NEXT-2)

def _coarse_setup(P, N, G, n, lam, seed):
    x, y, lo, hi = random_problem(P, N, n, seed=seed)
    Nc = spline.level_intervals(N, G, 1)
    A1 = spline.system(x, y, lo, hi, Nc, 3, lam)[0].toarray()
    return x, y, A1


@pytest.mark.parametrize("P,N,G,n,lam,iters,tol", [
    (2, [8, 8], 3, 3001, 1e-3, 120, 1e-10),      # K_1 = 25
    (3, [8, 8, 8], 3, 6007, 1e-2, 1500, 1e-8),   # K_1 = 125
])
def test_coarse_cg_reaches_direct_coarse_solve(P, N, G, n, lam, iters, tol):
    """With enough inner iterations the matrix-free coarse CG is the exact
    coarse solve: it matches LAPACK's solve of the oracle's A_1."""
    x, y, A1 = _coarse_setup(P, N, G, n, lam, 200 + P)
    r = np.random.default_rng(9).standard_normal(A1.shape[0])
    with B.Plan(P, N, G, lam, coarse_cg=1, coarse_iters=iters) as pl:
        pl.set_points(x, y)
        assert B.sps_level_matrix(pl.h, 1) == 0          # nothing assembled
        e = np.zeros_like(r)
        B.sps_coarse_solve(pl.h, r, e)
    assert rel_err(e, np.linalg.solve(A1, r)) < tol


def test_coarse_cg_energy_error_decreases(p5):
    """CG minimises the A_1-norm of the error over a growing Krylov space:
    more inner iterations never give a worse coarse solution (at P = 5 the
    Jacobi-scaled A_1 has a condition number near 1e11, so the decrease is slow)."""
    A1 = p5["A1"]
    r = np.random.default_rng(10).standard_normal(A1.shape[0])
    e_star = np.linalg.solve(A1, r)
    errs = []
    for iters in (4, 16, 64):
        with B.Plan(P5, N5, G5, LAM5, coarse_cg=1, coarse_iters=iters) as pl:
            pl.set_points(p5["x"], p5["y"])
            e = np.zeros_like(r)
            B.sps_coarse_solve(pl.h, r, e)
        d = e - e_star
        errs.append(float(np.sqrt(d @ A1 @ d)))
    print("P=5 inner coarse CG, A_1-norm error after 4 / 16 / 64 iterations:", errs)
    assert errs[0] > errs[1] > errs[2]


def test_coarse_cg_lifts_the_dense_limit():
    """K_1 = 67^2 = 4489 > 4096: the dense coarse solver is refused, the inner
    coarse CG solves the problem, and the result matches the direct solve."""
    P, N, G, lam = 2, [128, 128], 2, 1e-3
    x, y, lo, hi = random_problem(P, N, 40009, seed=11)
    with pytest.raises(B.SpsError) as e:
        B.Plan(P, N, G, lam)
    assert e.value.code == B.SPS_EINVAL
    with B.Plan(P, N, G, lam, coarse_cg=1, coarse_iters=32) as pl:
        pl.set_points(x, y)
        coef, res = pl.solve(1e-12)
    A, b, _, _ = spline.system(x, y, lo, hi, N, 3, lam)
    assert res.status == B.SPS_OK
    assert rel_err(coef, mgcg.solve_direct(A, b)) < 1e-7
