"""Helpers shared by the GPU tests: oracle-side references for a problem."""
import numpy as np

from oracle import mgcg, spline


def random_problem(P, intervals, n, seed, dtype=np.float64, lo=None, hi=None, edge_points=True):
    r = np.random.default_rng(seed)
    lo = lo if lo is not None else [0.0] * P
    hi = hi if hi is not None else [1.0] * P
    x = np.stack([lo[p] + (hi[p] - lo[p]) * r.random(n) for p in range(P)], axis=1)
    if edge_points and n >= 4:
        x[0] = lo
        x[1] = hi
        x[2, 0] = hi[0]
        x[3] = [lo[p] + (hi[p] - lo[p]) * 0.5 for p in range(P)]   # on interior knots
    y = np.sin(3.0 * x[:, 0]) + (x[:, 1] ** 2 if P > 1 else 0.0) + 0.1 * r.standard_normal(n)
    return np.ascontiguousarray(x.astype(dtype)), np.ascontiguousarray(y.astype(dtype)), lo, hi


def level_ops(x, y, lo, hi, intervals, q, lam, G):
    """Assembled A_g, Lambda_g, diag, prolongations and b for every level g = 1..G."""
    out = {}
    for g in range(1, G + 1):
        Ng = spline.level_intervals(intervals, G, g)
        A, b, Phi, Lam = spline.system(x, y, lo, hi, Ng, q, lam)
        out[g] = dict(N=Ng, A=A, b=b, Lam=Lam, I=spline.prolongation(spline.level_intervals(intervals, G, g - 1), q)
                      if g > 1 else None)
    return out


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def oracle_hierarchy(x, y, lo, hi, intervals, q, lam, G, omega):
    return mgcg.build_hierarchy(x, y, lo, hi, intervals, q, lam, G, omega=list(omega))
