"""Solvers of the oracle: direct solve and the MGCG of Algorithms 6-8.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64 throughout; all
operators are assembled sparse matrices, so every step can be checked by eye
against the algorithms of Section 3.2.

Readings of the paper used here:
* Step size of Algorithm 8: w = r'z / p'v (the preconditioned CG step; the
  printed |r|^2 is the unpreconditioned one and is inconsistent with the
  printed beta = r'z / r~'z~).
* Stopping criterion: |r|_2 <= tol |Phi'y|_2 on the recursive residual, tested
  before each iteration (Algorithm 8 leaves it unstated).
* Coarse operators: by default A_g = Phi_g'Phi_g + lambda Lambda_g with all n
  points on every level (Section 3.2, hierarchy); optionally the Galerkin
  products I' A_{g+1} I, which are equal in exact arithmetic (Section 3.2,
  grid transfer).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import spline


# ---------------------------------------------------------------- direct solve

def banded_upper(A: sp.spmatrix) -> tuple:
    """Upper band storage ab[u + i - j, j] = A[i, j] (i <= j) for LAPACK."""
    A = A.tocoo()
    mask = A.row <= A.col
    r, c, v = A.row[mask], A.col[mask], A.data[mask]
    u = int((c - r).max()) if len(r) else 0
    ab = np.zeros((u + 1, A.shape[0]))
    np.add.at(ab, (u + r - c, c), v)
    return ab, u


def solve_direct(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """alpha* = A^{-1} b for the SPD system of Section 2.2 by banded Cholesky
    (LAPACK pbtrf/pbtrs) in the natural ordering, whose bandwidth is
    q * sum_p stride_p."""
    ab, _ = banded_upper(A)
    cb = sla.cholesky_banded(ab, lower=False)
    return sla.cho_solve_banded((cb, False), b)


# ---------------------------------------------------------------- hierarchy

@dataclass
class Level:
    intervals: list
    A: sp.csr_matrix
    Dinv: np.ndarray
    omega: float
    I: sp.csr_matrix = None      # prolongation from the next coarser level to this one


@dataclass
class Hierarchy:
    levels: list = field(default_factory=list)   # index 0 = coarsest (g = 1)
    coarse_factor: tuple = None
    b: np.ndarray = None


def build_hierarchy(x, y, lo, hi, intervals, q, lam, G, omega=None, galerkin=False) -> Hierarchy:
    """Operators of every level g = 1..G (Section 3.2).  omega is one value
    for all levels, a list per level (coarsest first), or None for
    1 / lambda_max(D_g^-1 A_g) computed by a dense or Lanczos eigen-solve."""
    H = Hierarchy()
    A_fine, b, _, _ = spline.system(x, y, lo, hi, intervals, q, lam)
    H.b = b
    mats = [None] * G
    if galerkin:
        mats[G - 1] = A_fine
        for g in range(G - 1, 0, -1):
            Ic = spline.prolongation(spline.level_intervals(intervals, G, g), q)
            mats[g - 1] = (Ic.T @ mats[g] @ Ic).tocsr()
    else:
        for g in range(1, G + 1):
            Ng = spline.level_intervals(intervals, G, g)
            mats[g - 1] = A_fine if g == G else spline.system(x, y, lo, hi, Ng, q, lam)[0]
    for g in range(1, G + 1):
        Ng = spline.level_intervals(intervals, G, g)
        A = mats[g - 1]
        d = A.diagonal()
        Dinv = 1.0 / d
        if omega is None:
            om = 1.0 / lambda_max_jacobi(A, Dinv)
        elif np.isscalar(omega):
            om = float(omega)
        else:
            om = float(omega[g - 1])
        I = spline.prolongation(spline.level_intervals(intervals, G, g - 1), q) if g > 1 else None
        H.levels.append(Level(Ng, A, Dinv, om, I))
    A1 = H.levels[0].A.toarray()
    H.coarse_factor = sla.cho_factor(A1)
    return H


def lambda_max_jacobi(A: sp.spmatrix, Dinv: np.ndarray) -> float:
    """Largest eigenvalue of D^-1 A (similar to the symmetric D^-1/2 A D^-1/2)."""
    s = np.sqrt(Dinv)
    S = sp.diags(s) @ A @ sp.diags(s)
    if S.shape[0] <= 2000:
        return float(np.linalg.eigvalsh(S.toarray())[-1])
    import scipy.sparse.linalg as spla
    return float(spla.eigsh(S, k=1, which="LA", return_eigenvectors=False, tol=1e-10)[0])


# ---------------------------------------------------------------- Algorithms 6-8

def jacobi(L: Level, alpha: np.ndarray, b: np.ndarray, nu: int) -> np.ndarray:
    """Algorithm 6: nu damped Jacobi sweeps alpha <- alpha + omega D^-1 (b - A alpha)."""
    for _ in range(nu):
        r = b - L.A @ alpha
        alpha = alpha + L.omega * L.Dinv * r
    return alpha


def v_cycle(H: Hierarchy, g: int, b: np.ndarray, nu1: int, nu2: int) -> np.ndarray:
    """Algorithm 7 from alpha = 0 on level g (1-based): exact coarse solve on
    g = 1; otherwise pre-smooth, r = A alpha - b, restrict by I', recurse,
    alpha <- alpha - I e, post-smooth."""
    if g == 1:
        return sla.cho_solve(H.coarse_factor, b)
    L = H.levels[g - 1]
    alpha = jacobi(L, np.zeros_like(b), b, nu1)
    r = L.A @ alpha - b
    rc = L.I.T @ r
    e = v_cycle(H, g - 1, rc, nu1, nu2)
    alpha = alpha - L.I @ e
    return jacobi(L, alpha, b, nu2)


@dataclass
class CGResult:
    alpha: np.ndarray
    iterations: int
    rel_res: float
    history: list


def mgcg(H: Hierarchy, tol: float, nu1: int = 1, nu2: int = 1, max_iter: int = 500,
         precondition: bool = True) -> CGResult:
    """Algorithm 8 (MGCG) from alpha = 0; with precondition=False it is plain CG
    on A_G (the comparison method of Section 4)."""
    G = len(H.levels)
    A = H.levels[-1].A
    b = H.b
    nb = np.linalg.norm(b)
    alpha = np.zeros_like(b)
    r = b.copy()
    z = v_cycle(H, G, r, nu1, nu2) if precondition else r.copy()
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r) / nb]
    it = 0
    while hist[-1] > tol and it < max_iter:
        v = A @ p
        w = rz / (p @ v)
        alpha = alpha + w * p
        r = r - w * v
        z = v_cycle(H, G, r, nu1, nu2) if precondition else r.copy()
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        hist.append(np.linalg.norm(r) / nb)
    return CGResult(alpha, it, hist[-1], hist)


def solve_tier2(x, y, lo, hi, intervals, q, lam, G, tol, omega=None, nu1=1, nu2=1, max_iter=20000) -> CGResult:
    """alpha* = A^-1 b for problems too large for the banded Cholesky: Algorithm 8
    on assembled matrices with the Galerkin coarse operators I' A_{g+1} I
    (Section 3.2, grid transfer), run to |r| <= tol |b| (tol = 1e-13 or below).
    The coarse operators come from the fine matrix by another route than the
    rediscretisation that the CUDA path uses; both give A_g in exact arithmetic."""
    H = build_hierarchy(x, y, lo, hi, intervals, q, lam, G, omega=omega, galerkin=True)
    return mgcg(H, tol, nu1=nu1, nu2=nu2, max_iter=max_iter)
