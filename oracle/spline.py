"""Spline objects of the oracle: basis, Phi, Gram matrices, Lambda, transfers.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64 throughout.

Readings of the paper used here:
* Knots: extended uniform ("cardinal") knots.  With N intervals of width
  h = (hi - lo)/N on [lo, hi], knot t_i = lo + (i - q) h for i = 0..N+2q, and
  basis function j = 0..N+q-1 lives on [t_j, t_{j+q+1}].  J = N + q matches
  J = m + q + 1 with m = N - 1 interior knots (Section 2.1), and makes the
  subdivision matrix of Section 2.4 shift-invariant in every row.
* Linear index: row-major over the multi-index with the last dimension
  fastest, the order of the Kronecker products in Section 2.4.
* Penalty: Lambda = sum_{|r|=2} (2/r!) Psi_r with Psi_r = kron_p Psi^p_{r_p}
  and Gram integrals over Omega = prod [lo_p, hi_p] (Section 2.2, 2.4).
* Cell of a point: c = min(floor((x - lo) * (N/(hi - lo))), N - 1), evaluated
  in the precision of the input (a point at hi belongs to the last cell).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp


# ---------------------------------------------------------------- knots, cells

def intervals_at_level(N: int, G: int, g: int) -> int:
    """Intervals of grid level g (1 = coarsest, G = finest): the spacing halves
    from one level to the next (Section 3.2, hierarchy)."""
    return N >> (G - g)


def coef_count(intervals, q: int) -> int:
    """K = prod_p J_p with J_p = N_p + q (Section 2.1)."""
    return int(np.prod([N + q for N in intervals], dtype=np.int64))


def extended_knots(lo: float, hi: float, N: int, q: int) -> np.ndarray:
    h = (hi - lo) / N
    return lo + (np.arange(N + 2 * q + 1) - q) * h


def cell_index(x, lo: float, hi: float, N: int) -> np.ndarray:
    """Knot interval of each coordinate (reading of the support of B-splines,
    Section 2.1): floor((x - lo) * (N/(hi - lo))) clamped to N - 1, in the
    floating-point type of x."""
    x = np.asarray(x)
    dt = np.float32 if x.dtype == np.float32 else np.float64
    inv = dt(N / (hi - lo))
    u = (x.astype(dt) - dt(lo)) * inv
    c = np.floor(u).astype(np.int64)
    return np.minimum(c, N - 1)


def morton_key(cells: np.ndarray, bits: int) -> np.ndarray:
    """Sort key of a point: the bits of its finest-level cell multi-index
    interleaved from the most significant bit down, dimension 1 first within a
    bit.  Every power-of-two block of cells on every level is then a
    contiguous key range."""
    cells = np.asarray(cells, dtype=np.uint64)
    n, P = cells.shape
    key = np.zeros(n, dtype=np.uint64)
    for b in range(bits - 1, -1, -1):
        for p in range(P):
            key = (key << np.uint64(1)) | ((cells[:, p] >> np.uint64(b)) & np.uint64(1))
    return key


def sort_permutation(x: np.ndarray, lo, hi, intervals) -> tuple:
    """Stable order of the points by Morton key of their finest cells."""
    P = x.shape[1]
    cells = np.stack([cell_index(x[:, p], lo[p], hi[p], intervals[p]) for p in range(P)], axis=1)
    bits = max(int(N - 1).bit_length() for N in intervals)
    bits = max(bits, 1)
    key = morton_key(cells, bits)
    perm = np.argsort(key, kind="stable")
    return perm, key, cells


# ---------------------------------------------------------------- 1-D basis

def basis_1d(x: np.ndarray, lo: float, hi: float, N: int, q: int, deriv: int = 0) -> np.ndarray:
    """All J = N + q B-splines of degree q (or their deriv-th derivative) at the
    points, as a dense (n, J) array, by the Cox-de Boor recursion (de Boor
    1978; Section 2.1).  Degree 0 is the indicator of the point's cell, so the
    closed right end x = hi belongs to the last interval."""
    if deriv > q:
        raise ValueError("derivative order above the spline degree")
    cells = cell_index(x, lo, hi, N)               # in the input precision
    x = np.asarray(x).astype(np.float64)           # FP32 inputs widen exactly
    t = extended_knots(lo, hi, N, q)
    n = x.shape[0]
    nint = N + 2 * q
    B = np.zeros((n, nint))
    B[np.arange(n), cells + q] = 1.0
    top = q - deriv
    for k in range(1, top + 1):                    # raise the degree to q - deriv
        Bn = np.zeros((n, nint - k))
        for j in range(nint - k):
            d1 = t[j + k] - t[j]
            d2 = t[j + k + 1] - t[j + 1]
            Bn[:, j] = (x - t[j]) / d1 * B[:, j] + (t[j + k + 1] - x) / d2 * B[:, j + 1]
        B = Bn
    for k in range(top + 1, q + 1):                # differentiate: d/dx B_{j,k} in terms of degree k-1
        Bn = np.zeros((n, nint - k))
        for j in range(nint - k):
            Bn[:, j] = k * (B[:, j] / (t[j + k] - t[j]) - B[:, j + 1] / (t[j + k + 1] - t[j + 1]))
        B = Bn
    return B


def greville(lo: float, hi: float, N: int, q: int) -> np.ndarray:
    """Greville abscissae xi_j = mean of the q interior knots of B_j; with them
    sum_j xi_j B_j(x) = x (linear precision)."""
    t = extended_knots(lo, hi, N, q)
    J = N + q
    return np.array([t[j + 1:j + q + 1].mean() for j in range(J)])


# ---------------------------------------------------------------- Phi

def strides(J) -> list:
    """Row-major strides with the last dimension fastest."""
    P = len(J)
    s = [1] * P
    for p in range(P - 2, -1, -1):
        s[p] = s[p + 1] * J[p + 1]
    return s


def phi_matrix(x: np.ndarray, lo, hi, intervals, q: int, chunk: int = 20000) -> sp.csr_matrix:
    """Phi[i, k] = phi_k(x_i) = prod_p phi^p_{k_p}(x_i^p) (Section 2.1/2.2), as a
    sparse n x K matrix.  Row i is the Kronecker (Khatri-Rao) product of the
    1-D basis rows of x_i (Section 2.4); only the (q+1)^P nonzeros are kept."""
    x = np.asarray(x)
    n, P = x.shape
    J = [N + q for N in intervals]
    st = strides(J)
    K = int(np.prod(J))
    rows, cols, vals = [], [], []
    for s in range(0, n, chunk):
        xs = x[s:s + chunk]
        m = xs.shape[0]
        loc = []
        for p in range(P):
            Bp = basis_1d(xs[:, p], lo[p], hi[p], intervals[p], q)
            c = cell_index(xs[:, p], lo[p], hi[p], intervals[p])
            idx = c[:, None] + np.arange(q + 1)[None, :]
            loc.append((idx, np.take_along_axis(Bp, idx, axis=1)))
        for combo in itertools.product(range(q + 1), repeat=P):
            col = np.zeros(m, dtype=np.int64)
            val = np.ones(m)
            for p in range(P):
                col += loc[p][0][:, combo[p]] * st[p]
                val *= loc[p][1][:, combo[p]]
            rows.append(np.arange(s, s + m))
            cols.append(col)
            vals.append(val)
    rows = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    vals = np.concatenate(vals) if vals else np.zeros(0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, K))


# ---------------------------------------------------------------- Gram, Lambda

def gram_1d(lo: float, hi: float, N: int, q: int, r: int) -> np.ndarray:
    """Psi^p_r[j, l] = <d^r phi_j, d^r phi_l>_{L2[lo,hi]} (Section 2.4) by
    Gauss-Legendre quadrature with q+1 nodes per knot interval, exact for the
    piecewise polynomials of degree <= 2q that are integrated."""
    nodes, weights = np.polynomial.legendre.leggauss(q + 1)
    h = (hi - lo) / N
    xs, ws = [], []
    for c in range(N):
        a = lo + c * h
        xs.append(a + (nodes + 1.0) * 0.5 * h)
        ws.append(weights * 0.5 * h)
    xs = np.concatenate(xs)
    ws = np.concatenate(ws)
    D = basis_1d(xs, lo, hi, N, q, deriv=r)
    return D.T @ (ws[:, None] * D)


def penalty_multiindices(P: int) -> list:
    """All r in N_0^P with |r| = 2, with the weight 2/r! (Section 2.2)."""
    out = []
    for r in itertools.product(range(3), repeat=P):
        if sum(r) == 2:
            out.append((r, 2.0 / math.prod(math.factorial(v) for v in r)))
    return out


def penalty_matrix(lo, hi, intervals, q: int) -> sp.csr_matrix:
    """Lambda = sum_{|r|=2} (2/r!) kron_{p=1..P} Psi^p_{r_p} (Section 2.2, 2.4)."""
    P = len(intervals)
    grams = [[sp.csr_matrix(gram_1d(lo[p], hi[p], intervals[p], q, r)) for r in range(3)]
             for p in range(P)]
    K = coef_count(intervals, q)
    L = sp.csr_matrix((K, K))
    for r, w in penalty_multiindices(P):
        term = grams[0][r[0]]
        for p in range(1, P):
            term = sp.kron(term, grams[p][r[p]], format="csr")
        L = L + w * term
    return L.tocsr()


# ---------------------------------------------------------------- transfers

def subdivision_1d(N_coarse: int, q: int) -> sp.csr_matrix:
    """I^h_{2h}[i, j] = 2^-q binom(q+1, i - 2j + q) for the 0-based indices of
    the extended-knot basis (the 1-based formula of Section 2.4 shifted by
    one), J_fine x J_coarse with J = N + q."""
    Jc = N_coarse + q
    Jf = 2 * N_coarse + q
    rows, cols, vals = [], [], []
    for j in range(Jc):
        for k in range(q + 2):
            i = 2 * j - q + k
            if 0 <= i < Jf:
                rows.append(i); cols.append(j)
                vals.append(math.comb(q + 1, k) / 2.0 ** q)
    return sp.csr_matrix((vals, (rows, cols)), shape=(Jf, Jc))


def prolongation(intervals_coarse, q: int) -> sp.csr_matrix:
    """I_{g-1}^{g} = kron_p I^{h_p}_{2h_p} (Section 2.4, Section 3.2 grid transfer)."""
    M = subdivision_1d(intervals_coarse[0], q)
    for N in intervals_coarse[1:]:
        M = sp.kron(M, subdivision_1d(N, q), format="csr")
    return M.tocsr()


# ---------------------------------------------------------------- system

def system(x, y, lo, hi, intervals, q: int, lam: float) -> tuple:
    """A = Phi'Phi + lambda Lambda and b = Phi'y (the normal equations of
    Section 2.2).  Returns (A, b, Phi, Lambda)."""
    Phi = phi_matrix(x, lo, hi, intervals, q)
    Lam = penalty_matrix(lo, hi, intervals, q)
    A = (Phi.T @ Phi + lam * Lam).tocsr()
    b = Phi.T @ np.asarray(y, dtype=np.float64)
    return A, b, Phi, Lam


def diag_phitphi(Phi: sp.csr_matrix) -> np.ndarray:
    """diag(Phi'Phi)[j] = sum_i v_i[j]^2 (Algorithm 5)."""
    return np.asarray(Phi.multiply(Phi).sum(axis=0)).ravel()


def level_intervals(intervals, G: int, g: int) -> list:
    return [intervals_at_level(N, G, g) for N in intervals]
