"""Full-size checks of the oracle: outputs one coefficient at a time.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64 throughout.

At the full sizes of the workloads the explicit Phi of a whole level can be
too large to hold, so these functions compute the operator
u = (Phi'Phi + lambda Lambda) v (Section 2.2) either for chosen coefficients
k only, from the points inside the support of phi_k, or over all points in
chunks (the sum over points of Algorithm 3, applied to the gathered values of
Algorithm 4).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import spline


def _local_basis(xs, lo, hi, intervals, q):
    """Per point and dimension: the first active basis index and the q+1 values."""
    P = xs.shape[1]
    out = []
    for p in range(P):
        c = spline.cell_index(xs[:, p], lo[p], hi[p], intervals[p])
        B = spline.basis_1d(xs[:, p], lo[p], hi[p], intervals[p], q)
        idx = c[:, None] + np.arange(q + 1)[None, :]
        out.append((c, np.take_along_axis(B, idx, axis=1)))
    return out


def _point_rows(xs, lo, hi, intervals, q):
    """Column indices and values of the rows of Phi for the points xs."""
    P = xs.shape[1]
    J = [N + q for N in intervals]
    st = spline.strides(J)
    loc = _local_basis(xs, lo, hi, intervals, q)
    cols, vals = [], []
    for combo in itertools.product(range(q + 1), repeat=P):
        col = np.zeros(xs.shape[0], dtype=np.int64)
        val = np.ones(xs.shape[0])
        for p in range(P):
            col += (loc[p][0] + combo[p]) * st[p]
            val *= loc[p][1][:, combo[p]]
        cols.append(col)
        vals.append(val)
    return np.stack(cols, axis=1), np.stack(vals, axis=1)


def penalty_rows(ks, lo, hi, intervals, q) -> tuple:
    """Rows k of Lambda as (columns, values): products of 1-D Gram rows
    (Section 2.4, Kronecker structure of Psi_r)."""
    P = len(intervals)
    J = [N + q for N in intervals]
    st = spline.strides(J)
    grams = [[spline.gram_1d(lo[p], hi[p], intervals[p], q, r) for r in range(3)] for p in range(P)]
    out = []
    for k in ks:
        idx = []
        rem = int(k)
        for p in range(P):
            idx.append(rem // st[p]); rem %= st[p]
        acc = {}
        for r, w in spline.penalty_multiindices(P):
            # sparse product of the 1-D rows
            terms = [(0, w)]
            for p in range(P):
                row = grams[p][r[p]][idx[p]]
                nz = np.nonzero(row)[0]
                terms = [(c + j * st[p], v * row[j]) for (c, v) in terms for j in nz]
            for c, v in terms:
                acc[c] = acc.get(c, 0.0) + v
        cols = np.array(sorted(acc))
        out.append((cols, np.array([acc[c] for c in cols])))
    return out


def apply_rows(x, v, ks, lo, hi, intervals, q, lam) -> np.ndarray:
    """u[k] = sum_i phi_k(x_i) (Phi v)_i + lambda (Lambda v)_k for the chosen k."""
    x = np.asarray(x)
    P = x.shape[1]
    J = [N + q for N in intervals]
    st = spline.strides(J)
    cells = np.stack([spline.cell_index(x[:, p], lo[p], hi[p], intervals[p]) for p in range(P)], axis=1)
    pen = penalty_rows(ks, lo, hi, intervals, q)
    out = np.zeros(len(ks))
    for t, k in enumerate(ks):
        idx = []
        rem = int(k)
        for p in range(P):
            idx.append(rem // st[p]); rem %= st[p]
        mask = np.ones(x.shape[0], dtype=bool)
        for p in range(P):
            mask &= (cells[:, p] >= idx[p] - q) & (cells[:, p] <= idx[p])
        sel = np.nonzero(mask)[0]
        acc = 0.0
        if len(sel):
            cols, vals = _point_rows(x[sel], lo, hi, intervals, q)
            s = np.sum(vals * v[cols], axis=1)               # Algorithm 4 on the selected points
            acc = float(np.sum(np.where(cols == k, vals, 0.0) * s[:, None]))  # Algorithm 3
        pc, pv = pen[t]
        out[t] = acc + lam * float(pv @ v[pc])
    return out


def apply_phitphi_chunked(x, v, lo, hi, intervals, q, chunk: int = 20000) -> np.ndarray:
    """u = Phi'(Phi v) over all points in chunks, without forming Phi."""
    K = int(np.prod([N + q for N in intervals]))
    u = np.zeros(K)
    for s in range(0, x.shape[0], chunk):
        xs = x[s:s + chunk]
        cols, vals = _point_rows(xs, lo, hi, intervals, q)
        sv = np.sum(vals * v[cols], axis=1)
        u += np.bincount(cols.ravel(), weights=(vals * sv[:, None]).ravel(), minlength=K)
    return u


def rhs_chunked(x, y, lo, hi, intervals, q, chunk: int = 20000) -> np.ndarray:
    """b = Phi'y over all points in chunks (Algorithm 3 with the responses)."""
    K = int(np.prod([N + q for N in intervals]))
    b = np.zeros(K)
    y = np.asarray(y, dtype=np.float64)
    for s in range(0, x.shape[0], chunk):
        cols, vals = _point_rows(x[s:s + chunk], lo, hi, intervals, q)
        b += np.bincount(cols.ravel(), weights=(vals * y[s:s + chunk, None]).ravel(), minlength=K)
    return b


def penalty_apply_kron(v, lo, hi, intervals, q) -> np.ndarray:
    """Lambda v = sum_{|r|=2} (2/r!) (kron_p Psi^p_{r_p}) v without forming
    Lambda: v is reshaped to the J_1 x ... x J_P tensor (last index fastest)
    and each 1-D Gram matrix is applied along its own axis, the Kronecker
    matrix-vector product of Algorithm 2."""
    P = len(intervals)
    J = [N + q for N in intervals]
    grams = [[spline.gram_1d(lo[p], hi[p], intervals[p], q, r) for r in range(3)] for p in range(P)]
    V = np.asarray(v, dtype=np.float64).reshape(J)
    out = np.zeros_like(V)
    for r, w in spline.penalty_multiindices(P):
        T = V
        for p in range(P):
            T = np.moveaxis(np.tensordot(grams[p][r[p]], T, axes=([1], [p])), 0, p)
        out += w * T
    return out.ravel()


def residual_norm(x, y, alpha, lo, hi, intervals, q, lam, chunk: int = 20000) -> float:
    """|Phi'y - (Phi'Phi + lambda Lambda) alpha|_2 / |Phi'y|_2, matrix free."""
    b = rhs_chunked(x, y, lo, hi, intervals, q, chunk)
    Av = apply_phitphi_chunked(x, alpha, lo, hi, intervals, q, chunk) + lam * penalty_apply_kron(alpha, lo, hi,
                                                                                                intervals, q)
    return float(np.linalg.norm(b - Av) / np.linalg.norm(b))
