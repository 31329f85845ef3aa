"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value
printed in the paper, a closed form, an invariant, a special case that
reduces to a library routine, or brute force on a tiny input.  Together they
are chosen so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import mgcg, sampled, spline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ counts

def test_table1_coefficient_counts():
    """Table 1 (Section 2.3): K = 35^P for J_p = 35 cubic B-splines per dim."""
    for P, K in _read_golden("table1_K.txt"):
        assert spline.coef_count([32] * int(P), 3) == int(K)


def test_level_dimension_formula():
    """Section 3.2 (hierarchy): K_g = (2^g + 3)^P for m_p = 2^g - 1 interior knots."""
    for P in (1, 2, 3):
        for G in (3, 5):
            for g in range(1, G + 1):
                Ng = spline.level_intervals([2 ** G] * P, G, g)
                assert spline.coef_count(Ng, 3) == (2 ** g + 3) ** P


# ------------------------------------------------------------------ basis

@pytest.mark.parametrize("q", [1, 2, 3])
def test_partition_of_unity(q):
    lo, hi, N = -0.7, 2.3, 11
    x = np.concatenate([lo + (hi - lo) * RNG.random(500), [lo, hi], lo + (hi - lo) * np.arange(N + 1) / N])
    B = spline.basis_1d(x, lo, hi, N, q)
    assert B.shape == (x.size, N + q)
    assert np.all(B >= -1e-15)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)


def test_cubic_values_at_knots():
    """Uniform cubic B-spline takes 1/6, 2/3, 1/6 at its three interior knots."""
    N = 8
    x = np.arange(1, N) / N                     # interior knots of [0, 1]
    B = spline.basis_1d(x, 0.0, 1.0, N, 3)
    for i, xi in enumerate(x):
        nz = np.sort(B[i][B[i] > 1e-14])
        np.testing.assert_allclose(nz, [1 / 6, 1 / 6, 2 / 3], atol=1e-14)


@pytest.mark.parametrize("q", [2, 3])
def test_linear_and_quadratic_precision(q):
    """Marsden's identity: x = sum xi_j B_j, x^2 = sum sigma2(t_{j+1..j+q})/C(q,2) B_j."""
    lo, hi, N = 0.25, 1.75, 7
    x = lo + (hi - lo) * RNG.random(300)
    B = spline.basis_1d(x, lo, hi, N, q)
    t = spline.extended_knots(lo, hi, N, q)
    xi = spline.greville(lo, hi, N, q)
    np.testing.assert_allclose(B @ xi, x, atol=1e-13)
    c2 = np.array([sum(a * b for a, b in itertools.combinations(t[j + 1:j + q + 1], 2)) / math.comb(q, 2)
                   for j in range(N + q)])
    np.testing.assert_allclose(B @ c2, x * x, atol=1e-13)


def test_phi_tensor_order_unequal_grids():
    """Phi alpha reproduces x_p and x_1 x_3 for Greville tensors (catches a
    transposed multi-index order; grids differ per dimension)."""
    intervals = [4, 8, 2]
    lo, hi = [0.0, -1.0, 2.0], [1.0, 1.0, 5.0]
    q = 3
    n = 400
    x = np.stack([lo[p] + (hi[p] - lo[p]) * RNG.random(n) for p in range(3)], axis=1)
    Phi = spline.phi_matrix(x, lo, hi, intervals, q)
    J = [N + q for N in intervals]
    grids = np.meshgrid(*[spline.greville(lo[p], hi[p], intervals[p], q) for p in range(3)], indexing="ij")
    for p in range(3):
        np.testing.assert_allclose(Phi @ grids[p].ravel(), x[:, p], atol=1e-12)
    np.testing.assert_allclose(Phi @ (grids[0] * grids[2]).ravel(), x[:, 0] * x[:, 2], atol=1e-12)
    assert Phi.shape == (n, int(np.prod(J)))
    assert np.all(np.diff(Phi.indptr) == (q + 1) ** 3)


# ------------------------------------------------------------------ Gram / penalty

def _exact_gram_uniform_cubic(N, r):
    """Exact rational Gram matrix of the cubic B-splines on [0, N] (h = 1) by
    integrating the four uniform pieces symbolically (independent of the
    oracle's Cox-de Boor and Gauss-Legendre)."""
    sympy = pytest.importorskip("sympy")
    t = sympy.symbols("t")
    pieces = [(1 - t) ** 3 / 6, (3 * t ** 3 - 6 * t ** 2 + 4) / 6,
              (-3 * t ** 3 + 3 * t ** 2 + 3 * t + 1) / 6, t ** 3 / 6]
    d = [sympy.diff(pc, t, r) for pc in pieces]
    E = [[sympy.integrate(d[a] * d[b], (t, 0, 1)) for b in range(4)] for a in range(4)]
    J = N + 3
    G = [[sympy.Integer(0)] * J for _ in range(J)]
    for c in range(N):               # cell c carries functions c..c+3 with piece index j - c
        for a in range(4):
            for b in range(4):
                G[c + a][c + b] += E[a][b]
    return np.array([[float(v) for v in row] for row in G])


@pytest.mark.parametrize("r", [0, 1, 2])
def test_gram_matrices_exact(r):
    N = 6
    G = spline.gram_1d(0.0, float(N), N, 3, r)
    np.testing.assert_allclose(G, _exact_gram_uniform_cubic(N, r), atol=1e-13)


def test_gram_interior_closed_forms():
    """Interior rows from the B-spline convolution identity, scaled by h^(1-2r)."""
    h = 0.125
    M = np.array([1, 120, 1191, 2416, 1191, 120, 1]) / 5040 * h
    D1 = np.array([-1 / 120, -1 / 5, -1 / 8, 2 / 3, -1 / 8, -1 / 5, -1 / 120]) / h
    D2 = np.array([1 / 6, 0, -3 / 2, 8 / 3, -3 / 2, 0, 1 / 6]) / h ** 3
    for r, ref in enumerate([M, D1, D2]):
        G = spline.gram_1d(0.0, 1.0, 8, 3, r)
        np.testing.assert_allclose(G[5, 2:9], ref, rtol=1e-12, atol=1e-9 * np.abs(ref).max())


def _quadratic_coefs(lo, hi, intervals, q, H, g):
    """Spline coefficients of s(x) = 1/2 x'Hx + g'x (exactly representable)."""
    P = len(intervals)
    xi = [spline.greville(lo[p], hi[p], intervals[p], q) for p in range(P)]
    sq = []
    for p in range(P):
        t = spline.extended_knots(lo[p], hi[p], intervals[p], q)
        sq.append(np.array([sum(a * b for a, b in itertools.combinations(t[j + 1:j + q + 1], 2)) / math.comb(q, 2)
                            for j in range(intervals[p] + q)]))
    J = [N + q for N in intervals]
    alpha = np.zeros(J)
    one = [np.ones(Jp) for Jp in J]

    def outer(vs):
        out = vs[0]
        for v in vs[1:]:
            out = np.multiply.outer(out, v)
        return out
    for a in range(P):
        vs = list(one); vs[a] = sq[a]
        alpha += 0.5 * H[a, a] * outer(vs)
        vs = list(one); vs[a] = xi[a]
        alpha += g[a] * outer(vs)
        for b in range(a + 1, P):
            vs = list(one); vs[a] = xi[a]; vs[b] = xi[b]
            alpha += H[a, b] * outer(vs)
    return alpha.ravel()


@pytest.mark.parametrize("P", [1, 2, 3])
def test_penalty_is_thin_plate_energy(P):
    """alpha' Lambda alpha = vol(Omega) |Hessian|_F^2 for a quadratic (Section
    2.2 with the 2/r! weights), and Lambda annihilates affine functions."""
    intervals = [5, 3, 4][:P]
    lo = [0.0, -0.5, 1.0][:P]
    hi = [1.0, 1.5, 4.0][:P]
    q = 3
    Lam = spline.penalty_matrix(lo, hi, intervals, q)
    vol = float(np.prod(np.array(hi) - np.array(lo)))
    A = RNG.standard_normal((P, P))
    H = A + A.T
    g = RNG.standard_normal(P)
    alpha = _quadratic_coefs(lo, hi, intervals, q, H, g)
    np.testing.assert_allclose(alpha @ (Lam @ alpha), vol * np.sum(H * H), rtol=1e-10)
    aff = _quadratic_coefs(lo, hi, intervals, q, np.zeros((P, P)), g)
    assert np.abs(Lam @ aff).max() < 1e-9 * np.abs(Lam).max() * np.abs(aff).max()
    # Lambda is symmetric positive semidefinite
    Ld = Lam.toarray()
    np.testing.assert_allclose(Ld, Ld.T, atol=1e-12 * np.abs(Ld).max())
    assert np.linalg.eigvalsh(Ld).min() > -1e-9 * np.abs(Ld).max()


def test_penalty_by_2d_quadrature():
    """Lambda from tensor Gauss quadrature of sum_{p1,p2} d_p1 d_p2 phi_k d_p1 d_p2 phi_l
    over the 2-D domain equals the Kronecker-sum assembly (Section 2.4)."""
    intervals, q = [3, 4], 3
    lo, hi = [0.0, 0.0], [1.0, 2.0]
    nodes, weights = np.polynomial.legendre.leggauss(q + 1)
    pts, wts = [], []
    for p in range(2):
        h = (hi[p] - lo[p]) / intervals[p]
        xs = np.concatenate([lo[p] + c * h + (nodes + 1) * 0.5 * h for c in range(intervals[p])])
        ws = np.concatenate([weights * 0.5 * h for _ in range(intervals[p])])
        pts.append(xs); wts.append(ws)
    D = [[spline.basis_1d(pts[p], lo[p], hi[p], intervals[p], q, deriv=r) for r in range(3)] for p in range(2)]
    W = np.outer(wts[0], wts[1]).ravel()

    def tens(r0, r1):  # (quad points) x K values of d^(r0,r1) phi_k
        return np.einsum("ai,bj->abij", D[0][r0], D[1][r1]).reshape(W.size, -1)
    S = [(tens(2, 0), tens(2, 0)), (tens(0, 2), tens(0, 2)), (tens(1, 1), tens(1, 1)), (tens(1, 1), tens(1, 1))]
    L2 = sum(a.T @ (W[:, None] * b) for a, b in S)
    Lam = spline.penalty_matrix(lo, hi, intervals, q).toarray()
    np.testing.assert_allclose(Lam, L2, atol=1e-10 * np.abs(L2).max())


# ------------------------------------------------------------------ transfers

@pytest.mark.parametrize("P", [1, 2, 3])
def test_subdivision_reproduces_coarse_spline(P):
    """alpha^h = I alpha^2h gives the same function (Section 2.4)."""
    Nc = [3, 2, 4][:P]
    lo, hi = [0.0] * P, [1.0] * P
    q = 3
    x = RNG.random((300, P))
    x[0] = 0.0; x[1] = 1.0
    ac = RNG.standard_normal(spline.coef_count(Nc, q))
    I = spline.prolongation(Nc, q)
    sc = spline.phi_matrix(x, lo, hi, Nc, q) @ ac
    sf = spline.phi_matrix(x, lo, hi, [2 * N for N in Nc], q) @ (I @ ac)
    np.testing.assert_allclose(sf, sc, atol=1e-13)


def test_galerkin_identity():
    """A_g = I' A_{g+1} I with every level rediscretised on all points (Section 3.2)."""
    P, q, lam = 2, 3, 1e-2
    x = RNG.random((500, P)); y = RNG.standard_normal(500)
    lo, hi = [0.0] * P, [1.0] * P
    Af = spline.system(x, y, lo, hi, [8, 4], q, lam)[0]
    Ac = spline.system(x, y, lo, hi, [4, 2], q, lam)[0]
    I = spline.prolongation([4, 2], q)
    np.testing.assert_allclose((I.T @ Af @ I).toarray(), Ac.toarray(), atol=1e-12 * abs(Ac).max())


# ------------------------------------------------------------------ operator and solve

def _dense_phi_brute(x, lo, hi, intervals, q):
    """phi_k(x_i) = prod_p B^p_{k_p}(x_i^p) by looping over every k (no local window)."""
    P = x.shape[1]
    Bs = [spline.basis_1d(x[:, p], lo[p], hi[p], intervals[p], q) for p in range(P)]
    J = [N + q for N in intervals]
    cols = []
    for k in itertools.product(*[range(j) for j in J]):
        v = np.ones(x.shape[0])
        for p in range(P):
            v = v * Bs[p][:, k[p]]
        cols.append(v)
    return np.stack(cols, axis=1)


def test_brute_force_dense_solve():
    P, q, lam = 2, 3, 3e-3
    intervals = [4, 6]
    lo, hi = [0.0, 0.0], [1.0, 1.0]
    x = RNG.random((300, P)); y = np.sin(3 * x[:, 0]) + x[:, 1] ** 2 + 0.1 * RNG.standard_normal(300)
    A, b, Phi, Lam = spline.system(x, y, lo, hi, intervals, q, lam)
    Pd = _dense_phi_brute(x, lo, hi, intervals, q)
    np.testing.assert_allclose(Phi.toarray(), Pd, atol=1e-15)
    Ad = Pd.T @ Pd + lam * Lam.toarray()
    np.testing.assert_allclose(A.toarray(), Ad, atol=1e-12)
    np.testing.assert_allclose(A.toarray(), A.toarray().T, atol=1e-13)
    assert np.linalg.eigvalsh(Ad).min() > 0
    # Algorithm 5 against the brute-force diagonal
    np.testing.assert_allclose(spline.diag_phitphi(Phi), np.sum(Pd * Pd, axis=0), atol=1e-14)
    a_ref = np.linalg.solve(Ad, Pd.T @ y)
    np.testing.assert_allclose(mgcg.solve_direct(A, b), a_ref, rtol=1e-9, atol=1e-10 * np.abs(a_ref).max())


def test_direct_solve_matches_splu():
    P, q, lam = 3, 3, 1e-3
    intervals = [4, 4, 8]
    x = RNG.random((3000, P)); y = RNG.standard_normal(3000)
    A, b, _, _ = spline.system(x, y, [0.0] * 3, [1.0] * 3, intervals, q, lam)
    a1 = mgcg.solve_direct(A, b)
    a2 = spla.splu(A.tocsc()).solve(b)
    np.testing.assert_allclose(a1, a2, rtol=1e-9, atol=1e-11 * np.abs(a2).max())


@pytest.mark.parametrize("lam", [1e-4, 1e-1, 10.0])
def test_null_space_recovery(lam):
    """Affine data: alpha*_k = c0 + sum_p c_p xi_{k_p} for every lambda."""
    P, q = 3, 3
    intervals = [4, 2, 8]
    lo, hi = [0.0, -1.0, 0.5], [1.0, 1.0, 1.5]
    x = np.stack([lo[p] + (hi[p] - lo[p]) * RNG.random(800) for p in range(P)], axis=1)
    c = RNG.standard_normal(P + 1)
    y = c[0] + x @ c[1:]
    A, b, _, _ = spline.system(x, y, lo, hi, intervals, q, lam)
    alpha = mgcg.solve_direct(A, b)
    grids = np.meshgrid(*[spline.greville(lo[p], hi[p], intervals[p], q) for p in range(P)], indexing="ij")
    ref = c[0] + sum(c[p + 1] * grids[p] for p in range(P))
    np.testing.assert_allclose(alpha, ref.ravel(), atol=1e-9)


def test_lambda_zero_recovers_spline():
    P, q = 2, 3
    intervals = [4, 3]
    x = RNG.random((4000, P))
    a_true = RNG.standard_normal(spline.coef_count(intervals, q))
    Phi = spline.phi_matrix(x, [0.0] * P, [1.0] * P, intervals, q)
    y = Phi @ a_true
    A, b, _, _ = spline.system(x, y, [0.0] * P, [1.0] * P, intervals, q, 0.0)
    np.testing.assert_allclose(mgcg.solve_direct(A, b), a_true, atol=1e-8)


# ------------------------------------------------------------------ MGCG

def _pr1_like(n=2000, seed=7):
    r = np.random.default_rng(seed)
    x = r.random((n, 2))
    y = np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1]) + 0.1 * r.standard_normal(n)
    return x, y


def test_mgcg_converges_to_direct():
    x, y = _pr1_like()
    H = mgcg.build_hierarchy(x, y, [0.0, 0.0], [1.0, 1.0], [16, 16], 3, 1e-3, 3)
    res = mgcg.mgcg(H, 1e-13)
    a = mgcg.solve_direct(H.levels[-1].A, H.b)
    assert res.rel_res <= 1e-13
    np.testing.assert_allclose(res.alpha, a, rtol=0, atol=1e-9 * np.abs(a).max())


def test_v_cycle_is_symmetric_positive_definite():
    x, y = _pr1_like(800)
    H = mgcg.build_hierarchy(x, y, [0.0, 0.0], [1.0, 1.0], [8, 8], 3, 1e-2, 3)
    K = H.levels[-1].A.shape[0]
    M = np.stack([mgcg.v_cycle(H, 3, e, 1, 1) for e in np.eye(K)], axis=1)
    np.testing.assert_allclose(M, M.T, atol=1e-10 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_galerkin_and_rediscretised_hierarchies_agree():
    x, y = _pr1_like(1500)
    args = (x, y, [0.0, 0.0], [1.0, 1.0], [16, 16], 3, 1e-3, 3)
    H1 = mgcg.build_hierarchy(*args, omega=0.3)
    H2 = mgcg.build_hierarchy(*args, omega=0.3, galerkin=True)
    r1, r2 = mgcg.mgcg(H1, 1e-10), mgcg.mgcg(H2, 1e-10)
    assert r1.iterations == r2.iterations
    np.testing.assert_allclose(r1.alpha, r2.alpha, atol=1e-8 * np.abs(r1.alpha).max())


def test_mesh_independent_iterations():
    """Section 4, Fig. 2: MGCG iteration counts stay nearly constant under
    refinement while plain CG counts grow."""
    r = np.random.default_rng(3)
    n = 20000
    x = r.random((n, 2))
    y = 1.0 / (1.0 + np.exp(-16 * (np.sum(x * x, 1) / 2 - 0.5))) + 0.1 * r.standard_normal(n)
    its, cgs = [], []
    for G in (4, 5, 6):
        H = mgcg.build_hierarchy(x, y, [0.0, 0.0], [1.0, 1.0], [2 ** G] * 2, 3, 0.1, G)
        its.append(mgcg.mgcg(H, 1e-6).iterations)
        cgs.append(mgcg.mgcg(H, 1e-6, precondition=False).iterations)
    assert max(its) <= min(its) + 3
    assert cgs[-1] > 3 * cgs[0]
    assert cgs[-1] > 4 * its[-1]


# ------------------------------------------------------------------ cells, keys

def test_cell_index_edges():
    N = 16
    x = np.array([0.0, 1.0, 0.5, 0.0625, np.nextafter(0.0625, 0.0), 1 - 1e-16, 0.999999])
    np.testing.assert_array_equal(spline.cell_index(x, 0.0, 1.0, N), [0, 15, 8, 1, 0, 15, 15])
    x32 = np.array([0.0, 1.0, 0.5, 0.0625, np.nextafter(np.float32(0.0625), np.float32(0))], dtype=np.float32)
    np.testing.assert_array_equal(spline.cell_index(x32, 0.0, 1.0, N), [0, 15, 8, 1, 0])


def test_morton_key_hand_example():
    # cells (2, 1) with 2 bits: bit 1 -> (1, 0), bit 0 -> (0, 1): key 0b1001 = 9
    assert spline.morton_key(np.array([[2, 1]]), 2)[0] == 9
    assert spline.morton_key(np.array([[3, 3, 3]]), 2)[0] == 63
    assert spline.morton_key(np.array([[1, 0, 0]]), 1)[0] == 4


def test_morton_blocks_contiguous():
    """After the stable sort, every aligned 2^s block of cells on every level is one run."""
    P, N = 3, 16
    x = RNG.random((5000, P))
    perm, key, cells = spline.sort_permutation(x, [0.0] * P, [1.0] * P, [N] * P)
    c = cells[perm]
    assert np.all(np.diff(key[perm].astype(np.int64)) >= 0)
    for s in range(0, 5):
        blk = c >> s
        ids = [tuple(r) for r in blk]
        seen, prev = set(), None
        for t in ids:
            if t != prev:
                assert t not in seen
                seen.add(t)
                prev = t
    # stability: equal keys keep the original order
    ks = key[perm]
    eq = ks[1:] == ks[:-1]
    assert np.all(perm[1:][eq] > perm[:-1][eq])


# ------------------------------------------------------------------ full-size helpers

def test_sampled_and_chunked_apply_match_assembled():
    P, q, lam = 3, 3, 1e-2
    intervals = [4, 8, 4]
    lo, hi = [0.0] * 3, [1.0] * 3
    x = RNG.random((3000, P)); y = RNG.standard_normal(3000)
    A, b, Phi, Lam = spline.system(x, y, lo, hi, intervals, q, lam)
    v = RNG.standard_normal(A.shape[0])
    ks = RNG.choice(A.shape[0], 40, replace=False)
    np.testing.assert_allclose(sampled.apply_rows(x, v, ks, lo, hi, intervals, q, lam), (A @ v)[ks], rtol=1e-12,
                               atol=1e-12 * np.abs(A @ v).max())
    np.testing.assert_allclose(sampled.apply_phitphi_chunked(x, v, lo, hi, intervals, q, chunk=700),
                               Phi.T @ (Phi @ v), rtol=1e-12, atol=1e-12 * np.abs(A @ v).max())
    np.testing.assert_allclose(sampled.rhs_chunked(x, y, lo, hi, intervals, q, chunk=700), b, atol=1e-11)
    np.testing.assert_allclose(sampled.penalty_apply_kron(v, lo, hi, intervals, q), Lam @ v,
                               atol=1e-12 * np.abs(Lam @ v).max())
    alpha = mgcg.solve_direct(A, b)
    assert sampled.residual_norm(x, y, alpha, lo, hi, intervals, q, lam, chunk=900) < 1e-11


# ------------------------------------------------------------------ planted mistakes

def test_pins_catch_planted_mistakes(monkeypatch):
    """A wrong penalty weight or a transposed Kronecker order makes the pins fail."""
    good = spline.penalty_multiindices
    monkeypatch.setattr(spline, "penalty_multiindices", lambda P: [(r, 1.0) for r, _ in good(P)])
    with pytest.raises(AssertionError):
        test_penalty_is_thin_plate_energy(2)
    monkeypatch.setattr(spline, "penalty_multiindices", good)
    def first_fastest(J):              # column-major order instead of last-fastest
        s = [1] * len(J)
        for p in range(1, len(J)):
            s[p] = s[p - 1] * J[p - 1]
        return s
    monkeypatch.setattr(spline, "strides", first_fastest)
    with pytest.raises(AssertionError):
        test_phi_tensor_order_unequal_grids()


# ------------------------------------------------------------------ Jacobi spectrum, Lanczos branch

def _lmax_case(P, intervals, n, lam, seed):
    r = np.random.default_rng(seed)
    x = r.random((n, P))
    y = np.sin(3.0 * x[:, 0]) + 0.1 * r.standard_normal(n)
    A, _, _, _ = spline.system(x, y, [0.0] * P, [1.0] * P, intervals, 3, lam)
    return A


@pytest.mark.parametrize("P,intervals,n,lam", [(3, [8, 16, 8], 6007, 3e-3), (4, [4, 8, 4, 4], 4001, 1e-1)])
def test_lambda_max_jacobi_lanczos_branch(P, intervals, n, lam):
    """lambda_max(D^-1 A) by the oracle's Lanczos branch (K > 2000) against
    the dense symmetric eigensolver on D^-1/2 A D^-1/2, and two facts that hold
    for any SPD A: it is at least the largest Rayleigh quotient of D^-1 A over
    the unit vectors (which is 1) and at most the largest absolute row sum of
    D^-1 A (Gershgorin)."""
    A = _lmax_case(P, intervals, n, lam, seed=100 + P)
    K = A.shape[0]
    assert K > 2000          # the eigsh branch
    Dinv = 1.0 / A.diagonal()
    lm = mgcg.lambda_max_jacobi(A, Dinv)
    s = np.sqrt(Dinv)
    dense = np.linalg.eigvalsh(s[:, None] * A.toarray() * s[None, :])[-1]
    assert abs(lm - dense) <= 1e-9 * dense
    gersh = float(np.max(np.abs(A).sum(axis=1).A1 * Dinv))
    assert 1.0 <= lm <= gersh * (1 + 1e-12)
    # a planted mistake -- the spectrum of A instead of D^-1 A -- fails the first check
    wrong = float(spla.eigsh(A, k=1, which="LA", return_eigenvectors=False, tol=1e-10)[0])
    assert abs(wrong - dense) > 1e-3 * dense


# ------------------------------------------------------------------ tier-2 oracle (assembled MG-PCG)

def test_tier2_mgcg_matches_direct_on_clustered_cut():
    """The assembled Galerkin MG-PCG used for the large workloads (Algorithm 8
    with Galerkin coarse operators I' A I) reaches the direct solve on a cut of
    the clustered P = 3 workload: 2e4 of its points on 16^3 intervals (K =
    6859), 4 levels."""
    import workloads as W
    pr = W.scale(n=20000)
    res = mgcg.solve_tier2(pr.x, pr.y, pr.lo, pr.hi, [16, 16, 16], 3, pr.lam, 4, tol=1e-13)
    A, b, _, _ = spline.system(pr.x, pr.y, pr.lo, pr.hi, [16, 16, 16], 3, pr.lam)
    ref = mgcg.solve_direct(A, b)
    assert res.rel_res <= 1e-13
    assert np.linalg.norm(b - A @ res.alpha) / np.linalg.norm(b) <= 2e-13
    assert np.max(np.abs(res.alpha - ref)) <= 1e-8 * np.max(np.abs(ref))
