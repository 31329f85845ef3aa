"""Table 3 / Fig. 3 of the paper: the spectrum of A_G and of the
multigrid-preconditioned C_MG A_G at P = 2, G = 5 (K = 1225), assembled from
the GPU's operator apply and V-cycle, against the oracle's assembled matrices
and V-cycle with the same damping."""
import numpy as np
import pytest

import workloads as W
from oracle import mgcg, spline
from tests.gpu_util import oracle_hierarchy

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_1901_00654_gb300.binding")
analysis = pytest.importorskip("paper_1901_00654_gb300.analysis")


def test_spectrum_matches_oracle():
    P, G, lam = 2, 5, 0.1
    x, y = W.paper_sigmoid(5, 100_000, P)
    lo, hi = [0.0] * P, [1.0] * P
    with B.Plan(P, [32, 32], G, lam) as pl:
        pl.set_points(x, y)
        A, M = analysis.operator_matrices(pl, G)
        om = B.sps_get_omega(pl.h, G)
    gpu = analysis.spectra(A, M)
    # oracle: assembled A_G and its V-cycle on every unit vector, same omega
    Ao, _, _, _ = spline.system(x, y, lo, hi, [32, 32], 3, lam)
    H = oracle_hierarchy(x, y, lo, hi, [32, 32], 3, lam, G, om)
    K = Ao.shape[0]
    Mo = np.zeros((K, K))
    for j in range(K):
        e = np.zeros(K)
        e[j] = 1.0
        Mo[:, j] = mgcg.v_cycle(H, G, e, 1, 1)
    ref = analysis.spectra(Ao.toarray(), Mo)
    assert abs(gpu["kappa_A"] / ref["kappa_A"] - 1) < 1e-8
    assert abs(gpu["kappa_MA"] / ref["kappa_MA"] - 1) < 1e-6
    # the V-cycle is symmetric positive definite (so PCG applies) and pushes the spectrum towards 1
    assert np.allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    assert gpu["eig_MA"][0] > 0 and gpu["kappa_MA"] < gpu["kappa_A"] / 100
