"""Spectral analysis of the (preconditioned) system, as in Section 4 (Table 3,
Fig. 3): the matrix of A_G and of C_MG A_G is assembled column by column from
the library's own operator apply and V-cycle (one call per unit vector, on the
device), and its eigenvalues are computed on the host.  Only sensible for
small K_G (the paper uses P = 2, G = 5, K_G = 1225)."""
from __future__ import annotations

import numpy as np

from . import binding as B


def operator_matrices(plan, levels: int, prec: int = B.SPS_PREC_FP64):
    """(A, M): A[:, j] = A_G e_j and M[:, j] = V(e_j), the V-cycle of
    Algorithm 7 from zero on the unit vector e_j (C_MG,G e_j)."""
    import torch
    K = plan.coef_count(levels)
    A = torch.zeros((K, K), dtype=torch.float64, device="cuda")
    M = torch.zeros((K, K), dtype=torch.float64, device="cuda")
    e = torch.zeros(K, dtype=torch.float64, device="cuda")
    col = torch.zeros(K, dtype=torch.float64, device="cuda")
    for j in range(K):
        e.zero_()
        e[j] = 1.0
        B.sps_apply(plan.h, levels, prec, e, col)
        A[:, j] = col
        B.sps_vcycle(plan.h, prec, e, col)
        M[:, j] = col
    torch.cuda.synchronize()
    return A.cpu().numpy(), M.cpu().numpy()


def spectra(A: np.ndarray, M: np.ndarray) -> dict:
    """Eigenvalues of A (symmetric) and of M A (similar to the symmetric
    M^1/2 A M^1/2 when M is SPD, so real and positive), with condition numbers."""
    ea = np.linalg.eigvalsh(0.5 * (A + A.T))
    ema = np.sort(np.linalg.eigvals(M @ A).real)
    return {"eig_A": ea, "eig_MA": ema, "kappa_A": float(ea[-1] / ea[0]), "kappa_MA": float(ema[-1] / ema[0])}
