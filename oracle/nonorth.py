"""Non-orthonormal basis representations (Sec. V.A) -- oracle; test
infrastructure only.

With an overlap matrix S != I, matrices in the atomic-orbital representation
X and their orthonormalised forms X^perp are related by congruences with an
inverse factor Z of S (Z^T S Z = I):
    H^perp = Z^T H Z,   A^perp = Z^T A Z,   D = Z D^perp Z^T,
and D^perp = theta(mu I - H^perp) comes from the SP2 expansion (Eq. DM0).
The symmetric choice Z = S^(-1/2) is the Loewdin factor.

The derivative of a = Tr[A D] along a basis-set dependent perturbation tau
(Eq. NonOrthDer, with Z_tau = -(1/2) S^(-1) S_tau Z) is
    a_tau = Tr[A_tau D] + Tr[A^perp D^perp_tau]
            - 1/2 Tr[A S^(-1) S_tau D] - 1/2 Tr[A D S_tau S^(-1)],
and the dual form replaces Tr[A^perp D^perp_tau] by Tr[chi^(A^perp) H^perp_tau]
with H^perp_tau = Z_tau^T H Z + Z^T H_tau Z + Z^T H Z_tau. Moving every Z and
S^(-1) onto the tau-independent side gives three contractions per tau,
    a_tau = Tr[A_tau D] + Tr[W_H H_tau] + Tr[W_S S_tau],
    W_H = Z chi^perp Z^T,
    W_S = -1/2 (M + M^T) - 1/2 (P + P^T),
    M = S^(-1) H W_H,   P = S^(-1) A D,
so the whole family of perturbations costs O(N^2) each once W_H, W_S are known.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import exact


def lowdin(S: np.ndarray) -> np.ndarray:
    """Z = S^(-1/2) from the eigendecomposition of S (Loewdin)."""
    s, U = np.linalg.eigh(S)
    return (U * (1.0 / np.sqrt(s))[None, :]) @ U.T


def density_generalized(H: np.ndarray, S: np.ndarray, nocc: int) -> np.ndarray:
    """D = C_occ C_occ^T from the generalized eigenproblem H C = S C e (C^T S C = I),
    by LAPACK's generalized solver -- a path independent of Z."""
    e, C = scipy.linalg.eigh(H, S)
    Co = C[:, :nocc]
    return Co @ Co.T


def dual_weights(H: np.ndarray, S: np.ndarray, A: np.ndarray, nocc: int):
    """The steps of Sec. V.A in order: Z, H^perp, A^perp, D^perp and the
    susceptibility chi^(A^perp) (closed forms of Sec. II / the Appendix), D,
    then W_H and W_S of the three-contraction form. Returns (Z, D, W_H, W_S)."""
    Z = lowdin(S)
    Hp = Z.T @ H @ Z
    Ap = Z.T @ A @ Z
    e, V = exact.eigh(0.5 * (Hp + Hp.T))
    Dp = exact.density_zero_T(e, V, nocc)
    chip = exact.response_zero_T(e, V, nocc, 0.5 * (Ap + Ap.T))
    D = Z @ Dp @ Z.T
    Sinv = Z @ Z.T
    WH = Z @ chip @ Z.T
    M = Sinv @ H @ WH
    P = Sinv @ A @ D
    WS = -0.5 * (M + M.T) - 0.5 * (P + P.T)
    return Z, D, WH, WS


def derivative_dual(D, WH, WS, A_t, H_t, S_t) -> float:
    """a_tau = Tr[A_tau D] + Tr[W_H H_tau] + Tr[W_S S_tau] (all symmetric)."""
    return float(np.sum(A_t * D) + np.sum(WH * H_t) + np.sum(WS * S_t))
