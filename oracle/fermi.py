"""Finite-temperature density matrix and its first-order responses by a
recursive Fermi-operator expansion (oracle; test infrastructure only).

Sec. V.B replaces theta(mu I - H) by the Fermi function
    f(H) = (exp(beta (H - mu I)) + I)^(-1),   beta = 1/kT,
and obtains the canonical susceptibility as the response to A with the
chemical-potential response mu_1 chosen so that Tr[chi] = 0 (the same rule
as in Eq. CP_SCF). The paper cites, but does not print, the recursion; the
reading taken here is the odds-squaring recursion of the Fermi function,
f(2x) = f(x)^2 / (f(x)^2 + (1 - f(x))^2), started from the first-order
expansion at x / 2^n. Written for delta = f - 1/2 (= -tanh(x/2)/2) it reads

    delta_0     = -(beta / 2^(n+2)) (H - mu I)
    delta_{j+1} = 2 delta_j (I + 4 delta_j^2)^(-1)          (j = 0 .. n-1)
    D           = I/2 + delta_n,

which is the same map (tanh doubling) but keeps the small deviations from 1/2
at full relative precision. Its first-order response to a perturbation B is
the chain rule of each step, with W_j = (I + 4 delta_j^2)^(-1):

    d delta_0     = -(beta / 2^(n+2)) B
    dW_j          = -4 W_j (d delta_j delta_j + delta_j d delta_j) W_j
    d delta_{j+1} = 2 (d delta_j W_j + delta_j dW_j).

On one eigenvalue the recursion is delta_n = -tanh(2^n artanh(x / 2^(n+1))) / 2
with x = beta (e - mu), which tends to the exact Fermi function as n grows
(log-odds error 2 (x/2)^3 / (3 4^n) to leading order).
"""
from __future__ import annotations

import numpy as np

from . import exact


def fermi_recursion(H: np.ndarray, mu: float, kT: float, n: int, Bs=None,
                    canonical: bool = True):
    """Matrix recursion in FP64 (inverse by LAPACK solve). Returns (D, [D1_k])
    for the perturbations in Bs (a matrix or a stack)."""
    H = np.asarray(H, np.float64)
    N = H.shape[0]
    beta = 1.0 / kT
    c = beta / 2.0 ** (n + 2)
    I = np.eye(N)
    delta = -c * (H - mu * I)
    resp = []
    if Bs is not None:
        Bs = np.asarray(Bs, np.float64)
        if Bs.ndim == 2:
            Bs = Bs[None]
        resp = [-c * b for b in Bs]
    ident = -c * I if (canonical and Bs is not None) else None
    for _ in range(n):
        W = np.linalg.solve(I + 4.0 * delta @ delta, I)
        nd = []
        for d in resp + ([ident] if ident is not None else []):
            dW = -4.0 * W @ (d @ delta + delta @ d) @ W
            nd.append(2.0 * (d @ W + delta @ dW))
        if ident is not None:
            ident = nd[-1]
            nd = nd[:-1]
        resp = nd
        delta = 2.0 * delta @ W
    D = 0.5 * I + delta
    if ident is not None:
        # canonical: D1 <- D1 - (Tr D1 / Tr R_I) R_I, R_I the response to I (Tr D1 = 0)
        tr_i = float(np.trace(ident))
        resp = [d - (float(np.trace(d)) / tr_i) * ident for d in resp]
    return D, resp


# ---------------------------------------------------------- eigenvalue form
def scalar_deltas(x0: np.ndarray, n: int) -> list[np.ndarray]:
    """delta_0 .. delta_n on the eigenvalues: delta <- 2 delta / (1 + 4 delta^2)."""
    ds = [np.asarray(x0, np.float64)]
    for _ in range(n):
        d = ds[-1]
        ds.append(2.0 * d / (1.0 + 4.0 * d * d))
    return ds


def step_divided_difference(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Divided difference of phi(d) = 2 d / (1 + 4 d^2):
    (phi(a) - phi(b)) / (a - b) = 2 (1 - 4 a b) / ((1 + 4 a^2)(1 + 4 b^2)),
    which is also phi'(a) at a = b."""
    return 2.0 * (1.0 - 4.0 * a * b) / ((1.0 + 4.0 * a * a) * (1.0 + 4.0 * b * b))


def fermi_recursion_reference(e: np.ndarray, V: np.ndarray, mu: float, kT: float, n: int,
                              Bs=None, canonical: bool = True):
    """The same recursion carried out exactly on the eigenvalues: D_n =
    V diag(1/2 + delta_n) V^T and D1 = V (L o (V^T B V)) V^T with
    L_ij = -(beta / 2^(n+2)) prod_j phi[delta_j(e_i), delta_j(e_j)]."""
    beta = 1.0 / kT
    c = beta / 2.0 ** (n + 2)
    ds = scalar_deltas(-c * (np.asarray(e, np.float64) - mu), n)
    D = (V * (0.5 + ds[-1])[None, :]) @ V.T
    if Bs is None:
        return D, []
    L = np.full((len(e), len(e)), -c)
    for d in ds[:-1]:
        L = L * step_divided_difference(d[:, None], d[None, :])
    Bs = np.asarray(Bs, np.float64)
    if Bs.ndim == 2:
        Bs = Bs[None]
    out = [exact.daleckii_krein(V, L, b) for b in Bs]
    if canonical:
        gp = np.diag(L).copy()              # response to I in the eigenbasis: diag(L_ii)
        RI = (V * gp[None, :]) @ V.T
        tr_i = float(np.sum(gp))
        out = [d - (float(np.trace(d)) / tr_i) * RI for d in out]
    return D, out


def delta_closed_form(x: np.ndarray, n: int) -> np.ndarray:
    """delta_n on one eigenvalue x = beta (e - mu): -tanh(2^n artanh(x / 2^(n+1))) / 2."""
    return -0.5 * np.tanh(2.0 ** n * np.arctanh(np.asarray(x, np.float64) / 2.0 ** (n + 1)))
