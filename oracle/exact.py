"""Closed forms the SP2 path approximates (oracle; test infrastructure only).

* Zero-temperature density matrix D = theta(mu I - H) (Sec. II, Eq. 1):
  with H = V diag(e) V^T, D = V_occ V_occ^T over the N_occ lowest states.
* First-order response by Daleckii-Krein (Appendix, proof of Eq. Equivalence):
  D1 = V (L o (V^T H1 V)) V^T with the Loewner matrix L_ij = f[e_i, e_j] of
  divided differences. The susceptibility is the same map applied to A
  (Eq. Suscept_Der), so chi^A = V (L o (V^T A V)) V^T.
* Finite-M reference: the SP2 recursion of Eq. DM0 acts on the eigenvalues
  of X_1 = alpha I + beta H one by one, x -> (1 - sigma) x + sigma x^2, and the
  response recursion of Eq. DM1 multiplies each eigenbasis entry (i, j) by the
  divided difference of that step's polynomial, (1 - sigma) + sigma (x_i + x_j)
  (chain rule for divided differences of a composition). For a given branch
  sequence this is the exact value of X_{M+1} and Y_{M+1} up to rounding.
* Fermi-Dirac occupations and their Loewner matrix (Sec. V.B) for the
  finite-temperature variant, with the canonical chemical-potential response
  mu_1 fixed by Tr[D1] = 0.
"""
from __future__ import annotations

import numpy as np


def eigh(H: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Eigenvalues (ascending) and orthonormal eigenvectors (LAPACK dsyevd)."""
    e, V = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    return e, V


def density_zero_T(e: np.ndarray, V: np.ndarray, nocc: int) -> np.ndarray:
    """D = theta(mu I - H) = sum over the nocc lowest states |v><v| (Eq. 1)."""
    order = np.argsort(e, kind="stable")
    Vo = V[:, order[:nocc]]
    return Vo @ Vo.T


def occupations_zero_T(e: np.ndarray, nocc: int) -> np.ndarray:
    """f_i in {0, 1}: 1 for the nocc lowest eigenvalues."""
    f = np.zeros_like(e)
    f[np.argsort(e, kind="stable")[:nocc]] = 1.0
    return f


def loewner(e: np.ndarray, f: np.ndarray, fprime: np.ndarray | None = None,
            degenerate: float = 1e-12) -> np.ndarray:
    """Loewner matrix of divided differences L_ij = (f_i - f_j) / (e_i - e_j),
    with L_ij = f'(e_i) (or 0 if fprime is None) where |e_i - e_j| <= degenerate."""
    de = e[:, None] - e[None, :]
    df = f[:, None] - f[None, :]
    close = np.abs(de) <= degenerate
    L = np.where(close, 0.0, df / np.where(close, 1.0, de))
    if fprime is not None:
        fp = 0.5 * (fprime[:, None] + fprime[None, :])
        L = np.where(close, fp, L)
    return L


def daleckii_krein(V: np.ndarray, L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """V (L o (V^T B V)) V^T (Appendix, Daleckii-Krein formula)."""
    return V @ (L * (V.T @ np.asarray(B, np.float64) @ V)) @ V.T


def response_zero_T(e: np.ndarray, V: np.ndarray, nocc: int, B: np.ndarray) -> np.ndarray:
    """Exact zero-temperature first-order response to B (D1 for B = H1, chi^A
    for B = A): the sum-over-states form D1_ij (eigenbasis) = B_ij (f_i - f_j)/(e_i - e_j)."""
    f = occupations_zero_T(e, nocc)
    return daleckii_krein(V, loewner(e, f), B)


# ----------------------------------------------------- finite-M reference
def sp2_scalar(x: np.ndarray, sigma: list[int]) -> list[np.ndarray]:
    """The Eq. DM0 branch polynomials applied to each eigenvalue of X_1:
    returns [x^(1), ..., x^(M+1)]."""
    xs = [np.asarray(x, np.float64)]
    for s in sigma:
        y = xs[-1]
        xs.append(y * y if s > 0 else 2.0 * y - y * y)
    return xs


def sp2_divided_difference(xs: list[np.ndarray], sigma: list[int], beta: float) -> np.ndarray:
    """Eigenbasis multiplier of Eq. DM1 / DM3 after M steps:
    L_ij = beta * prod_n [(1 - sigma_n) + sigma_n (x_i^(n) + x_j^(n))]."""
    n = xs[0].shape[0]
    L = np.full((n, n), float(beta))
    for x, s in zip(xs[:-1], sigma):
        L = L * ((1.0 - s) + s * (x[:, None] + x[None, :]))
    return L


def finite_m_reference(e: np.ndarray, V: np.ndarray, alpha: float, beta: float,
                       sigma: list[int], Bs: np.ndarray | None = None):
    """Exact X_{M+1} (and Y_{M+1} for each B in Bs) for a given branch sequence.
    Returns (D_M, [Y_M(B) ...])."""
    x1 = alpha + beta * np.asarray(e, np.float64)
    xs = sp2_scalar(x1, sigma)
    D = (V * xs[-1][None, :]) @ V.T
    if Bs is None:
        return D, []
    L = sp2_divided_difference(xs, sigma, beta)
    Bs = np.asarray(Bs, np.float64)
    if Bs.ndim == 2:
        Bs = Bs[None]
    return D, [daleckii_krein(V, L, b) for b in Bs]


# ----------------------------------------------------- finite temperature
def fermi(e: np.ndarray, mu: float, kT: float) -> np.ndarray:
    """f(e) = 1 / (exp((e - mu)/kT) + 1) (Sec. V.B)."""
    z = (np.asarray(e, np.float64) - mu) / kT
    return 0.5 * (1.0 - np.tanh(0.5 * z))


def fermi_prime(e: np.ndarray, mu: float, kT: float) -> np.ndarray:
    """df/de = -f (1 - f) / kT."""
    f = fermi(e, mu, kT)
    return -f * (1.0 - f) / kT


def response_fermi(e: np.ndarray, V: np.ndarray, mu: float, kT: float,
                   B: np.ndarray, canonical: bool = True) -> np.ndarray:
    """Finite-temperature first-order response d/dlambda f(H + lambda B) by
    Daleckii-Krein (Sec. V.B). canonical=True adds the chemical-potential
    response mu_1 chosen so that Tr[D1] = 0: D1 <- D1 - mu_1' V diag(f') V^T
    with mu_1' = Tr[D1_gc] / sum_i f'(e_i)."""
    f = fermi(e, mu, kT)
    fp = fermi_prime(e, mu, kT)
    L = loewner(e, f, fp)
    D1 = daleckii_krein(V, L, B)
    if canonical:
        s = float(np.sum(fp))
        if s != 0.0:
            shift = float(np.trace(D1)) / s
            D1 = D1 - shift * (V * fp[None, :]) @ V.T
    return D1
