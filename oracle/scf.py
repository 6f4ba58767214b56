"""Self-consistent linear response and its mixers (oracle; test
infrastructure only).

The self-consistent response of the Appendix (Eq. DM_CP_SCF, and its dual
Eq. CP_SCF) replaces H1 by H1 + G(D1). The workload takes G from
site charges: a site-diagonal perturbation with potential u_a on every
orbital of site a gives site charges q_a = sum_{mu in a} D1_{mu mu}; the
induced potential is K q. So one response evaluation is the linear map
    q_out(q_in) = chi0 (V_ext + K q_in),
with chi0 the site-resolved static response (chi0_ab = d q_a / d u_b),
and the self-consistent solution is q* = (I - chi0 K)^(-1) chi0 V_ext.

Mixers (the paper uses linear mixing with a constant c_mix and mentions
more advanced SCF acceleration; Eq. CP_SCF):
  linear:   q <- q + alpha (q_out - q)
  Anderson: q <- sum_i c_i (q_i + alpha r_i), c minimising ||sum_i c_i r_i||
            with sum_i c_i = 1 over the last m iterates (r = q_out - q), from
            the KKT system [G 1; 1^T 0] with G_ij = <r_i, r_j> shifted by
            1e-12 of its mean diagonal (rank-deficient histories).
The learned preconditioner is a 2-layer MLP without biases,
y = W2 relu(W1 x), applied as a correction to linear mixing,
q <- q + alpha r + ||r|| MLP(r / ||r||) (the map is positively homogeneous,
so this equals q + alpha r + MLP(r)); trained on (r_i / ||r_i||,
(q* - q_i - alpha r_i) / ||r_i||) pairs it learns the slow modes that linear
mixing leaves, and an untrained (zero) MLP is plain linear mixing.
anderson_mlp: Anderson with that learned step as its preconditioner,
q <- sum_i c_i (q_i + P(r_i)), P(r) = alpha r + ||r|| MLP(r / ||r||), the c_i as
for Anderson; a zero network gives Anderson, a history of one the MLP mixer.
"""
from __future__ import annotations

import numpy as np

from . import exact


def chi0_sites(e: np.ndarray, V: np.ndarray, nocc: int, norb: int) -> np.ndarray:
    """chi0_ab = d q_a / d u_b by Daleckii-Krein, one site-diagonal
    perturbation per column (zero temperature)."""
    n = V.shape[0]
    ns = n // norb
    f = exact.occupations_zero_T(e, nocc)
    L = exact.loewner(e, f)
    out = np.zeros((ns, ns))
    for b in range(ns):
        P = np.zeros(n)
        P[b * norb:(b + 1) * norb] = 1.0
        D1 = V @ (L * ((V.T * P[None, :]) @ V)) @ V.T
        out[:, b] = np.diag(D1).reshape(ns, norb).sum(axis=1)
    return out


def chi0_sites_fermi(e: np.ndarray, V: np.ndarray, mu: float, kT: float, norb: int,
                     canonical: bool = True) -> np.ndarray:
    """Finite-temperature chi0_ab = d q_a / d u_b (Sec. V.B): the Daleckii-Krein
    response of the Fermi function to each site-diagonal perturbation, with
    the canonical mu_1 (Tr[D1] = 0) when asked, then summed over site a."""
    n = V.shape[0]
    ns = n // norb
    out = np.zeros((ns, ns))
    for b in range(ns):
        P = np.zeros(n)
        P[b * norb:(b + 1) * norb] = 1.0
        D1 = exact.response_fermi(e, V, mu, kT, np.diag(P), canonical=canonical)
        out[:, b] = np.diag(D1).reshape(ns, norb).sum(axis=1)
    return out


def scf_exact(chi0: np.ndarray, K: np.ndarray, Vext: np.ndarray) -> np.ndarray:
    """q* = (I - chi0 K)^(-1) chi0 V_ext for every field (rows of Vext)."""
    ns = chi0.shape[0]
    rhs = (chi0 @ Vext.T)
    return np.linalg.solve(np.eye(ns) - chi0 @ K, rhs).T


def scf_iterate(chi0, K, Vext, mixer="linear", alpha=0.3, hist=8, tol=1e-6, max_iter=200,
                mlp=None):
    """Plain SCF iterations on the exact linear response map. Returns
    (q, residual history) with residual ||q_out - q||_2 / ||q_out(0)||_2 over
    all fields."""
    q = np.zeros_like(Vext)
    res = []
    norm0 = None
    qs, rs, ps = [], [], []     # iterates, residuals and preconditioned steps of the history
    for it in range(max_iter):
        qout = (chi0 @ (Vext + q @ K.T).T).T
        r = qout - q
        if norm0 is None:
            norm0 = np.linalg.norm(qout)
        res.append(np.linalg.norm(r) / norm0)
        if res[-1] <= tol:
            break
        if mixer == "linear":
            q = q + alpha * r
        elif mixer in ("anderson", "anderson_mlp"):
            qs.append(q.copy())
            rs.append(r.copy())
            if mixer == "anderson":
                ps.append(alpha * r)
            else:
                W1, W2 = mlp
                nr = np.linalg.norm(r, axis=1, keepdims=True)
                x = r / np.where(nr > 0, nr, 1.0)
                ps.append(alpha * r + nr * mlp_forward(W1, W2, x))
            qs, rs, ps = qs[-hist:], rs[-hist:], ps[-hist:]
            new = np.zeros_like(q)
            for f in range(q.shape[0]):
                R = np.stack([x[f] for x in rs])          # m x ns
                m = R.shape[0]
                G = R @ R.T
                scale = np.trace(G) / m
                scale = scale if scale > 0 else 1.0
                A = np.zeros((m + 1, m + 1))
                A[:m, :m] = G / scale + 1e-12 * np.eye(m)
                A[m, :m] = A[:m, m] = 1.0
                rhs = np.zeros(m + 1)
                rhs[m] = 1.0
                c = np.linalg.solve(A, rhs)[:m]
                new[f] = sum(c[i] * (qs[i][f] + ps[i][f]) for i in range(m))
            q = new
        elif mixer == "mlp":
            W1, W2 = mlp
            nr = np.linalg.norm(r, axis=1, keepdims=True)
            x = r / np.where(nr > 0, nr, 1.0)
            q = q + alpha * r + nr * mlp_forward(W1, W2, x)
        else:
            raise ValueError(mixer)
    return q, res


# ------------------------------------------------------------------ MLP
def mlp_forward(W1: np.ndarray, W2: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y = relu(X W1^T) W2^T for a batch X (P x d_in); W1: d_h x d_in, W2: d_in x d_h."""
    return np.maximum(X @ W1.T, 0.0) @ W2.T


def mlp_loss_grad(W1, W2, X, T):
    """Mean squared error over the batch, L = sum (Y - T)^2 / P, and its
    gradients (backpropagation through y = W2 relu(W1 x))."""
    P = X.shape[0]
    Hp = X @ W1.T
    Hr = np.maximum(Hp, 0.0)
    Y = Hr @ W2.T
    E = Y - T
    L = float(np.sum(E * E)) / P
    dY = 2.0 * E / P
    dW2 = dY.T @ Hr
    dH = (dY @ W2) * (Hp > 0)
    dW1 = dH.T @ X
    return L, dW1, dW2


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), returning the new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
