"""Thresholded block-sparse SP2 (oracle; test infrastructure only).

Sec. II notes that the generalized matrix products of Eq. DM0 can be carried
out in numerically thresholded sparse matrix algebra, which gives linear
scaling for large non-metallic systems. The paper fixes no threshold rule;
the reading taken here (the same the CUDA path takes) is blockwise:

  * the matrix is cut into b x b blocks (the last block row/column ragged);
  * T_tau(X) sets to zero every off-diagonal block whose Frobenius norm is
    <= tau; diagonal blocks are always kept, so the trace is never touched
    (tau = 0 drops only blocks that are exactly zero, which changes nothing);
  * X~_1 = T_tau(alpha I + beta H);
  * step n: sigma_n from the traces of X~_n as in Eq. DM0, X^2 = X~_n X~_n,
    f_n = ||X~_n - X^2||_F^2, X'_{n+1} = X^2 or 2 X~_n - X^2, and
    X~_{n+1} = T_tau(X'_{n+1});
  * the trace error e_{n+1} = Tr X~_{n+1} - ||X~_{n+1}||_F^2 and the stopping
    and floor rules are those of the dense recursion (oracle.sp2), applied to
    the thresholded iterates, plus one floor test for the threshold's own
    floor: after two steps of opposite branches that start from
    f <= RATIO_GATE = 1e-4, f must have fallen by a factor of at least 600 in
    exact arithmetic (every eigenvalue is then within d <= 0.01 of 0 or 1 and
    the pair maps d to at most 4 d^2); when it fell by less than 2 the
    iterates sit on the floor that dropping blocks sets, where f only creeps
    down and the dense rules (a rise of f, or four steps without a new
    minimum) need not fire.

Only the values matter here: the products are plain dense numpy matmuls of
the thresholded iterates (zero blocks add exact zeros). Which blocks a
product can skip is the CUDA path's business.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .sp2 import choose_sigma, floor_best, gershgorin_bounds, idem_fro, sp2_scaling, stop_now, traces

RATIO_GATE = 1e-4   # f below which a pair of opposite steps must cut f at least 600-fold


def threshold_floor(n: int, f: list[float], sig: list[int]) -> bool:
    """The threshold-floor test (module docstring) after step n: f[k] is f of
    X~_{k+1} (newest f[n-1], of X~_n), sig[k] is sigma_{k+1}."""
    return (n >= 3 and sig[n - 3] != sig[n - 2] and f[n - 3] <= RATIO_GATE
            and f[n - 1] >= 0.5 * f[n - 3])


def block_norms(X: np.ndarray, b: int) -> np.ndarray:
    """Frobenius norm of every b x b block of X, shape (nb, nb), nb = ceil(N / b)."""
    n = X.shape[0]
    nb = (n + b - 1) // b
    out = np.zeros((nb, nb))
    for i in range(nb):
        for j in range(nb):
            blk = X[i * b:(i + 1) * b, j * b:(j + 1) * b]
            out[i, j] = np.sqrt(np.sum(blk * blk))
    return out


def threshold_blocks(X: np.ndarray, tau: float, b: int) -> tuple[np.ndarray, np.ndarray]:
    """T_tau(X) and its block mask (True where a block is kept)."""
    nrm = block_norms(X, b)
    nb = nrm.shape[0]
    keep = (nrm > tau) | np.eye(nb, dtype=bool)
    Y = X.copy()
    for i in range(nb):
        for j in range(nb):
            if not keep[i, j]:
                Y[i * b:(i + 1) * b, j * b:(j + 1) * b] = 0.0
    return Y, keep


@dataclasses.dataclass
class SparseSP2Result:
    D: np.ndarray                 # X~_{M+1} (or the floor-best iterate)
    alpha: float
    beta: float
    sigma: list[int]
    errors: list[float]           # e of X~_1..X~_{M+1}
    fro: list[float]              # f of X~_1..X~_M
    masks: list[np.ndarray]       # block masks of X~_1..X~_{M+1}
    norms: list[np.ndarray]       # block norms of X_1, X'_2, ..., X'_{M+1} (before T_tau)
    converged: bool

    @property
    def M(self) -> int:
        return len(self.sigma)


def sp2_density_thresholded(H: np.ndarray, nocc: float, tau: float, block: int = 256,
                            idem_tol: float = 1e-10, max_iter: int = 100, min_iter: int = 4,
                            floor_gate: float = 0.03,
                            sigma: list[int] | None = None) -> SparseSP2Result:
    """Eq. DM0 in thresholded block-sparse algebra (module docstring)."""
    H = np.asarray(H, dtype=np.float64)
    n_ = H.shape[0]
    emin, emax = gershgorin_bounds(H)
    alpha, beta = sp2_scaling(emin, emax)
    X1 = alpha * np.eye(n_) + beta * H
    norms = [block_norms(X1, block)]
    X, m = threshold_blocks(X1, tau, block)
    masks = [m]
    t1, t2 = traces(X)
    errs = [t1 - t2]
    fro: list[float] = []
    sig: list[int] = []
    kept: dict[int, tuple[np.ndarray, int]] = {}
    converged = False
    steps = len(sigma) if sigma is not None else max_iter
    for n in range(1, steps + 1):
        s = sigma[n - 1] if sigma is not None else choose_sigma(t1, t2, nocc)
        X2 = X @ X
        fro.append(idem_fro(X, X2))
        if sigma is None and fro[-1] <= floor_gate:
            kept[n] = (X, len(masks) - 1)
        Xn = X2 if s > 0 else 2.0 * X - X2
        sig.append(int(s))
        norms.append(block_norms(Xn, block))
        X, m = threshold_blocks(Xn, tau, block)
        masks.append(m)
        t1, t2 = traces(X)
        errs.append(t1 - t2)
        why = stop_now(n, errs, fro, sig, idem_tol, floor_gate, min_iter) if sigma is None else 0
        if not why and sigma is None and floor_gate > 0.0 and n >= min_iter and threshold_floor(n, fro, sig):
            why = 2
        if why:
            converged = True
            nb = floor_best(fro, floor_gate) if why == 2 else 0
            if nb >= 2 and nb - 1 < n:
                mm = nb - 1
                X, mi = kept[nb]
                sig, errs, fro = sig[:mm], errs[:mm + 1], fro[:mm]
                masks, norms = masks[:mi + 1], norms[:mi + 1]
            break
    if sigma is not None:
        converged = True
    return SparseSP2Result(D=X, alpha=alpha, beta=beta, sigma=sig, errors=errs, fro=fro,
                           masks=masks, norms=norms, converged=converged)


def block_fill(masks: list[np.ndarray]) -> float:
    """Mean fraction of the upper-triangle blocks (with the diagonal) that the
    products X~_n X~_n of steps 1..M can produce nonzero: block (I, J) is
    formed when some K has both (I, K) and (K, J) in X~_n's mask."""
    tot = 0.0
    for m in masks[:-1]:
        mi = m.astype(np.int64)
        reach = (mi @ mi) > 0
        nb = m.shape[0]
        tot += np.triu(reach).sum() / (nb * (nb + 1) / 2)
    return tot / max(1, len(masks) - 1)
