"""Plain FP64 SP2 recursions (oracle; test infrastructure only).

Everything here is numpy FP64 with ``@`` (dgemm) as the only library
primitive. No blocking, fusion or reordering beyond what the equations state.

Notation follows the paper (arXiv 2409.17033):
  X_1 = alpha I + beta H                      (Eq. DM0, Sec. II)
  X_{n+1} = (1 - sigma_n) X_n + sigma_n X_n^2  (Eq. DM0)
  Y_1 = beta H1;  Y_{n+1} = (1 - sigma_n) Y_n + sigma_n (Y_n X_n + X_n Y_n)   (Eq. DM1)
  backward: Y_M = A;  Y_{n-1} = (1 - sigma_n) Y_n + sigma_n (Y_n X_n + X_n Y_n), n = M..1;
            chi = beta Y_0                    (Eq. DM2)
  forward:  Y_1 = beta A, same recursion as Eq. DM1, chi = Y_{M+1}   (Eq. DM3)

Readings where the paper is silent (the same readings the CUDA path takes):
  * spectral bounds: Gershgorin discs (the paper only asks for "estimates" of
    the extreme eigenvalues, Sec. II);
  * branch choice: sigma = +1 (square) when |Tr[X^2] - N_occ| <= |Tr[2X - X^2] - N_occ|,
    ties go to squaring; Tr[X^2] is ||X||_F^2 for symmetric X (Sec. II asks
    for the trace of X_{n+1} closest to N_occ);
  * stopping: two idempotency errors are tracked, the trace form
    e_n = Tr[X_n] - ||X_n||_F^2 (sum of lambda (1 - lambda)) and the squared
    Frobenius form f_n = ||X_n - X_n^2||_F^2 (sum of lambda^2 (1 - lambda)^2),
    f_n being known once step n has formed X_n^2. After step n >= min_iter
    stop when |e_{n+1}| <= idem_tol (tolerance test), or when n >= 3, the
    two steps n-2, n-1 took opposite branches, f_{n-2} <= floor_gate and
    f_n >= f_{n-2}, or when the smallest f so far is <= floor_gate and none
    of the last STALL = 4 steps went below it (the precision floor).
    Why these mark a floor: a pair of opposite branches maps an eigenvalue
    at distance d from 0 or 1 to one at distance at most 4 d^2, so once every
    d < 1/4 (guaranteed by f <= 0.03 < (3/16)^2) f must fall over such a
    pair in exact arithmetic, and over any four steps it reaches a new
    minimum; a rise or a stall is rounding. Pairs of equal branches alone
    are not tested: they double d on one side, so f may rise legitimately.
    The test uses f, not e: with split low-precision products e carries a
    systematic trace bias of order N times the unit roundoff that can
    exceed the true error of the slow near-gap eigenvalues, whereas f
    weights every eigenvalue by its squared error. ``max_iter`` steps
    without any test firing is non-convergence.
  * result at the floor: when a floor test fires, the result is the iterate
    X_{n*} with the smallest f among those with f <= floor_gate (n* >= 2),
    i.e. M = n* - 1 steps, not the last one formed. Past the floor, rounding
    makes f cycle (it grows about fourfold per 2X - X^2 step until a squaring
    resets it), and the response's near-gap terms follow that cycle: the
    error of chi against the exact form tracks sqrt(f) of the returned
    iterate. The tolerance test returns the last iterate as before.
"""
from __future__ import annotations

import dataclasses

import numpy as np


STALL = 4  # steps without a new minimum of f that mark the precision floor


# ---------------------------------------------------------------- Sec. II
def gershgorin_bounds(H: np.ndarray) -> tuple[float, float]:
    """Lower and upper spectral bound estimates of symmetric H (Sec. II:
    eps_min, eps_max), read as Gershgorin discs: H_ii -/+ sum_{j != i} |H_ij|."""
    H = np.asarray(H, dtype=np.float64)
    d = np.diag(H)
    r = np.abs(H).sum(axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def sp2_scaling(eps_min: float, eps_max: float) -> tuple[float, float]:
    """alpha = eps_max / (eps_max - eps_min), beta = -1 / (eps_max - eps_min)
    (Sec. II, after Eq. DM0): maps the spectrum in reversed order onto [0, 1].
    A point spectrum (eps_min == eps_max, e.g. H = c I or N = 1) has no width
    to divide by; any interval around it does, and [eps - 1/2, eps + 1/2] is
    the one taken (X_1 = I/2)."""
    if not eps_max > eps_min:
        eps_min, eps_max = eps_min - 0.5, eps_max + 0.5
    w = eps_max - eps_min
    return eps_max / w, -1.0 / w


def choose_sigma(t1: float, t2: float, nocc: float) -> int:
    """Branch choice of Eq. DM0: trace after squaring is t2 = Tr[X^2], after
    2X - X^2 it is 2 t1 - t2; pick the one closer to N_occ (ties: square)."""
    return 1 if abs(t2 - nocc) <= abs(2.0 * t1 - t2 - nocc) else -1


def traces(X: np.ndarray) -> tuple[float, float]:
    """(Tr[X], Tr[X^2]) with Tr[X^2] written as sum_ij X_ij X_ji."""
    return float(np.trace(X)), float(np.sum(X * X.T))


def idem_fro(X: np.ndarray, X2: np.ndarray) -> float:
    """f = ||X - X^2||_F^2 given X and its square."""
    d = X - X2
    return float(np.sum(d * d))


def stop_now(n: int, e: list[float], f: list[float], sig: list[int], idem_tol: float,
             floor_gate: float, min_iter: int) -> int:
    """Stopping reading (module docstring). ``e[k]`` is the trace error of
    X_{k+1} (after step n the newest is e[n], of X_{n+1}); ``f[k]`` is the
    squared Frobenius error of X_{k+1} (after step n the newest is f[n-1], of
    X_n); ``sig[k]`` is sigma_{k+1}. Returns 0 (go on), 1 (tolerance test) or
    2 (a precision-floor test)."""
    if n < min_iter:
        return 0
    if idem_tol > 0.0 and abs(e[n]) <= idem_tol:
        return 1
    if floor_gate <= 0.0:
        return 0
    if n >= 3 and sig[n - 3] != sig[n - 2] and f[n - 3] <= floor_gate and f[n - 1] >= f[n - 3]:
        return 2
    if n > STALL:
        best = min(f[:n - STALL])
        if best <= floor_gate and min(f[n - STALL:n]) >= best:
            return 2
    return 0


def floor_best(f: list[float], floor_gate: float) -> int:
    """n* = the index (1-based, >= 2) of the iterate X_{n*} with the smallest f
    among those with f <= floor_gate, from f[k] = f of X_{k+1}; 0 if none."""
    best, nb = None, 0
    for k in range(1, len(f)):
        if f[k] <= floor_gate and (best is None or f[k] < best):
            best, nb = f[k], k + 1
    return nb


@dataclasses.dataclass
class SP2Result:
    D: np.ndarray                 # X_{M+1}
    alpha: float
    beta: float
    sigma: list[int]              # sigma_1..sigma_M
    errors: list[float]           # e for X_1..X_{M+1}
    fro: list[float]              # f for X_1..X_M
    X: list[np.ndarray] | None    # X_1..X_M (inputs of each step) when kept
    converged: bool
    stop_step: int = 0            # the step after which a stop test fired (>= M)

    @property
    def M(self) -> int:
        return len(self.sigma)


def sp2_density(H: np.ndarray, nocc: float, idem_tol: float = 1e-10,
                max_iter: int = 100, min_iter: int = 4, floor_gate: float = 0.03,
                sigma: list[int] | None = None, keep: bool = False,
                bounds: tuple[float, float] | None = None) -> SP2Result:
    """SP2 recursive Fermi-operator expansion, Eq. DM0.

    If ``sigma`` is given, exactly those branches are taken (M = len(sigma))
    and no stopping test is made; otherwise sigma_n comes from
    ``choose_sigma`` and the stopping reading of the module docstring."""
    H = np.asarray(H, dtype=np.float64)
    n_ = H.shape[0]
    emin, emax = gershgorin_bounds(H) if bounds is None else bounds
    alpha, beta = sp2_scaling(emin, emax)
    X = alpha * np.eye(n_) + beta * H
    t1, t2 = traces(X)
    errs = [t1 - t2]
    fro: list[float] = []
    sig: list[int] = []
    hist: list[np.ndarray] | None = [] if keep else None
    converged = False
    steps = len(sigma) if sigma is not None else max_iter
    kept: dict[int, np.ndarray] = {}          # X_n of the floor candidates
    for n in range(1, steps + 1):
        s = sigma[n - 1] if sigma is not None else choose_sigma(t1, t2, nocc)
        if keep:
            hist.append(X)
        X2 = X @ X
        fro.append(idem_fro(X, X2))
        if sigma is None and fro[-1] <= floor_gate:
            kept[n] = X
        X = X2 if s > 0 else 2.0 * X - X2
        sig.append(int(s))
        t1, t2 = traces(X)
        errs.append(t1 - t2)
        why = stop_now(n, errs, fro, sig, idem_tol, floor_gate, min_iter) if sigma is None else 0
        if why:
            converged = True
            nb = floor_best(fro, floor_gate) if why == 2 else 0
            if nb >= 2 and nb - 1 < n:
                m = nb - 1                       # return X_{n*}: M = n* - 1 steps
                X = kept[nb]
                sig, errs, fro = sig[:m], errs[:m + 1], fro[:m]
                if keep:
                    hist = hist[:m]
            break
    if sigma is not None:
        converged = True
    return SP2Result(D=X, alpha=alpha, beta=beta, sigma=sig, errors=errs, fro=fro,
                     X=hist, converged=converged, stop_step=n if steps > 0 else 0)


# ---------------------------------------------------------------- Sec. III
def _response_step(Y: np.ndarray, X: np.ndarray, s: int) -> np.ndarray:
    """(1 - sigma) Y + sigma (Y X + X Y): the update shared by Eqs. DM1-DM3."""
    P = Y @ X + X @ Y
    return P if s > 0 else 2.0 * Y - P


def dm_response(X_hist: list[np.ndarray], sigma: list[int], beta: float,
                H1: np.ndarray) -> np.ndarray:
    """First-order density-matrix response D^(1), Eq. DM1, over the stored
    X_1..X_M of the ground-state run."""
    Y = beta * np.asarray(H1, dtype=np.float64)
    for X, s in zip(X_hist, sigma):
        Y = _response_step(Y, X, s)
    return Y


# ---------------------------------------------------------------- Sec. IV
def susceptibility_backward(X_hist: list[np.ndarray], sigma: list[int],
                            beta: float, A: np.ndarray) -> np.ndarray:
    """Backward (adjoint) susceptibility, Eq. DM2: start from A at n = M and
    run the response update against X_M, X_{M-1}, ..., X_1; chi = beta Y_0."""
    Y = np.asarray(A, dtype=np.float64)
    for X, s in zip(reversed(X_hist), reversed(sigma)):
        Y = _response_step(Y, X, s)
    return beta * Y


def susceptibility_forward(X_hist: list[np.ndarray], sigma: list[int],
                           beta: float, A: np.ndarray) -> np.ndarray:
    """Forward susceptibility, Eq. DM3: Eq. DM1 with A in place of H1."""
    return dm_response(X_hist, sigma, beta, A)


# ---------------------------------------------------------------- Appendix
def merged_response(H: np.ndarray, nocc: float, B: np.ndarray, **kw):
    """Merged forms of the Appendix (Eq. DMSuscept with B = A, Eq. DMPert with
    B = H1): the response Y runs beside X in one loop, so no X_n is stored.
    B may be one matrix or a stack (B_k). Returns (SP2Result, Y_{M+1}).
    The branch sequence and M are the ones the ground-state loop takes."""
    H = np.asarray(H, dtype=np.float64)
    n_ = H.shape[0]
    Bs = np.asarray(B, dtype=np.float64)
    single = Bs.ndim == 2
    if single:
        Bs = Bs[None]
    idem_tol = kw.get("idem_tol", 1e-10)
    max_iter = kw.get("max_iter", 100)
    min_iter = kw.get("min_iter", 4)
    floor_gate = kw.get("floor_gate", 0.03)
    sigma = kw.get("sigma")
    emin, emax = kw.get("bounds") or gershgorin_bounds(H)
    alpha, beta = sp2_scaling(emin, emax)
    X = alpha * np.eye(n_) + beta * H
    Y = [beta * b for b in Bs]
    t1, t2 = traces(X)
    errs = [t1 - t2]
    fro: list[float] = []
    sig: list[int] = []
    converged = sigma is not None
    steps = len(sigma) if sigma is not None else max_iter
    kept: dict[int, tuple] = {}              # (X_n, Y_n) of the floor candidates
    for n in range(1, steps + 1):
        s = sigma[n - 1] if sigma is not None else choose_sigma(t1, t2, nocc)
        Yn = Y
        Y = [_response_step(y, X, s) for y in Y]
        X2 = X @ X
        fro.append(idem_fro(X, X2))
        if sigma is None and fro[-1] <= floor_gate:
            kept[n] = (X, Yn)
        X = X2 if s > 0 else 2.0 * X - X2
        sig.append(int(s))
        t1, t2 = traces(X)
        errs.append(t1 - t2)
        why = stop_now(n, errs, fro, sig, idem_tol, floor_gate, min_iter) if sigma is None else 0
        if why:
            converged = True
            nb = floor_best(fro, floor_gate) if why == 2 else 0
            if nb >= 2 and nb - 1 < n:
                m = nb - 1
                X, Y = kept[nb]
                sig, errs, fro = sig[:m], errs[:m + 1], fro[:m]
            break
    res = SP2Result(D=X, alpha=alpha, beta=beta, sigma=sig, errors=errs, fro=fro,
                    X=None, converged=converged)
    Yo = np.stack(Y)
    return res, (Yo[0] if single else Yo)


# ---------------------------------------------------------------- contractions
def trace_product(P: np.ndarray, Q: np.ndarray) -> float:
    """Tr[P Q] = sum_ij P_ij Q_ji (Eqs. expectation, direct, dual)."""
    return float(np.sum(np.asarray(P, np.float64) * np.asarray(Q, np.float64).T))


def contract(Ps: np.ndarray, Qs: np.ndarray) -> np.ndarray:
    """Matrix of responses out[l, k] = Tr[P_l Q_k] for stacks P (L,N,N) and
    Q (K,N,N): a^(1) = Tr[chi^A_l H1_k] (Eq. dual) or Tr[A_l D1_k] (Eq. direct)."""
    Ps = np.asarray(Ps, np.float64)
    Qs = np.asarray(Qs, np.float64)
    out = np.empty((Ps.shape[0], Qs.shape[0]))
    for l in range(Ps.shape[0]):
        for k in range(Qs.shape[0]):
            out[l, k] = trace_product(Ps[l], Qs[k])
    return out


def contract_diag(Ps: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Same as ``contract`` for diagonal Q_k = diag(q_k): sum_i P_l,ii q_k,i."""
    Ps = np.asarray(Ps, np.float64)
    q = np.asarray(q, np.float64)
    dg = np.stack([np.diag(p) for p in Ps])
    return dg @ q.T
