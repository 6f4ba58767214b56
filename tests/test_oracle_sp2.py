"""Pins for the FP64 oracle (CPU only).

Each test checks an oracle function against something other than itself: a
closed form, an invariant the paper states, brute force on a tiny input, or
a library routine that solves the same problem another way.
"""
import numpy as np
import pytest

import workloads
from oracle import exact, sp2


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------------ Sec. II
def test_gershgorin_encloses_spectrum():
    rng = np.random.default_rng(3)
    for n in (5, 17, 64):
        H = workloads.sym_gaussian(rng, n, 1.0) + np.diag(rng.uniform(-3, 3, n))
        lo, hi = sp2.gershgorin_bounds(H)
        ev = np.linalg.eigvalsh(H)
        assert lo <= ev[0] + 1e-12 and ev[-1] <= hi + 1e-12
    # diagonal matrix: the discs are points, the bounds are exact
    d = np.array([0.3, -2.0, 5.0, 1.0])
    assert sp2.gershgorin_bounds(np.diag(d)) == (-2.0, 5.0)


def test_scaling_maps_spectrum_reversed_onto_unit_interval():
    a, b = sp2.sp2_scaling(-2.0, 6.0)
    assert a + b * 6.0 == pytest.approx(0.0, abs=1e-15)    # eps_max -> 0
    assert a + b * -2.0 == pytest.approx(1.0, abs=1e-15)   # eps_min -> 1
    assert b < 0


def test_choose_sigma_brute_force():
    rng = np.random.default_rng(4)
    for _ in range(50):
        n = 7
        Q = workloads.haar_orthogonal(rng, n)
        x = rng.uniform(0, 1, n)
        X = (Q * x) @ Q.T
        nocc = int(rng.integers(1, n))
        t_sq = np.trace(X @ X)
        t_2x = np.trace(2 * X - X @ X)
        want = 1 if abs(t_sq - nocc) <= abs(t_2x - nocc) else -1
        t1, t2 = sp2.traces(X)
        assert sp2.choose_sigma(t1, t2, nocc) == want


def test_sp2_density_matches_eigen_projector(cfg1):
    p = cfg1
    r = sp2.sp2_density(p.H, p.nocc, idem_tol=1e-10)
    assert r.converged
    D_ex = exact.density_zero_T(p.e, p.Q, p.nocc)
    assert rel(r.D, D_ex) < 1e-11
    assert abs(np.trace(r.D) - p.nocc) < 1e-9
    assert rel(r.D @ r.D, r.D) < 1e-11
    # an occupied-projector mistake (alpha/beta sign) would give Tr = N - nocc
    assert r.M < 40


def test_sp2_finite_m_matches_scalar_recursion(cfg1):
    """For ANY branch sequence, X_{M+1} is the branch polynomial applied to the
    eigenvalues of X_1 (exact reference), converged or not."""
    p = cfg1
    r = sp2.sp2_density(p.H, p.nocc, idem_tol=1e-10)
    bounds = sp2.gershgorin_bounds(p.H)
    rng = np.random.default_rng(5)
    for m in (1, 2, 5, 9):
        sig = list(rng.choice([-1, 1], size=m))
        rr = sp2.sp2_density(p.H, p.nocc, sigma=sig)
        D_ref, _ = exact.finite_m_reference(p.e, p.Q, rr.alpha, rr.beta, sig)
        assert rel(rr.D, D_ref) < 1e-12
    rr = sp2.sp2_density(p.H, p.nocc, sigma=r.sigma, bounds=bounds)
    D_ref, _ = exact.finite_m_reference(p.e, p.Q, r.alpha, r.beta, r.sigma)
    assert rel(rr.D, D_ref) < 1e-12


def test_frobenius_idempotency_error_closed_form(cfg1):
    """f_n = ||X_n - X_n^2||_F^2 = sum_i x_i^2 (1 - x_i)^2 over the eigenvalues
    x_i of X_n (finite-M eigenvalue reference)."""
    p = cfg1
    r = sp2.sp2_density(p.H, p.nocc, idem_tol=1e-10)
    xs = exact.sp2_scalar(r.alpha + r.beta * p.e, r.sigma)
    for n in range(r.M):
        x = xs[n]
        ref = float(np.sum(x * x * (1 - x) ** 2))
        assert r.fro[n] == pytest.approx(ref, rel=1e-9, abs=1e-22)


def test_floor_rule_in_emulated_split_precision():
    """With X kept in FP32 and products in the split form of Eq. MixPrecMult,
    the floor test stops only after the slow near-gap eigenvalues have
    converged (f has fallen to the rounding floor, far below the gate) and
    the result matches the exact projector to the accuracy the split form
    allows at this gap (about 1.3e-4 here; the scaled gap is 4.5e-3)."""
    from oracle import split
    tb = workloads.tight_binding(512, seed=0)
    e, V = exact.eigh(tb.H)
    emin, emax = sp2.gershgorin_bounds(tb.H)
    a, b = sp2.sp2_scaling(emin, emax)
    X = (a * np.eye(512) + b * tb.H).astype(np.float32).astype(np.float64)
    fro, errs, sig = [], [sp2.traces(X)[0] - sp2.traces(X)[1]], []
    M = None
    for n in range(1, 100):
        t1, t2 = sp2.traces(X)
        s = sp2.choose_sigma(t1, t2, tb.nocc)
        sig.append(s)
        X2 = split.mixed_product(X, X, "bf16")
        fro.append(sp2.idem_fro(X, X2))
        X = (X2 if s > 0 else 2 * X - X2).astype(np.float32).astype(np.float64)
        t1, t2 = sp2.traces(X)
        errs.append(t1 - t2)
        if sp2.stop_now(n, errs, fro, sig, 0.0, 0.03, 4):
            M = n
            break
    assert M is not None
    assert min(fro) < 1e-7 and fro[M - 3] < 1e-6
    D = exact.density_zero_T(e, V, tb.nocc)
    assert np.linalg.norm(X - D) / np.linalg.norm(D) < 3e-4


def test_stop_rule_reaches_tolerance_and_floor(cfg1):
    p = cfg1
    r = sp2.sp2_density(p.H, p.nocc, idem_tol=1e-10)
    assert abs(r.errors[-1]) <= 1e-10
    assert all(abs(e) > 1e-10 for e in r.errors[4:-1])
    # floor-only (no tolerance): keeps going until the error stalls, and the
    # result is still the projector
    r2 = sp2.sp2_density(p.H, p.nocc, idem_tol=0.0)
    assert r2.converged and r2.M >= r.M
    assert rel(r2.D, exact.density_zero_T(p.e, p.Q, p.nocc)) < 1e-11
    # max_iter too small: reported as not converged
    r3 = sp2.sp2_density(p.H, p.nocc, idem_tol=1e-10, max_iter=5)
    assert not r3.converged and r3.M == 5


# ------------------------------------------------------------------ Sec. III / IV
@pytest.fixture(scope="module")
def run1(cfg1):
    return sp2.sp2_density(cfg1.H, cfg1.nocc, idem_tol=1e-10, keep=True)


def test_dm1_matches_loewner_closed_form(cfg1, run1):
    p, r = cfg1, run1
    for k in range(3):
        D1 = sp2.dm_response(r.X, r.sigma, r.beta, p.H1[k])
        D1_ex = exact.response_zero_T(p.e, p.Q, p.nocc, p.H1[k])
        assert rel(D1, D1_ex) < 1e-8
        _, (Y_ref,) = exact.finite_m_reference(p.e, p.Q, r.alpha, r.beta, r.sigma, p.H1[k])
        assert rel(D1, Y_ref) < 1e-12


def test_dm1_finite_m_unconverged(cfg1):
    """Branch sequence cut short (not converged): still the exact divided
    difference product of the branch polynomials."""
    p = cfg1
    sig = [1, -1, -1, 1, 1, -1, 1]
    r = sp2.sp2_density(p.H, p.nocc, sigma=sig, keep=True)
    Y = sp2.dm_response(r.X, r.sigma, r.beta, p.A)
    _, (Y_ref,) = exact.finite_m_reference(p.e, p.Q, r.alpha, r.beta, sig, p.A)
    assert rel(Y, Y_ref) < 1e-12


def test_backward_equals_forward_susceptibility(cfg1, run1):
    """Eq. MatFuncRel: the backward (Eq. DM2) and forward (Eq. DM3)
    susceptibilities are the same matrix for the same branch sequence."""
    p, r = cfg1, run1
    chi_b = sp2.susceptibility_backward(r.X, r.sigma, r.beta, p.A)
    chi_f = sp2.susceptibility_forward(r.X, r.sigma, r.beta, p.A)
    assert rel(chi_b, chi_f) < 1e-12
    chi_ex = exact.response_zero_T(p.e, p.Q, p.nocc, p.A)
    assert rel(chi_b, chi_ex) < 1e-8


def test_duality_identity(cfg1, run1):
    """Eq. Equivalence: Tr[A D1_k] = Tr[chi^A H1_k] (the paper reports 12
    matching digits in FP64)."""
    p, r = cfg1, run1
    chi = sp2.susceptibility_backward(r.X, r.sigma, r.beta, p.A)
    for k in range(p.H1.shape[0]):
        D1 = sp2.dm_response(r.X, r.sigma, r.beta, p.H1[k])
        a_direct = sp2.trace_product(p.A, D1)
        a_dual = sp2.trace_product(chi, p.H1[k])
        assert a_direct == pytest.approx(a_dual, rel=1e-12, abs=1e-14)


def test_central_difference_of_observable(cfg1, run1):
    """a^(1) = d Tr[A D(H + lambda H1)]/d lambda (Eq. dual) by central
    differences with the branch sequence and the spectral bounds frozen, so
    the differences follow the same polynomial; error O(h^2)."""
    p, r = cfg1, run1
    bounds = sp2.gershgorin_bounds(p.H)
    chi = sp2.susceptibility_backward(r.X, r.sigma, r.beta, p.A)
    h = 1e-4
    for k in range(2):
        Dp = sp2.sp2_density(p.H + h * p.H1[k], p.nocc, sigma=r.sigma, bounds=bounds).D
        Dm = sp2.sp2_density(p.H - h * p.H1[k], p.nocc, sigma=r.sigma, bounds=bounds).D
        fd = (sp2.trace_product(p.A, Dp) - sp2.trace_product(p.A, Dm)) / (2 * h)
        assert fd == pytest.approx(sp2.trace_product(chi, p.H1[k]), rel=1e-6, abs=1e-9)


def test_susceptibility_elementwise_brute_force():
    """Eq. Suscept: chi_ij = d Tr[A D] / d H_ij, entry by entry, on a tiny
    problem (each entry perturbed alone, branch sequence frozen)."""
    p = workloads.random_spectrum(8, nocc=4, k=0, seed=11)
    r = sp2.sp2_density(p.H, p.nocc, idem_tol=1e-12, keep=True)
    bounds = sp2.gershgorin_bounds(p.H)
    chi = sp2.susceptibility_backward(r.X, r.sigma, r.beta, p.A)
    h = 1e-5
    fd = np.zeros_like(chi)
    for i in range(8):
        for j in range(8):
            E = np.zeros((8, 8))
            E[i, j] = h
            dp = sp2.sp2_density(p.H + E, p.nocc, sigma=r.sigma, bounds=bounds).D
            dm = sp2.sp2_density(p.H - E, p.nocc, sigma=r.sigma, bounds=bounds).D
            fd[i, j] = (sp2.trace_product(p.A, dp) - sp2.trace_product(p.A, dm)) / (2 * h)
    assert np.max(np.abs(fd - chi)) < 1e-7 * max(1.0, np.max(np.abs(chi)))


def test_merged_forms_match_stored_history(cfg1, run1):
    """Appendix Eq. DMSuscept / DMPert: the merged loop gives the same
    D, chi and D1 as Eq. DM0 + DM3 / DM1 over stored X_n."""
    p, r = cfg1, run1
    res, chi = sp2.merged_response(p.H, p.nocc, p.A, idem_tol=1e-10)
    assert res.sigma == r.sigma
    assert rel(res.D, r.D) < 1e-14
    assert rel(chi, sp2.susceptibility_forward(r.X, r.sigma, r.beta, p.A)) < 1e-13
    res2, D1s = sp2.merged_response(p.H, p.nocc, p.H1[:3], idem_tol=1e-10)
    for k in range(3):
        assert rel(D1s[k], sp2.dm_response(r.X, r.sigma, r.beta, p.H1[k])) < 1e-13


def test_contractions_against_matrix_product_trace(cfg1):
    p = cfg1
    P = p.H1[:3]
    Q = p.H1[3:8]
    out = sp2.contract(P, Q)
    for l in range(3):
        for k in range(5):
            assert out[l, k] == pytest.approx(np.trace(P[l] @ Q[k]), rel=1e-12, abs=1e-14)
    q = np.random.default_rng(1).standard_normal((4, 128))
    od = sp2.contract_diag(P, q)
    for l in range(3):
        for k in range(4):
            assert od[l, k] == pytest.approx(np.trace(P[l] @ np.diag(q[k])), rel=1e-12, abs=1e-14)


def test_tight_binding_gap_and_sp2(tmp_path):
    """Tight-binding construction at N=512 (128 sites x 4 orbitals) is gapped
    at half filling, and SP2 reproduces its projector."""
    tb = workloads.tight_binding(512, seed=0)
    assert np.allclose(tb.H, tb.H.T)
    e, V = exact.eigh(tb.H)
    assert e[tb.nocc] - e[tb.nocc - 1] > 0.05
    r = sp2.sp2_density(tb.H, tb.nocc, idem_tol=1e-10)
    assert r.converged
    assert rel(r.D, exact.density_zero_T(e, V, tb.nocc)) < 1e-10


def test_floor_best_index():
    """floor_best: the smallest f at or below the gate, from X_2 on, 1-based."""
    f = [0.5, 0.02, 1e-6, 3e-9, 4e-8, 1e-9, 2e-8]
    assert sp2.floor_best(f, 0.03) == 6           # f[5] = 1e-9 is X_6
    assert sp2.floor_best([0.5, 0.2], 0.03) == 0
    assert sp2.floor_best([1e-9, 0.5, 0.01], 0.03) == 3   # X_1 is never chosen


def test_floor_stop_returns_best_iterate(cfg1):
    """With the tolerance test off, FP64 reaches its rounding floor; the run
    returns the floor candidate with the smallest f among X_2..X_s (s the step
    at which the floor test fired), and that iterate replays exactly from its
    own branch sequence."""
    p = cfg1
    r = sp2.sp2_density(p.H, p.nocc, idem_tol=0.0)
    assert r.converged and r.stop_step >= r.M
    long = sp2.sp2_density(p.H, p.nocc, idem_tol=0.0, floor_gate=0.0, max_iter=r.stop_step)
    cand = [(f, k + 1) for k, f in enumerate(long.fro) if k >= 1 and f <= 0.03]
    assert r.M + 1 == min(cand)[1]
    replay = sp2.sp2_density(p.H, p.nocc, sigma=r.sigma)
    assert np.array_equal(replay.D, r.D)
    assert sp2.idem_fro(r.D, r.D @ r.D) <= 1e-20
