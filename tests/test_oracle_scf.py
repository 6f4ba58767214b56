"""Pins for the self-consistent response oracle and its MLP (CPU only)."""
import numpy as np
import pytest

import workloads
from oracle import exact, scf


@pytest.fixture(scope="module")
def small():
    tb = workloads.tight_binding(256, seed=0)          # 64 sites x 4 orbitals
    e, V = exact.eigh(tb.H)
    chi0 = scf.chi0_sites(e, V, tb.nocc, tb.norb)
    K = workloads.site_kernel(tb, "regularised")
    Vx = workloads.site_fields(tb, 6, seed=3)
    return tb, e, V, chi0, K, Vx


def test_chi0_matches_finite_differences(small):
    """chi0_ab = d q_a / d u_b against central differences of the projector."""
    tb, e, V, chi0, K, Vx = small
    h = 1e-5
    for b in (0, 17):
        P = np.zeros(tb.n)
        P[b * 4:(b + 1) * 4] = 1.0
        ep, Vp = exact.eigh(tb.H + h * np.diag(P))
        em, Vm = exact.eigh(tb.H - h * np.diag(P))
        dD = (exact.density_zero_T(ep, Vp, tb.nocc) - exact.density_zero_T(em, Vm, tb.nocc)) / (2 * h)
        col = np.diag(dD).reshape(-1, 4).sum(axis=1)
        assert np.allclose(chi0[:, b], col, rtol=1e-6, atol=1e-9)


def test_chi0_symmetric_and_charge_conserving(small):
    """chi0 is symmetric (Eq. Equivalence for site perturbations) and a
    uniform potential moves no charge at fixed N_occ (rows sum to zero)."""
    tb, e, V, chi0, K, Vx = small
    assert np.allclose(chi0, chi0.T, atol=1e-12)
    assert np.allclose(chi0.sum(axis=1), 0.0, atol=1e-10)


def test_scf_solution_is_fixed_point(small):
    tb, e, V, chi0, K, Vx = small
    qs = scf.scf_exact(chi0, K, Vx)
    qout = (chi0 @ (Vx + qs @ K.T).T).T
    assert np.linalg.norm(qout - qs) < 1e-10 * max(1.0, np.linalg.norm(qs))


@pytest.mark.parametrize("mixer", ["linear", "anderson"])
def test_mixers_converge_to_exact_solution(small, mixer):
    tb, e, V, chi0, K, Vx = small
    q, res = scf.scf_iterate(chi0, K, Vx, mixer=mixer, alpha=0.3, tol=1e-10, max_iter=500)
    assert res[-1] <= 1e-10
    assert np.linalg.norm(q - scf.scf_exact(chi0, K, Vx)) < 1e-8 * np.linalg.norm(q)


def test_anderson_beats_linear(small):
    tb, e, V, chi0, K, Vx = small
    _, rl = scf.scf_iterate(chi0, K, Vx, mixer="linear", tol=1e-8, max_iter=500)
    _, ra = scf.scf_iterate(chi0, K, Vx, mixer="anderson", tol=1e-8, max_iter=500)
    assert len(ra) < len(rl)


def test_mlp_gradients_by_finite_differences():
    rng = np.random.default_rng(0)
    W1 = rng.standard_normal((7, 5)) * 0.5
    W2 = rng.standard_normal((5, 7)) * 0.5
    X = rng.standard_normal((9, 5))
    T = rng.standard_normal((9, 5))
    L, g1, g2 = scf.mlp_loss_grad(W1, W2, X, T)
    h = 1e-6
    for W, g in ((W1, g1), (W2, g2)):
        for idx in [(0, 0), (3, 2), (4, 4)]:
            Wp = W.copy(); Wp[idx] += h
            Wm = W.copy(); Wm[idx] -= h
            args_p = (Wp, W2) if W is W1 else (W1, Wp)
            args_m = (Wm, W2) if W is W1 else (W1, Wm)
            fd = (scf.mlp_loss_grad(*args_p, X, T)[0] - scf.mlp_loss_grad(*args_m, X, T)[0]) / (2 * h)
            assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_mlp_is_positively_homogeneous():
    rng = np.random.default_rng(1)
    W1 = rng.standard_normal((6, 4))
    W2 = rng.standard_normal((4, 6))
    X = rng.standard_normal((3, 4))
    assert np.allclose(scf.mlp_forward(W1, W2, 3.5 * X), 3.5 * scf.mlp_forward(W1, W2, X))


def test_adam_matches_definition():
    w, g = np.array([1.0, -2.0]), np.array([0.5, 0.25])
    m, v = np.zeros(2), np.zeros(2)
    w1, m1, v1 = scf.adam_step(w, g, m, v, 1, 0.1)
    # first step: m_hat = g, v_hat = g^2 -> w - lr * g / (|g| + eps) = w - lr * sign(g)
    assert np.allclose(w1, w - 0.1 * np.sign(g), atol=1e-7)


def test_scf_dual_equals_primal(small):
    """Self-consistent duality (Eq. CP_SCF for the site-charge model): for a
    site observable a and an external field V, a . q*(V) = q*(a) . V, because
    (I - chi0 K)^(-1) chi0 = chi0 (I - K chi0)^(-1) is symmetric for symmetric
    chi0 and K. One self-consistent solve per observable then gives the
    response to every field. A solve with the transposed operator or the
    factors in the other order breaks the identity."""
    tb, e, V, chi0, K, Vx = small
    ctr = tb.pos - 0.5 * tb.box
    obs = ctr.T.copy()                                  # x, y, z site dipoles
    primal = obs @ scf.scf_exact(chi0, K, Vx).T         # [l, k] = a_l . q*(V_k)
    dual = scf.scf_exact(chi0, K, obs) @ Vx.T           # [l, k] = q*(a_l) . V_k
    assert np.allclose(primal, dual, rtol=1e-10, atol=1e-12 * np.abs(primal).max())
    # the non-self-consistent limit K = 0 is the plain symmetry of chi0
    Z = np.zeros_like(K)
    assert np.allclose(obs @ scf.scf_exact(chi0, Z, Vx).T, (obs @ chi0) @ Vx.T, rtol=1e-10)


def test_finite_t_chi0_and_scf_duality(small):
    """Finite-temperature site susceptibility (canonical): symmetric, charge
    conserving (a uniform potential moves no charge: Tr[D1] = 0 by mu_1), equal
    to central differences of the Fermi-Dirac site charges at fixed electron
    count, and the self-consistent duality a . q*(V) = q*(a) . V holds."""
    from oracle import exact
    tb, e, V, chi0, K, Vx = small
    mu = 0.5 * (e[tb.nocc - 1] + e[tb.nocc])
    kT = 0.05
    c0 = scf.chi0_sites_fermi(e, V, mu, kT, tb.norb, canonical=True)
    assert np.allclose(c0, c0.T, atol=1e-12)
    assert np.allclose(c0.sum(axis=0), 0.0, atol=1e-10)
    # grand canonical: central differences of the site charges at fixed mu
    cg = scf.chi0_sites_fermi(e, V, mu, kT, tb.norb, canonical=False)
    h = 1e-5
    b = 5
    P = np.zeros(tb.n)
    P[b * 4:(b + 1) * 4] = 1.0

    def q(t):
        ee, VV = exact.eigh(tb.H + t * np.diag(P))
        D = (VV * exact.fermi(ee, mu, kT)[None, :]) @ VV.T
        return np.diag(D).reshape(-1, 4).sum(axis=1)
    assert np.allclose(cg[:, b], (q(h) - q(-h)) / (2 * h), rtol=1e-6, atol=1e-9)
    obs = (tb.pos - 0.5 * tb.box).T.copy()
    primal = obs @ scf.scf_exact(c0, K, Vx).T
    dual = scf.scf_exact(c0, K, obs) @ Vx.T
    assert np.allclose(primal, dual, rtol=1e-10, atol=1e-12 * np.abs(primal).max())


# ------------------------------------------------------------ the learned mixer
# The MLP mixer of scf_iterate: q <- q + alpha r + ||r|| MLP(r / ||r||) with
# MLP(x) = W2 relu(W1 x), no biases.

def test_mlp_mixer_with_zero_network_is_linear_mixing(small):
    """An MLP whose output layer is zero adds nothing: the residual history and
    the iterate equal plain linear mixing with the same alpha, step for step."""
    tb, e, V, chi0, K, Vx = small
    ns = chi0.shape[0]
    rng = np.random.default_rng(1)
    W1 = rng.standard_normal((16, ns))
    W2 = np.zeros((ns, 16))
    ql, rl = scf.scf_iterate(chi0, K, Vx, mixer="linear", alpha=0.3, tol=1e-9, max_iter=40)
    qm, rm = scf.scf_iterate(chi0, K, Vx, mixer="mlp", alpha=0.3, tol=1e-9, max_iter=40,
                             mlp=(W1, W2))
    assert rm == rl
    assert np.array_equal(qm, ql)


# Two sites, one field, no interaction (K = 0), chi0 = I/2, V = [2, -2]: the
# output charges are q_out = [1, -1] whatever q is. alpha = 0.3,
# W1 = [[1, 0.5], [0, 1]], W2 = [[0.2, 0.6], [-0.4, 0.8]]. Worked by hand
# (||r|| MLP(r/||r||) = MLP(r), the map being positively homogeneous):
#   it 0: q = 0, r = [1, -1], residual ||r|| / ||q_out(0)|| = 1;
#         W1 r = [0.5, -1] -> relu [0.5, 0] -> W2 . = [0.1, -0.2];
#         q = 0.3 r + [0.1, -0.2] = [0.4, -0.5]
#   it 1: r = [0.6, -0.5], residual sqrt(0.61 / 2) = sqrt(0.305);
#         W1 r = [0.35, -0.5] -> relu [0.35, 0] -> W2 . = [0.07, -0.14];
#         q = [0.4, -0.5] + [0.18, -0.15] + [0.07, -0.14] = [0.65, -0.79]
#   it 2: r = [0.35, -0.21], residual sqrt(0.1666 / 2) = sqrt(0.0833)
_HAND = dict(chi0=np.eye(2) / 2, K=np.zeros((2, 2)), V=np.array([[2.0, -2.0]]),
             W1=np.array([[1.0, 0.5], [0.0, 1.0]]), W2=np.array([[0.2, 0.6], [-0.4, 0.8]]))


def test_mlp_mixer_two_steps_worked_by_hand():
    h = _HAND
    kw = dict(mixer="mlp", alpha=0.3, tol=0.0, mlp=(h["W1"], h["W2"]))
    q1, r1 = scf.scf_iterate(h["chi0"], h["K"], h["V"], max_iter=1, **kw)
    q2, r2 = scf.scf_iterate(h["chi0"], h["K"], h["V"], max_iter=2, **kw)
    _, r3 = scf.scf_iterate(h["chi0"], h["K"], h["V"], max_iter=3, **kw)
    assert np.allclose(q1, [[0.4, -0.5]], rtol=0, atol=1e-15)
    assert np.allclose(q2, [[0.65, -0.79]], rtol=0, atol=1e-15)
    assert np.allclose(r3, [1.0, np.sqrt(0.305), np.sqrt(0.0833)], rtol=1e-14, atol=0)


def test_mlp_mixer_with_the_exact_correction_converges_in_one_step(small):
    """For q_out(q) = chi0 (V + K q) the exact step from q = 0 is
    q* = (I - chi0 K)^(-1) r_0 = alpha r_0 + C r_0 with C = (I - chi0 K)^(-1) - alpha I.
    The ReLU pair W1 = [I; -I], W2 = [C, -C] represents C exactly
    (relu(x) - relu(-x) = x), so one mixer step lands on the closed-form solution."""
    tb, e, V, chi0, K, Vx = small
    ns = chi0.shape[0]
    alpha = 0.3
    C = np.linalg.inv(np.eye(ns) - chi0 @ K) - alpha * np.eye(ns)
    W1 = np.vstack([np.eye(ns), -np.eye(ns)])
    W2 = np.hstack([C, -C])
    q, res = scf.scf_iterate(chi0, K, Vx, mixer="mlp", alpha=alpha, tol=1e-11, max_iter=5,
                             mlp=(W1, W2))
    assert len(res) == 2 and res[1] < 1e-11
    assert np.allclose(q, scf.scf_exact(chi0, K, Vx), rtol=1e-10, atol=1e-13)


# ------------------------------------------------------------ Anderson with the learned step
# anderson_mlp: q <- sum_i c_i (q_i + P(r_i)), P(r) = alpha r + ||r|| MLP(r / ||r||).

def test_anderson_mlp_with_zero_network_is_anderson(small):
    tb, e, V, chi0, K, Vx = small
    ns = chi0.shape[0]
    W1 = np.random.default_rng(2).standard_normal((8, ns))
    W2 = np.zeros((ns, 8))
    qa, ra = scf.scf_iterate(chi0, K, Vx, mixer="anderson", alpha=0.3, tol=1e-9, max_iter=40)
    qm, rm = scf.scf_iterate(chi0, K, Vx, mixer="anderson_mlp", alpha=0.3, tol=1e-9, max_iter=40,
                             mlp=(W1, W2))
    assert rm == ra
    assert np.array_equal(qm, qa)


def test_anderson_mlp_with_history_one_is_the_mlp_mixer(small):
    """With one stored iterate the Anderson coefficient is 1, so the step is
    q + P(r): the MLP mixer, iterate for iterate."""
    tb, e, V, chi0, K, Vx = small
    ns = chi0.shape[0]
    rng = np.random.default_rng(3)
    W1 = rng.standard_normal((16, ns)) / np.sqrt(ns)
    W2 = 0.05 * rng.standard_normal((ns, 16)) / 4.0
    q1, r1 = scf.scf_iterate(chi0, K, Vx, mixer="mlp", alpha=0.3, tol=1e-8, max_iter=60,
                             mlp=(W1, W2))
    q2, r2 = scf.scf_iterate(chi0, K, Vx, mixer="anderson_mlp", alpha=0.3, hist=1, tol=1e-8,
                             max_iter=60, mlp=(W1, W2))
    # the one-by-one KKT solve gives c = 1 up to rounding, which the residuals
    # carry relative to their own size as they fall to 1e-8 (measured 3.4e-9)
    assert len(r1) == len(r2)
    assert np.allclose(r1, r2, rtol=1e-7, atol=0)
    assert np.allclose(q1, q2, rtol=1e-9, atol=1e-12)


def test_anderson_mlp_with_the_exact_preconditioner_converges_in_one_step(small):
    """P(r) = (I - chi0 K)^(-1) r (the ReLU pair representing (I - chi0 K)^(-1) - alpha I):
    the first step from q = 0 lands on the closed-form solve."""
    tb, e, V, chi0, K, Vx = small
    ns = chi0.shape[0]
    alpha = 0.3
    C = np.linalg.inv(np.eye(ns) - chi0 @ K) - alpha * np.eye(ns)
    W1 = np.vstack([np.eye(ns), -np.eye(ns)])
    W2 = np.hstack([C, -C])
    q, res = scf.scf_iterate(chi0, K, Vx, mixer="anderson_mlp", alpha=alpha, tol=1e-11,
                             max_iter=5, mlp=(W1, W2))
    assert len(res) == 2 and res[1] < 1e-11
    assert np.allclose(q, scf.scf_exact(chi0, K, Vx), rtol=1e-10, atol=1e-13)
