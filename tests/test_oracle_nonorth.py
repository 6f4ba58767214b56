"""Pins for the non-orthonormal representation oracle (Sec. V.A), CPU only.

The dual three-contraction derivative is checked against central differences
of a(tau) = Tr[A(tau) D(tau)] with D(tau) from LAPACK's generalized
eigensolver on (H + tau H_t, S + tau S_t) -- a path that never forms Z,
H^perp or chi -- so a dropped term, a sign or a transposed factor in W_H or
W_S fails it.
"""
import numpy as np
import pytest

import workloads
from oracle import nonorth


@pytest.fixture(scope="module")
def prob():
    return workloads.nonorth_problem(96, nocc=40, seed=0)


def test_lowdin_factor(prob):
    Z = nonorth.lowdin(prob.S)
    assert np.allclose(Z, Z.T, atol=1e-13)
    assert np.allclose(Z.T @ prob.S @ Z, np.eye(len(Z)), atol=1e-12)


def test_density_is_s_projector(prob):
    """D S D = D, Tr[D S] = N_occ, and the congruence route of Sec. V.A
    (D = Z theta(mu - Z^T H Z) Z^T) equals the generalized eigensolver's D."""
    D = nonorth.density_generalized(prob.H, prob.S, prob.nocc)
    assert np.allclose(D @ prob.S @ D, D, atol=1e-11)
    assert abs(np.trace(D @ prob.S) - prob.nocc) < 1e-10
    _, D2, _, _ = nonorth.dual_weights(prob.H, prob.S, prob.A, prob.nocc)
    assert np.allclose(D2, D, atol=1e-11)


def test_dual_derivative_matches_finite_differences(prob):
    _, D, WH, WS = nonorth.dual_weights(prob.H, prob.S, prob.A, prob.nocc)
    h = 1e-5
    for k in range(3):
        At, Ht, St = prob.A_t[k], prob.H_t[k], prob.S_t[k]

        def a(t):
            Dt = nonorth.density_generalized(prob.H + t * Ht, prob.S + t * St, prob.nocc)
            return float(np.sum((prob.A + t * At) * Dt))
        fd = (a(h) - a(-h)) / (2 * h)
        dual = nonorth.derivative_dual(D, WH, WS, At, Ht, St)
        assert dual == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_orthonormal_limit(prob):
    """S = I, S_tau = 0: W_H is chi^A and the derivative is Tr[A_t D] + Tr[chi H_t]."""
    from oracle import exact
    I = np.eye(len(prob.H))
    _, D, WH, WS = nonorth.dual_weights(prob.H, I, prob.A, prob.nocc)
    e, V = exact.eigh(prob.H)
    assert np.allclose(WH, exact.response_zero_T(e, V, prob.nocc, prob.A), atol=1e-12)
    assert np.allclose(D, exact.density_zero_T(e, V, prob.nocc), atol=1e-12)


@pytest.mark.parametrize("mistake", ["ws_sign", "ws_drop_ad", "wh_transpose_z"])
def test_planted_mistakes_fail_the_pin(prob, mistake):
    """A plausible slip in the weights (a flipped sign, a dropped term, Z on the
    wrong side) breaks agreement with the finite differences of the generalized
    eigenproblem, so the pin above would catch it."""
    Z, D, WH, WS = nonorth.dual_weights(prob.H, prob.S, prob.A, prob.nocc)
    Sinv = Z @ Z.T
    if mistake == "ws_sign":
        WS = -WS
    elif mistake == "ws_drop_ad":
        P = Sinv @ prob.A @ D
        WS = WS + 0.5 * (P + P.T)
    else:
        WH = Z.T @ WH @ Z     # chi moved through the congruence twice
    At, Ht, St = prob.A_t[0], prob.H_t[0], prob.S_t[0]
    h = 1e-5

    def a(t):
        Dt = nonorth.density_generalized(prob.H + t * Ht, prob.S + t * St, prob.nocc)
        return float(np.sum((prob.A + t * At) * Dt))
    fd = (a(h) - a(-h)) / (2 * h)
    assert nonorth.derivative_dual(D, WH, WS, At, Ht, St) != pytest.approx(fd, rel=1e-4)
