"""Pins for the finite-temperature recursion of the oracle (CPU only)."""
import numpy as np
import pytest

import workloads
from oracle import exact, fermi


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def metal():
    """Gapless spectrum U[-1, 1] (the metallic finite-T workload), small N."""
    return workloads.metallic_spectrum(64, k=3, seed=5)


def test_scalar_recursion_closed_form():
    """delta_n = -tanh(2^n artanh(x / 2^(n+1))) / 2 (tanh doubling), for
    starts inside the parametrised range |x| < 2^(n+1)."""
    for n in (1, 4, 12):
        x = np.linspace(-40, 40, 161)
        x = x[np.abs(x) < 0.99 * 2.0 ** (n + 1)]
        ds = fermi.scalar_deltas(-x / 2.0 ** (n + 2), n)
        assert np.allclose(ds[-1], fermi.delta_closed_form(x, n), rtol=1e-12, atol=1e-15)


def test_recursion_converges_to_fermi_function():
    """With n doublings the log-odds error is 2 (x/2)^3 / (3 4^n) to leading order."""
    x = np.linspace(-20, 20, 81)
    exact_f = 1.0 / (np.exp(x) + 1.0)
    for n in (8, 14, 20):
        f = 0.5 + fermi.delta_closed_form(x, n)
        bound = exact_f * (1 - exact_f) * 2 * (np.abs(x) / 2) ** 3 / (3 * 4.0 ** n) * 1.05 + 5e-14
        assert np.all(np.abs(f - exact_f) <= bound)


def test_step_divided_difference_is_exact():
    a = np.array([0.3, -0.1, 0.45])
    b = np.array([-0.2, -0.1, 0.05])
    phi = lambda d: 2 * d / (1 + 4 * d * d)  # noqa: E731
    dd = fermi.step_divided_difference(a, b)
    for i in range(3):
        if a[i] != b[i]:
            assert dd[i] == pytest.approx((phi(a[i]) - phi(b[i])) / (a[i] - b[i]))
        else:
            h = 1e-6
            assert dd[i] == pytest.approx((phi(a[i] + h) - phi(a[i] - h)) / (2 * h), rel=1e-8)


@pytest.mark.parametrize("canonical", [False, True])
def test_matrix_recursion_matches_eigen_reference(metal, canonical):
    p = metal
    D, R = fermi.fermi_recursion(p.H, 0.0, 0.05, 10, p.H1, canonical=canonical)
    Dr, Rr = fermi.fermi_recursion_reference(p.e, p.Q, 0.0, 0.05, 10, p.H1, canonical=canonical)
    assert rel(D, Dr) < 1e-13
    for a, b in zip(R, Rr):
        assert rel(a, b) < 1e-11
    if canonical:
        assert all(abs(np.trace(a)) < 1e-10 for a in R)


def test_large_n_matches_exact_fermi_dirac(metal):
    """At n = 20 the recursion equals the exact Fermi-Dirac density and its
    (grand-canonical and canonical) Daleckii-Krein responses."""
    p = metal
    kT = 0.05
    D, R = fermi.fermi_recursion(p.H, 0.1, kT, 20, p.H1, canonical=False)
    f = exact.fermi(p.e, 0.1, kT)
    assert rel(D, (p.Q * f) @ p.Q.T) < 1e-9
    for b, r in zip(p.H1, R):
        assert rel(r, exact.response_fermi(p.e, p.Q, 0.1, kT, b, canonical=False)) < 1e-8
    D, R = fermi.fermi_recursion(p.H, 0.1, kT, 20, p.H1, canonical=True)
    for b, r in zip(p.H1, R):
        assert rel(r, exact.response_fermi(p.e, p.Q, 0.1, kT, b, canonical=True)) < 1e-8


def test_finite_temperature_duality(metal):
    """Eq. Equivalence at finite T: Tr[A D1(B)] = Tr[B chi^A] with chi^A the
    response to A, for the grand-canonical and the canonical response."""
    p = metal
    for canonical in (False, True):
        _, (chi,) = fermi.fermi_recursion(p.H, 0.0, 0.05, 12, p.A, canonical=canonical)
        _, R = fermi.fermi_recursion(p.H, 0.0, 0.05, 12, p.H1, canonical=canonical)
        for b, r in zip(p.H1, R):
            assert np.sum(p.A * r) == pytest.approx(np.sum(b * chi), rel=1e-10, abs=1e-13)
