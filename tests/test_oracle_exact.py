"""Pins for the closed forms and the split-precision helpers (CPU only)."""
import numpy as np
import pytest
import torch

import workloads
from oracle import exact, split


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_density_is_projector_with_right_trace():
    p = workloads.random_spectrum(40, nocc=13, k=0, seed=2)
    D = exact.density_zero_T(p.e, p.Q, p.nocc)
    assert rel(D @ D, D) < 1e-13
    assert np.trace(D) == pytest.approx(13, abs=1e-12)
    # D commutes with H and kills the empty states
    assert np.linalg.norm(D @ p.H - p.H @ D) < 1e-12
    empty = p.Q[:, np.argsort(p.e)[13:]]
    assert np.linalg.norm(D @ empty) < 1e-12


def test_sum_over_states_brute_force():
    """Daleckii-Krein against the explicit sum over state pairs at N=6."""
    p = workloads.random_spectrum(6, nocc=3, k=1, seed=7)
    B = p.H1[0]
    f = exact.occupations_zero_T(p.e, 3)
    D1 = exact.response_zero_T(p.e, p.Q, 3, B)
    bb = p.Q.T @ B @ p.Q
    ref = np.zeros((6, 6))
    for i in range(6):
        for j in range(6):
            s = 0.0
            for a in range(6):
                for b in range(6):
                    if f[a] != f[b]:
                        s += p.Q[i, a] * p.Q[j, b] * bb[a, b] * (f[a] - f[b]) / (p.e[a] - p.e[b])
            ref[i, j] = s
    assert np.max(np.abs(D1 - ref)) < 1e-13


def test_zero_T_response_is_derivative_of_projector():
    """D1 = d theta(mu - H - lambda H1)/d lambda by central differences of the
    eigen-decomposed projector (LAPACK), sign and scale included."""
    p = workloads.random_spectrum(24, nocc=10, k=1, seed=8)
    B = p.H1[0]
    h = 1e-5
    ep, Vp = exact.eigh(p.H + h * B)
    em, Vm = exact.eigh(p.H - h * B)
    fd = (exact.density_zero_T(ep, Vp, 10) - exact.density_zero_T(em, Vm, 10)) / (2 * h)
    assert rel(exact.response_zero_T(p.e, p.Q, 10, B), fd) < 1e-8


def test_hadamard_trace_symmetry():
    """Tr[(L o X) Y] = Tr[(L o Y) X] for symmetric L, X, Y (Appendix)."""
    rng = np.random.default_rng(9)
    L = workloads.sym_gaussian(rng, 9, 1.0)
    X = workloads.sym_gaussian(rng, 9, 1.0)
    Y = workloads.sym_gaussian(rng, 9, 1.0)
    assert np.trace((L * X) @ Y) == pytest.approx(np.trace((L * Y) @ X), rel=1e-13)


def test_divided_difference_of_square_maps():
    """Scalar pins: x^2 has divided difference x_i + x_j, 2x - x^2 has
    2 - x_i - x_j; on the diagonal these are the derivatives 2x and 2 - 2x."""
    x = np.array([0.1, 0.45, 0.9])
    L1 = exact.sp2_divided_difference(exact.sp2_scalar(x, [1]), [1], 1.0)
    Lm = exact.sp2_divided_difference(exact.sp2_scalar(x, [-1]), [-1], 1.0)
    for i in range(3):
        for j in range(3):
            if i != j:
                assert L1[i, j] == pytest.approx((x[i] ** 2 - x[j] ** 2) / (x[i] - x[j]))
                g = lambda t: 2 * t - t * t  # noqa: E731
                assert Lm[i, j] == pytest.approx((g(x[i]) - g(x[j])) / (x[i] - x[j]))
        assert L1[i, i] == pytest.approx(2 * x[i])
        assert Lm[i, i] == pytest.approx(2 - 2 * x[i])


def test_fermi_function_and_derivative():
    e = np.linspace(-1, 1, 41)
    f = exact.fermi(e, 0.1, 0.05)
    assert np.allclose(f, 1.0 / (np.exp((e - 0.1) / 0.05) + 1.0), rtol=1e-13, atol=1e-15)
    h = 1e-6
    fd = (exact.fermi(e + h, 0.1, 0.05) - exact.fermi(e - h, 0.1, 0.05)) / (2 * h)
    assert np.allclose(exact.fermi_prime(e, 0.1, 0.05), fd, rtol=1e-6, atol=1e-8)


def test_fermi_response_grand_canonical_and_canonical():
    """Grand-canonical D1 equals the central difference of V f(e) V^T; the
    canonical one differs by a multiple of V diag(f') V^T and has Tr = 0."""
    p = workloads.random_spectrum(20, nocc=10, k=1, seed=10, lo=(-1, 0), hi=(0, 1))
    B = p.H1[0]
    mu, kT = 0.0, 0.1
    h = 1e-5

    def dens(H):
        e, V = exact.eigh(H)
        return (V * exact.fermi(e, mu, kT)) @ V.T

    fd = (dens(p.H + h * B) - dens(p.H - h * B)) / (2 * h)
    gc = exact.response_fermi(p.e, p.Q, mu, kT, B, canonical=False)
    assert rel(gc, fd) < 1e-8
    c = exact.response_fermi(p.e, p.Q, mu, kT, B, canonical=True)
    assert abs(np.trace(c)) < 1e-12
    diff = gc - c
    G = (p.Q * exact.fermi_prime(p.e, mu, kT)) @ p.Q.T
    coef = np.sum(diff * G) / np.sum(G * G)
    assert rel(diff, coef * G) < 1e-10


def test_bf16_rounding_matches_library_cast():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200000) * 10.0 ** rng.integers(-20, 20, 200000)).astype(np.float32)
    ours = split.round_bf16(x)
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours, lib)


def test_split_error_bounds():
    """Eq. doubleHalf: hi + lo recovers x to about two narrow mantissas."""
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, 100000).astype(np.float32)
    for kind, bits in (("bf16", 8), ("fp16", 11)):
        hi, lo = split.split_hi_lo(x, kind)
        err = np.abs(x.astype(np.float64) - hi - lo)
        # |x - hi| <= 2^-bits |x|, and lo rounds that residual to `bits` bits
        bound = np.abs(x) * 2.0 ** (-2 * bits) + (6e-8 if kind == "fp16" else 0.0)
        assert np.all(err <= bound * 1.0001 + 1e-38)
        assert np.array_equal(hi, split.round_bf16(x) if kind == "bf16" else split.round_fp16(x))


def test_mixed_product_accuracy():
    """Eq. MixPrecMult without lo*lo: relative error near the split's unit
    roundoff, far below a single narrow product."""
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (96, 96))
    Y = rng.uniform(-1, 1, (96, 96))
    ref = X @ Y
    for kind, tol, single in (("bf16", 4e-5, 1e-3), ("fp16", 1e-6, 2e-4)):
        mp = split.mixed_product(X, Y, kind)
        xh, _ = split.split_hi_lo(X, kind)
        yh, _ = split.split_hi_lo(Y, kind)
        one = xh.astype(np.float64) @ yh.astype(np.float64)
        assert rel(mp, ref) < tol
        assert rel(one, ref) > single * 0.1
    # lo scaling by a power of two leaves the product unchanged up to rounding
    a = split.mixed_product(X, Y, "fp16", lo_scale=2.0 ** 12)
    assert rel(a, ref) < 1e-6


def test_pow2_scale_keeps_fp16_range():
    for b in (1e-30, 3e-8, 0.7, 1.0, 17.0, 1e5, 6.5e4):
        s = split.pow2_scale(b)
        assert np.log2(s) == int(np.log2(s))
        assert 2.0 ** 13 <= b * s <= 2.0 ** 14
    assert split.pow2_scale(0.0) == 1.0 and split.pow2_scale(float("nan")) == 1.0


def test_scaled_fp16_split_product():
    """A power-of-two plane scale changes nothing but the range: the product of
    scaled splits equals the unscaled one where neither under- nor overflows,
    and it rescues entries that would overflow FP16."""
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (64, 64))
    Y = rng.uniform(-1, 1, (64, 64)) * 1e6          # overflows FP16 unscaled
    s = split.pow2_scale(np.max(np.abs(Y)))
    P = split.mixed_product(Y, X, "fp16", lo_scale=2048.0, sx=s)
    assert np.isfinite(P).all()
    assert np.linalg.norm(P - Y @ X) / np.linalg.norm(Y @ X) < 1e-6


def test_three_plane_split_is_exact_and_ordered():
    """hi + mid + lo reconstructs FP32 exactly; each plane is a bfloat16 value
    at most 2^-8 of the previous residual (relative to x: mid <= 2^-8 |x|,
    lo <= 2^-16 |x|, up to the rounding of each step)."""
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    h, m, lo = split.split_hi_mid_lo(x)
    for p in (h, m, lo):
        assert np.array_equal(p, split.round_bf16(p))          # representable in bf16
    assert np.array_equal((h.astype(np.float64) + m + lo).astype(np.float32), x)
    assert np.array_equal(h.astype(np.float64) + m + lo, x.astype(np.float64))
    ax = np.abs(x.astype(np.float64))
    assert np.all(np.abs(m) <= 2.0 ** -8 * ax * (1 + 2.0 ** -7))
    assert np.all(np.abs(lo) <= 2.0 ** -16 * ax * (1 + 2.0 ** -6))


def test_three_plane_product_accuracy():
    """The six-term product is within a few 2^-24 of the exact FP32-input
    product (the dropped terms are 2^-24 relative per element pair), far below
    the two-plane form's 2^-16."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((96, 96)).astype(np.float32)
    Y = rng.standard_normal((96, 96)).astype(np.float32)
    exact_ = X.astype(np.float64) @ Y.astype(np.float64)
    scale = np.abs(X).astype(np.float64) @ np.abs(Y).astype(np.float64)
    e3 = np.max(np.abs(split.mixed_product3(X, Y) - exact_) / scale)
    e2 = np.max(np.abs(split.mixed_product(X, Y, "bf16") - exact_) / scale)
    assert e3 < 4 * 2.0 ** -24
    assert e2 > 16 * e3


def test_three_plane_pin_catches_a_dropped_term():
    """Dropping one of the 2^-16 terms (mid.mid) from the six-term product
    moves it far outside the 4 * 2^-24 bound of the accuracy pin."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((64, 64)).astype(np.float32)
    Y = rng.standard_normal((64, 64)).astype(np.float32)
    exact_ = X.astype(np.float64) @ Y.astype(np.float64)
    scale = np.abs(X).astype(np.float64) @ np.abs(Y).astype(np.float64)
    xh, xm, xl = (a.astype(np.float64) for a in split.split_hi_mid_lo(X))
    yh, ym, yl = (a.astype(np.float64) for a in split.split_hi_mid_lo(Y))
    wrong = xh @ yh + (xh @ ym + xm @ yh) + (xh @ yl + xl @ yh)
    assert np.max(np.abs(wrong - exact_) / scale) > 4 * 2.0 ** -24
