"""Split-tail arithmetic (sp2_opts.tail_f): single-plane 16-bit products in the
steps whose last measured idempotency error f = ||X - X^2||_F^2 exceeds tail_f,
split products (Eq. MixPrecMult) from there on -- low precision in the bulk of
the iterations and the split form in the idempotency tail (Sec. VI.B).

What sets its accuracy: for a near-idempotent X = P + E both branches map the
occupied-virtual block of a perturbation E to itself (P E + E P and
2E - (P E + E P) both leave E_ov unchanged), so the rounding of every bulk step
stays in the eigenvector subspace of the result, and the split tail restores
idempotency but not the subspace. The density error is then u_hi * kappa
(u_hi the unit roundoff of the hi planes, kappa the spectral width over the
gap): measured 2.4e-3 (fp16 hi) and 2.0e-2 (bfloat16 hi) at kappa = 5, against
7e-6 for the split products in every step.

Checked: a step in single-plane arithmetic equals the product of the hi planes
(FP64 evaluation of the same fp16 values); the converged result stays within
twice u_hi * kappa (D) of the closed forms, forward and backward (the adjoint
replaying the forward's per-step choice); a threshold of 0 is the plain split
mode, bit for bit."""
import numpy as np
import pytest
import torch

import workloads
from oracle import exact, split

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sp2():
    import __graft_entry__ as g
    g.build()
    import paper_2409_17033_gb300 as p
    return p


@pytest.fixture(scope="module")
def c1():
    return workloads.random_spectrum(128, nocc=64, k=3, seed=0)


def f32(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


def test_single_plane_step_is_the_hi_product(sp2, c1):
    p = c1
    for s in (1, -1):
        D, info = sp2.sp2_density(f32(p.H), p.nocc, mode="fp16x2", sigma=[s], tail_f=1e30)
        assert info["tail_single_steps"] == 1
        a, b = info["alpha"], info["beta"]
        X1 = (a * np.eye(128) + b * p.H.astype(np.float32).astype(np.float64)).astype(np.float32)
        xh, _ = split.split_hi_lo(X1, "fp16")
        P = xh.astype(np.float64) @ xh.astype(np.float64)
        ref = P if s > 0 else 2.0 * X1.astype(np.float64) - P
        assert rel(D.cpu().numpy(), ref) < 1e-6


U_HI = {"fp16x2": 2.0 ** -11, "bf16x3": 2.0 ** -8}   # unit roundoff of the hi planes


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3"])
def test_tail_mode_accuracy_is_set_by_the_bulk_planes(sp2, c1, mode):
    p = c1
    H, A = f32(p.H), f32(p.A[None])
    kw = dict(mode=mode, tail_f=1e-2)
    chi_b, D, info = sp2.sp2_susceptibility(H, p.nocc, A, "backward", want_density=True, **kw)
    chi_f, _, info_f = sp2.sp2_susceptibility(H, p.nocc, A, "forward", **kw)
    assert info["converged"] and 0 < info["tail_single_steps"] < info["M"]
    assert info_f["tail_single_steps"] == info["tail_single_steps"]
    kappa = (p.e.max() - p.e.min()) / (p.e[np.argsort(p.e)[p.nocc]] - p.e[np.argsort(p.e)[p.nocc - 1]])
    chi_ex = exact.response_zero_T(p.e, p.Q, p.nocc, p.A)
    eD = rel(D.cpu().numpy(), exact.density_zero_T(p.e, p.Q, p.nocc))
    eb = rel(chi_b[0].cpu().numpy(), chi_ex)
    ef = rel(chi_f[0].cpu().numpy(), chi_ex)
    bar = U_HI[mode] * kappa
    print(f"tail {mode}: single-plane steps {info['tail_single_steps']} of {info['M']}, "
          f"kappa {kappa:.2f}, rel err D {eD:.2e} chi bwd {eb:.2e} fwd {ef:.2e} (u_hi kappa {bar:.2e})")
    assert eD < 2.0 * bar
    assert eb < 20.0 * bar and ef < 20.0 * bar


def test_zero_threshold_is_the_split_mode(sp2, c1):
    p = c1
    H, A = f32(p.H), f32(p.A[None])
    chi0, D0, i0 = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode="fp16x2",
                                          want_density=True)
    chi1, D1, i1 = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode="fp16x2",
                                          want_density=True, tail_f=0.0)
    assert i1["tail_single_steps"] == 0 and i0["sigma"] == i1["sigma"]
    assert torch.equal(chi0, chi1) and torch.equal(D0, D1)


def test_named_bf16_tail_mode_is_bf16x2_with_the_split_tail(sp2, c1):
    """SP2_MODE_BF16_TAIL (the boundary's bfloat16-bulk / split-tail mode) is
    BF16X2 with tail_f = SP2_DEFAULT_TAIL_F unless tail_f is given: bit for bit
    the same results, and single-plane steps in the bulk only."""
    from paper_2409_17033_gb300 import _lib
    p = c1
    H, A = f32(p.H), f32(p.A[None])
    for tf in (0.0, 1e-2):
        chi_n, D_n, i_n = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode="bf16_tail",
                                                 want_density=True, tail_f=tf)
        chi_x, D_x, i_x = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode="bf16x2",
                                                 want_density=True,
                                                 tail_f=tf if tf > 0 else _lib.DEFAULT_TAIL_F)
        assert i_n["converged"] and 0 < i_n["tail_single_steps"] < i_n["M"]
        assert i_n["sigma"] == i_x["sigma"] and i_n["tail_single_steps"] == i_x["tail_single_steps"]
        assert torch.equal(chi_n, chi_x) and torch.equal(D_n, D_x)
