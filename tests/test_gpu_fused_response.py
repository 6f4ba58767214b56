"""The fused response step (sp2_set_option SP2_OPTION_FUSED_RESPONSE): with X
and Y symmetric, Y X + X Y over an upper tile (I, J) is one accumulation
[Y(I,:) | X(I,:)] . [X(:,J) ; Y(:,J)], and the branch update of Eqs. DM1 / DM2 /
DM3 runs in the product's epilogue (EPI_SYMM). Checked against the oracle's
emulation of the split products on the same planes (one step), against the
closed forms (converged), against the unfused path, and on stacked batches of
ragged size (tiles of several batch entries, straddling the diagonal)."""
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
def fused(sp2):
    h = sp2.Handle()
    h.set_option("fused_response", 1)
    return h


@pytest.fixture(scope="module")
def c1():
    return workloads.random_spectrum(128, nocc=64, k=3, seed=0)


def f32(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


@pytest.mark.parametrize("mode", ["bf16x2", "fp16x2", "bf16x3"])
def test_single_fused_step_matches_emulated_split(sp2, fused, c1, mode):
    p = c1
    H = f32(p.H)
    for s in (1, -1):
        chi, _, info = sp2.sp2_susceptibility(H, p.nocc, f32(p.A[None]), "forward", mode=mode,
                                              sigma=[s], handle=fused)
        a, b = info["alpha"], info["beta"]
        X1 = (a * np.eye(128) + b * p.H.astype(np.float32).astype(np.float64)).astype(np.float32)
        Y1 = (b * p.A.astype(np.float32).astype(np.float64)).astype(np.float32)
        if mode == "bf16x3":
            Z = split.mixed_product3(Y1, X1)
        elif mode == "fp16x2":
            sy = split.pow2_scale(float(np.max(np.abs(Y1))))
            Z = split.mixed_product(Y1, X1, "fp16", lo_scale=2048.0, sx=sy)
        else:
            Z = split.mixed_product(Y1, X1, "bf16")
        P = Z + Z.T
        ref = P if s > 0 else 2.0 * Y1.astype(np.float64) - P
        got = chi[0].cpu().numpy()
        assert rel(got, ref) < (2e-6 if mode == "bf16x2" else 1e-6)
        assert np.array_equal(got, got.T)


@pytest.mark.parametrize("mode", ["bf16x2", "fp16x2", "bf16x3"])
def test_fused_converged_against_closed_forms_and_unfused(sp2, fused, c1, mode):
    p = c1
    H = f32(p.H)
    A = f32(p.A[None])
    tolD, tolC = (1e-4, 1e-2) if mode == "bf16x2" else (3e-5, 1e-3)
    chi_b, D, info = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode=mode,
                                            want_density=True, handle=fused)
    chi_f, _, _ = sp2.sp2_susceptibility(H, p.nocc, A, "forward", mode=mode, handle=fused)
    D1, _, _ = sp2.sp2_response(H, p.nocc, f32(p.H1), mode=mode, handle=fused)
    assert info["converged"]
    chi_ex = exact.response_zero_T(p.e, p.Q, p.nocc, p.A)
    assert rel(D.cpu().numpy(), exact.density_zero_T(p.e, p.Q, p.nocc)) < tolD
    assert rel(chi_b[0].cpu().numpy(), chi_ex) < tolC
    assert rel(chi_f[0].cpu().numpy(), chi_ex) < tolC
    for k in range(3):
        assert rel(D1[k].cpu().numpy(), exact.response_zero_T(p.e, p.Q, p.nocc, p.H1[k])) < tolC
    # the unfused path computes the same sums in another order
    chi_u, _, info_u = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode=mode)
    assert info_u["sigma"] == info["sigma"]
    assert rel(chi_b[0].cpu().numpy(), chi_u[0].cpu().numpy()) < (1e-3 if mode == "bf16x2" else 1e-5)


@pytest.mark.parametrize("n", [130, 300])
def test_fused_batches_of_ragged_size(sp2, fused, n):
    """Stacked batches (three perturbations, two observables) at sizes that are
    not a multiple of the 256 padding: every batch entry's upper tiles, the
    mirror within its own matrix, and the per-entry FP16 plane scales."""
    p = workloads.random_spectrum(n, nocc=n // 2, k=3, seed=1)
    H = f32(p.H)
    D1, _, info = sp2.sp2_response(H, p.nocc, f32(p.H1), mode="fp16x2", handle=fused)
    assert info["converged"]
    for k in range(3):
        ref = exact.response_zero_T(p.e, p.Q, p.nocc, p.H1[k])
        assert rel(D1[k].cpu().numpy(), ref) < 1e-3
        assert np.array_equal(D1[k].cpu().numpy(), D1[k].cpu().numpy().T)
    A2 = np.stack([p.A, p.H1[0]])
    chi, _, _ = sp2.sp2_susceptibility(H, p.nocc, f32(A2), "backward", mode="fp16x2",
                                       handle=fused)
    for l in range(2):
        assert rel(chi[l].cpu().numpy(), exact.response_zero_T(p.e, p.Q, p.nocc, A2[l])) < 1e-3
