"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative Frobenius norm unless stated):
  FP64 mode      1e-10 against the oracle for D, chi, D1 and a1.
  FP32 mode      D 1e-5, chi / D1 / a1 1e-3 (single-precision products).
  BF16X2 mode    one product against the oracle's emulation of the same split
                 products (Eq. MixPrecMult in FP64): 2e-6 (FP32 accumulation
                 only); converged D 1e-4, chi / D1 / a1 1e-2 against the
                 exact closed forms (hi+lo carries ~16 significant bits).
  FP16X2 mode    one product 1e-6 against the emulation; converged D 3e-5,
                 chi / D1 / a1 1e-3 (hi+lo carries ~22 bits; the tensor-core
                 accumulation is drained to FP32 registers every K chunk).
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import exact, split
from oracle import sp2 as osp2

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def sp2():
    import __graft_entry__ as g
    g.build()
    import paper_2409_17033_gb300 as pkg
    assert torch.cuda.is_available()
    return pkg


@pytest.fixture(scope="module")
def c1():
    p = workloads.random_spectrum(128, nocc=64, k=8, seed=0)
    o = osp2.sp2_density(p.H, p.nocc, idem_tol=1e-10, keep=True)
    return p, o


def cuda(x, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()


def host(t):
    return t.double().cpu().numpy()


# ------------------------------------------------------------------ FP64
def test_fp64_density_matches_oracle(sp2, c1):
    p, o = c1
    D, info = sp2.sp2_density(cuda(p.H), p.nocc, mode="fp64", idem_tol=1e-10)
    assert info["converged"]
    assert info["sigma"] == o.sigma and info["M"] == o.M
    assert info["alpha"] == pytest.approx(o.alpha, rel=1e-14)
    assert info["beta"] == pytest.approx(o.beta, rel=1e-14)
    assert rel(host(D), o.D) < 1e-10
    assert rel(host(D), exact.density_zero_T(p.e, p.Q, p.nocc)) < 1e-10
    assert info["trace"] == pytest.approx(p.nocc, abs=1e-8)
    for a, b in zip(info["errors"], o.errors):
        assert a == pytest.approx(b, rel=1e-8, abs=1e-12)
    for a, b in zip(info["idem_fro"], o.fro):
        assert a == pytest.approx(b, rel=1e-6, abs=1e-20)


def test_fp64_susceptibility_forward_backward(sp2, c1):
    p, o = c1
    A = cuda(p.A[None])
    chi_f, D, inf_f = sp2.sp2_susceptibility(cuda(p.H), p.nocc, A, "forward", mode="fp64",
                                             idem_tol=1e-10, want_density=True)
    chi_b, _, inf_b = sp2.sp2_susceptibility(cuda(p.H), p.nocc, A, "backward", mode="fp64",
                                             idem_tol=1e-10, ckpt_k=3)
    ref = osp2.susceptibility_forward(o.X, o.sigma, o.beta, p.A)
    assert inf_f["sigma"] == o.sigma and inf_b["sigma"] == o.sigma
    assert rel(host(chi_f[0]), ref) < 1e-10
    assert rel(host(chi_b[0]), ref) < 1e-10
    assert rel(host(chi_b[0]), exact.response_zero_T(p.e, p.Q, p.nocc, p.A)) < 1e-8
    assert rel(host(D), o.D) < 1e-10


@pytest.mark.parametrize("k", [1, 2, 4, 7, 40])
def test_fp64_backward_checkpoint_segments(sp2, c1, k):
    """Every checkpoint spacing (1 = all X_n kept; > M = one segment) gives
    the same adjoint."""
    p, o = c1
    chi_b, _, _ = sp2.sp2_susceptibility(cuda(p.H), p.nocc, cuda(p.A[None]), "backward",
                                         mode="fp64", idem_tol=1e-10, ckpt_k=k)
    ref = osp2.susceptibility_backward(o.X, o.sigma, o.beta, p.A)
    assert rel(host(chi_b[0]), ref) < 1e-10


@pytest.mark.parametrize("mode", ["bf16x2", "fp16x2", "bf16x3", "fp32"])
def test_checkpoint_policies_agree_bitwise(sp2, c1, mode):
    """Keeping every X_n (split modes: its hi/lo planes), every 3rd with segment
    recompute, and the memory-sized automatic choice run the same products on
    the same operands, so chi is bit-identical; at N=128 the automatic choice
    keeps every step."""
    p, _ = c1
    H = cuda(p.H, torch.float32)
    A = cuda(p.A[None], torch.float32)
    out = {}
    for k in (1, 3, "auto"):
        chi, _, info = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode=mode, ckpt_k=k)
        out[k] = (chi, info)
    assert out["auto"][1]["ckpt_k"] == 1 and out[3][1]["ckpt_k"] == 3
    assert torch.equal(out[1][0], out[3][0])
    assert torch.equal(out[1][0], out["auto"][0])


def test_fp64_response_batch_and_duality(sp2, c1):
    p, o = c1
    D1, _, info = sp2.sp2_response(cuda(p.H), p.nocc, cuda(p.H1), mode="fp64", idem_tol=1e-10)
    for k in range(p.H1.shape[0]):
        ref = osp2.dm_response(o.X, o.sigma, o.beta, p.H1[k])
        assert rel(host(D1[k]), ref) < 1e-10
    chi, _, _ = sp2.sp2_susceptibility(cuda(p.H), p.nocc, cuda(p.A[None]), "forward",
                                       mode="fp64", idem_tol=1e-10)
    a_dual = host(sp2.response_contract(chi, cuda(p.H1)))[0]
    a_dir = host(sp2.response_contract(cuda(p.A[None]), D1))[0]
    assert np.allclose(a_dual, a_dir, rtol=1e-11, atol=1e-13)  # Eq. Equivalence
    chi_o = osp2.susceptibility_forward(o.X, o.sigma, o.beta, p.A)
    a_ref = osp2.contract(chi_o[None], p.H1)[0]
    assert rel(a_dual, a_ref) < 1e-10


def test_fp64_fixed_branches_unconverged(sp2, c1):
    """A preset branch sequence (not converged) reproduces the finite-M
    eigenvalue reference: the GPU polynomial is the oracle's, step by step."""
    p, _ = c1
    sig = [1, -1, -1, 1, 1, -1, 1]
    D, info = sp2.sp2_density(cuda(p.H), p.nocc, mode="fp64", sigma=sig)
    assert info["M"] == len(sig) and info["sigma"] == sig
    D_ref, (Y_ref,) = exact.finite_m_reference(p.e, p.Q, info["alpha"], info["beta"], sig, p.A)
    assert rel(host(D), D_ref) < 1e-12
    chi, _, _ = sp2.sp2_susceptibility(cuda(p.H), p.nocc, cuda(p.A[None]), "forward",
                                       mode="fp64", sigma=sig)
    assert rel(host(chi[0]), Y_ref) < 1e-11


# ------------------------------------------------------------------ FP32
def test_fp32_against_oracle(sp2, c1):
    p, o = c1
    H = cuda(p.H, torch.float32)
    chi, D, info = sp2.sp2_susceptibility(H, p.nocc, cuda(p.A[None], torch.float32), "backward",
                                          mode="fp32", want_density=True)
    assert info["converged"]
    assert rel(host(D), exact.density_zero_T(p.e, p.Q, p.nocc)) < 1e-5
    assert rel(host(chi[0]), exact.response_zero_T(p.e, p.Q, p.nocc, p.A)) < 1e-3
    D1, _, _ = sp2.sp2_response(H, p.nocc, cuda(p.H1, torch.float32), mode="fp32")
    for k in range(3):
        assert rel(host(D1[k]), exact.response_zero_T(p.e, p.Q, p.nocc, p.H1[k])) < 1e-3


# ------------------------------------------------------------------ BF16X2 (tcgen05)
def test_bf16x2_single_square_step_matches_emulated_split(sp2, c1):
    """One product kernel launch: X_2 = X_1^2 (sigma=+1) or 2 X_1 - X_1^2, with
    X_1 = alpha I + beta H in FP32, against Eq. MixPrecMult evaluated in FP64."""
    p, _ = c1
    H = cuda(p.H, torch.float32)
    for s in (1, -1):
        D, info = sp2.sp2_density(H, p.nocc, mode="bf16x2", sigma=[s])
        a, b = info["alpha"], info["beta"]
        X1 = (a * np.eye(128) + b * p.H.astype(np.float32).astype(np.float64)).astype(np.float32)
        P = split.mixed_product(X1, X1, "bf16")
        ref = P if s > 0 else 2.0 * X1.astype(np.float64) - P
        assert rel(host(D), ref) < 2e-6
        assert np.array_equal(host(D), host(D).T)


def test_bf16x2_single_response_step_matches_emulated_split(sp2, c1):
    p, _ = c1
    H = cuda(p.H, torch.float32)
    for s in (1, -1):
        chi, _, info = sp2.sp2_susceptibility(H, p.nocc, cuda(p.A[None], torch.float32), "forward",
                                              mode="bf16x2", sigma=[s])
        a, b = info["alpha"], info["beta"]
        X1 = (a * np.eye(128) + b * p.H.astype(np.float32).astype(np.float64)).astype(np.float32)
        Y1 = (b * p.A.astype(np.float32).astype(np.float64)).astype(np.float32)
        Z = split.mixed_product(Y1, X1, "bf16")
        P = Z + Z.T
        ref = P if s > 0 else 2.0 * Y1.astype(np.float64) - P
        assert rel(host(chi[0]), ref) < 2e-6


def test_fp16x2_single_steps_match_emulated_split(sp2, c1):
    """FP16X2: one square step and one response step against Eq. MixPrecMult on
    fp16 planes (lo scaled by 2^11, Y with its power-of-two plane scale)."""
    p, _ = c1
    H = cuda(p.H, torch.float32)
    for s in (1, -1):
        D, info = sp2.sp2_density(H, p.nocc, mode="fp16x2", sigma=[s])
        a, b = info["alpha"], info["beta"]
        X1 = (a * np.eye(128) + b * p.H.astype(np.float32).astype(np.float64)).astype(np.float32)
        P = split.mixed_product(X1, X1, "fp16", lo_scale=2048.0)
        ref = P if s > 0 else 2.0 * X1.astype(np.float64) - P
        assert rel(host(D), ref) < 1e-6
        chi, _, _ = sp2.sp2_susceptibility(H, p.nocc, cuda(p.A[None], torch.float32), "forward",
                                           mode="fp16x2", sigma=[s])
        Y1 = (b * p.A.astype(np.float32).astype(np.float64)).astype(np.float32)
        sy = split.pow2_scale(float(np.max(np.abs(Y1))))
        Z = split.mixed_product(Y1, X1, "fp16", lo_scale=2048.0, sx=sy)
        Pz = Z + Z.T
        ref = Pz if s > 0 else 2.0 * Y1.astype(np.float64) - Pz
        assert rel(host(chi[0]), ref) < 1e-6


def test_bf16x3_single_steps_match_emulated_split(sp2, c1):
    """BF16X3: one square step and one response step against the six-term
    product of the three-plane split (hi + mid + lo) evaluated in FP64. What
    remains is the FP32 accumulation, which the 256-wide chunks keep near the
    FP32 rounding of the result."""
    p, _ = c1
    H = cuda(p.H, torch.float32)
    for s in (1, -1):
        D, info = sp2.sp2_density(H, p.nocc, mode="bf16x3", sigma=[s])
        a, b = info["alpha"], info["beta"]
        X1 = (a * np.eye(128) + b * p.H.astype(np.float32).astype(np.float64)).astype(np.float32)
        P = split.mixed_product3(X1, X1)
        ref = P if s > 0 else 2.0 * X1.astype(np.float64) - P
        assert rel(host(D), ref) < 1e-6
        assert np.array_equal(host(D), host(D).T)
        chi, _, _ = sp2.sp2_susceptibility(H, p.nocc, cuda(p.A[None], torch.float32), "forward",
                                           mode="bf16x3", sigma=[s])
        Y1 = (b * p.A.astype(np.float32).astype(np.float64)).astype(np.float32)
        Z = split.mixed_product3(Y1, X1)
        Pz = Z + Z.T
        ref = Pz if s > 0 else 2.0 * Y1.astype(np.float64) - Pz
        assert rel(host(chi[0]), ref) < 1e-6


def test_fp16x2_large_response_entries_do_not_overflow(sp2, c1):
    """Observables with entries far beyond the FP16 range (1e6) still give the
    exact response up to the split precision (per-matrix plane scales)."""
    p, _ = c1
    H = cuda(p.H, torch.float32)
    A = p.A * 1e6
    chi, _, info = sp2.sp2_susceptibility(H, p.nocc, cuda(A[None], torch.float32), "backward",
                                          mode="fp16x2")
    c = host(chi[0])
    assert np.isfinite(c).all()
    assert rel(c, exact.response_zero_T(p.e, p.Q, p.nocc, A)) < 1e-3


@pytest.mark.parametrize("mode", ["bf16x2", "fp16x2", "bf16x3"])
def test_split_modes_converged_against_closed_forms(sp2, c1, mode):
    p, _ = c1
    H = cuda(p.H, torch.float32)
    A = cuda(p.A[None], torch.float32)
    tolD, tolC = (1e-4, 1e-2) if mode == "bf16x2" else (3e-5, 1e-3)
    chi_b, D, info = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode=mode, want_density=True)
    chi_f, _, _ = sp2.sp2_susceptibility(H, p.nocc, A, "forward", mode=mode)
    assert info["converged"]
    D_ex = exact.density_zero_T(p.e, p.Q, p.nocc)
    chi_ex = exact.response_zero_T(p.e, p.Q, p.nocc, p.A)
    assert rel(host(D), D_ex) < tolD
    assert rel(host(chi_b[0]), chi_ex) < tolC
    assert rel(host(chi_f[0]), chi_ex) < tolC
    D1, _, _ = sp2.sp2_response(H, p.nocc, cuda(p.H1, torch.float32), mode=mode)
    for k in range(3):
        assert rel(host(D1[k]), exact.response_zero_T(p.e, p.Q, p.nocc, p.H1[k])) < tolC


def test_bf16x2_converged_against_closed_forms(sp2, c1):
    p, _ = c1
    H = cuda(p.H, torch.float32)
    A = cuda(p.A[None], torch.float32)
    chi_b, D, info = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode="bf16x2",
                                            want_density=True)
    chi_f, _, _ = sp2.sp2_susceptibility(H, p.nocc, A, "forward", mode="bf16x2")
    assert info["converged"]
    D_ex = exact.density_zero_T(p.e, p.Q, p.nocc)
    chi_ex = exact.response_zero_T(p.e, p.Q, p.nocc, p.A)
    assert rel(host(D), D_ex) < 1e-4
    assert rel(host(chi_b[0]), chi_ex) < 1e-2
    assert rel(host(chi_f[0]), chi_ex) < 1e-2
    a = host(sp2.response_contract(chi_b, cuda(p.H1, torch.float32)))[0]
    a_ex = np.array([np.sum(chi_ex * h) for h in p.H1])
    assert rel(a, a_ex) < 1e-2


# ------------------------------------------------------------------ ragged sizes / edges
@pytest.mark.parametrize("n", [1, 17, 130, 300])
@pytest.mark.parametrize("mode", ["fp64", "bf16x2", "fp16x2", "bf16x3"])
def test_ragged_sizes(sp2, n, mode):
    nocc = max(1, n // 3) if n > 1 else 1
    p = workloads.random_spectrum(n, nocc=nocc, k=1, seed=n)
    dt = torch.float64 if mode == "fp64" else torch.float32
    chi, D, info = sp2.sp2_susceptibility(cuda(p.H, dt), p.nocc, cuda(p.A[None], dt), "backward",
                                          mode=mode, want_density=True,
                                          idem_tol=1e-10 if mode == "fp64" else 0.0)
    tolD, tolC = {"fp64": (1e-10, 1e-8), "bf16x2": (1e-4, 1e-2), "fp16x2": (3e-5, 1e-3),
                  "bf16x3": (3e-5, 1e-3)}[mode]
    assert rel(host(D), exact.density_zero_T(p.e, p.Q, p.nocc)) < tolD
    chi_ex = exact.response_zero_T(p.e, p.Q, p.nocc, p.A)
    if np.linalg.norm(chi_ex) > 0:
        assert rel(host(chi[0]), chi_ex) < tolC


def test_empty_and_trivial_occupations(sp2):
    D, info = sp2.sp2_density(torch.zeros((0, 0), dtype=torch.float64, device="cuda"), 0.0,
                              mode="fp64")
    assert D.shape == (0, 0) and info["M"] == 0
    p = workloads.random_spectrum(64, nocc=32, k=0, seed=3)
    for nocc, ref in ((0, np.zeros((64, 64))), (64, np.eye(64))):
        D, info = sp2.sp2_density(cuda(p.H), nocc, mode="fp64", idem_tol=1e-12)
        assert rel(host(D) + (1.0 if nocc == 0 else 0.0), ref + (1.0 if nocc == 0 else 0.0)) < 1e-10


def test_errors_are_reported(sp2):
    from paper_2409_17033_gb300 import _lib
    p = workloads.random_spectrum(64, nocc=32, k=0, seed=4)
    H = cuda(p.H)
    with pytest.raises(sp2.SP2Error) as e:
        sp2.sp2_density(H, 65.0, mode="fp64")
    assert e.value.code == _lib.EINVAL
    Hn = H.clone()
    Hn[3, 5] = float("nan")
    with pytest.raises(sp2.SP2Error) as e:
        sp2.sp2_density(Hn, 32.0, mode="fp64")
    assert e.value.code == _lib.ENONFINITE
    with pytest.raises(sp2.SP2Error) as e:
        sp2.sp2_density(H, 32.0, mode="fp64", idem_tol=1e-10, max_iter=3)
    assert e.value.code == _lib.ENOCONV
    h = sp2.Handle()
    with pytest.raises(sp2.SP2Error) as e:
        sp2.sp2_adjoint(H, h)
    assert e.value.code == _lib.ENOSTATE


def test_host_buffers_match_device_buffers(sp2, c1):
    p, _ = c1
    Hh = np.ascontiguousarray(p.H.astype(np.float32))
    Ah = np.ascontiguousarray(p.A[None].astype(np.float32))
    chi_h, D_h, _ = sp2.sp2_susceptibility(Hh, p.nocc, Ah, "backward", mode="bf16x2",
                                           want_density=True)
    chi_d, D_d, _ = sp2.sp2_susceptibility(cuda(Hh, torch.float32), p.nocc,
                                           cuda(Ah, torch.float32), "backward", mode="bf16x2",
                                           want_density=True)
    assert isinstance(chi_h, np.ndarray)
    assert np.array_equal(chi_h, chi_d.cpu().numpy())
    assert np.array_equal(D_h, D_d.cpu().numpy())
    # caller-owned page-locked result buffers receive the same values
    out = torch.empty((1, 128, 128), dtype=torch.float32).pin_memory().numpy()
    Dout = torch.empty((128, 128), dtype=torch.float32).pin_memory().numpy()
    chi_p, D_p, _ = sp2.sp2_susceptibility(Hh, p.nocc, Ah, "backward", mode="bf16x2",
                                           want_density=True, out=out, D_out=Dout)
    assert chi_p is out and D_p is Dout
    assert np.array_equal(out, chi_h) and np.array_equal(Dout, D_h)


def test_response_contract_dense_and_diagonal(sp2):
    rng = np.random.default_rng(0)
    for n in (5, 130):
        P = rng.standard_normal((3, n, n))
        Q = rng.standard_normal((4, n, n))
        q = rng.standard_normal((4, n))
        out = host(sp2.response_contract(cuda(P), cuda(Q)))
        ref = np.einsum("lij,kij->lk", P, Q)
        assert np.allclose(out, ref, rtol=1e-12, atol=1e-12)
        out = host(sp2.response_contract(cuda(P), cuda(q), diag_only=True))
        assert np.allclose(out, osp2.contract_diag(P, q), rtol=1e-12, atol=1e-12)
        o32 = host(sp2.response_contract(cuda(P, torch.float32), cuda(Q, torch.float32)))
        ref32 = np.einsum("lij,kij->lk", P.astype(np.float32).astype(np.float64),
                          Q.astype(np.float32).astype(np.float64))
        assert np.allclose(o32, ref32, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("case", ["f64_dense", "f32_diag", "f32_dense"])
def test_response_contract_beyond_65535_grid_rows(sp2, case):
    """More (observable, perturbation) work rows than one launch's gridDim.y
    (65535) holds: the rows go out in several launches, and every pair must
    equal the FP64 einsum of the same values."""
    rng = np.random.default_rng(5)
    if case == "f64_dense":
        L, K, n, diag, dt = 7, 10000, 16, False, torch.float64
    elif case == "f32_diag":
        L, K, n, diag, dt = 7, 10000, 16, True, torch.float32
    else:   # FP32 dense groups 8 perturbations per row: L * ceil(K / 8) rows
        L, K, n, diag, dt = 70000, 1, 8, False, torch.float32
    P = rng.standard_normal((L, n, n)).astype(np.float32).astype(np.float64)
    Q = rng.standard_normal((K, n) if diag else (K, n, n)).astype(np.float32).astype(np.float64)
    out = host(sp2.response_contract(cuda(P, dt), cuda(Q, dt), diag_only=diag))
    ref = (np.einsum("lii,ki->lk", P, Q) if diag else
           np.einsum("lij,kij->lk", P, Q))
    assert out.shape == (L, K)
    assert np.allclose(out, ref, rtol=1e-12, atol=1e-10)


def test_diagonal_perturbations(sp2):
    """Site-potential perturbations passed as diagonals equal the dense form."""
    tb = workloads.tight_binding(512, seed=0)
    v = workloads.tb_site_potentials(tb, 3, seed=1)
    D1d, _, info = sp2.sp2_response(cuda(tb.H), tb.nocc, cuda(v), diag_only=True, mode="fp64",
                                    idem_tol=1e-10)
    D1, _, _ = sp2.sp2_response(cuda(tb.H), tb.nocc, cuda(np.stack([np.diag(x) for x in v])),
                                mode="fp64", idem_tol=1e-10)
    assert rel(host(D1d), host(D1)) < 1e-13
    e, V = exact.eigh(tb.H)
    for k in range(3):
        assert rel(host(D1d[k]), exact.response_zero_T(e, V, tb.nocc, np.diag(v[k]))) < 1e-8
