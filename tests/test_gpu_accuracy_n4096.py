"""Accuracy of every arithmetic mode on the N=4096 tight-binding workload
(1024 sites x 4 orbitals, N_occ = 2048; 4 diagonal observables, 64 diagonal
site-potential perturbations) against the exact closed forms of the oracle:
D = theta(mu I - H) and the Daleckii-Krein / Loewner form of chi^A (Sec. II,
Appendix), and a1[l, k] = Tr[chi_l H1_k] (Eq. dual).

Tolerances: the stated per-mode constants times the conditioning measure
u * kappa (D) and u * kappa * N (chi, a1) of tests/tolerances.py, kappa being
the spectral width over the HOMO-LUMO gap (5.5e-3 against a width of about
31.5 here, kappa = 5.7e3). chi carries a 1/gap amplification of the
per-product rounding: plain FP32 products end near 0.5 in chi. FP16X2 (hi +
2^-11 lo, FP32 accumulation in 256-wide chunks) and BF16X3 reach 3e-3, two
orders better; the precision-floor stop returns the iterate with the smallest
idempotency error, on which the near-gap response terms depend. BF16X2 (~16
bits) cannot resolve the gap: its chi bound exceeds 1 at this size, and its D
error is 2e-2; that is reported, not hidden.
"""
import numpy as np
import pytest
import torch

import tolerances
import workloads
from oracle import exact

pytestmark = pytest.mark.gpu

N = 4096


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2409_17033_gb300 as p
    return p


@pytest.fixture(scope="module")
def ref():
    tb = workloads.tight_binding(N, seed=0, dtype=np.float32)
    H = tb.H.astype(np.float64)
    e, V = exact.eigh(H)
    A = workloads.tb_dipole_observables(tb)                 # (4, N) diagonals
    v = workloads.tb_site_potentials(tb, 64, seed=1)        # (64, N) diagonals
    D = exact.density_zero_T(e, V, tb.nocc)
    chi = np.stack([exact.response_zero_T(e, V, tb.nocc, np.diag(a)) for a in A])
    a1 = np.einsum("li,ki->lk", np.diagonal(chi, axis1=1, axis2=2), v)
    return tb, A, v, D, chi, a1, e[tb.nocc] - e[tb.nocc - 1], e


MEASURED = {   # rel err D, chi (4 observables), a1 (4 x 64) at N=4096, for the record
    "fp32": (6.5e-5, 4.7e-1, 5.3e-1),
    "fp16x2": (7.7e-6, 3.0e-3, 1.8e-3),
    "bf16x2": (1.9e-2, 1.05, 1.15),
    "bf16x3": (8.2e-6, 3.0e-3, 1.8e-3),
}
ERRS = {}


@pytest.mark.parametrize("mode", ["fp32", "fp16x2", "bf16x2", "bf16x3"])
def test_mode_against_exact(pkg, ref, mode):
    tb, A, v, D_ex, chi_ex, a1_ex, gap, e_ref = ref
    H = torch.from_numpy(tb.H).cuda()
    chi, D, info = pkg.sp2_susceptibility(H, tb.nocc, torch.from_numpy(A.astype(np.float32)).cuda(),
                                          "backward", diag_only=True, mode=mode, want_density=True)
    a1 = pkg.response_contract(chi, torch.from_numpy(v.astype(np.float32)).cuda(),
                               diag_only=True).cpu().numpy()
    eD = rel(D.cpu().numpy(), D_ex)
    eC = rel(chi.cpu().numpy(), chi_ex)
    eA = rel(a1, a1_ex)
    per = " ".join(f"{rel(chi[l].cpu().numpy(), chi_ex[l]):.1e}" for l in range(len(A)))
    print(f"N=4096 {mode}: M={info['M']} gap={gap:.2e} rel err D {eD:.2e} chi {eC:.2e} "
          f"(per observable {per}) a1 {eA:.2e}")
    ERRS[mode] = (eD, eC, eA)
    assert info["converged"]
    kap = tolerances.kappa(e_ref, tb.nocc)
    bD, bC = tolerances.tol_d(mode, kap), tolerances.tol_chi(mode, kap, N)
    print(f"  kappa={kap:.3g}: bounds D {bD:.2e} chi/a1 {bC:.2e}"
          + ("  (chi bound > 1: the mode cannot resolve this gap)" if bC > 1 else ""))
    assert eD < bD
    assert eC < bC
    assert eA < bC


def test_fp16x2_at_least_as_accurate_as_fp32():
    """The split FP16 tensor-core products (Eq. MixPrecMult, FP32 accumulation in
    256-wide chunks) are no less accurate than plain FP32 CUDA-core products."""
    if "fp32" not in ERRS or "fp16x2" not in ERRS:
        pytest.skip("needs the fp32 and fp16x2 cases of this module")
    assert all(a <= b for a, b in zip(ERRS["fp16x2"], ERRS["fp32"]))


def test_fp64_against_exact_and_duality(pkg, ref):
    """FP64: D and chi of the x-dipole to 1e-10 of the closed forms, and the
    primal responses of two perturbations agree with the dual contraction
    Tr[A D1_k] = Tr[chi^A H1_k] (Eq. Equivalence) to 1e-10."""
    tb, A, v, D_ex, chi_ex, a1_ex, _, _ = ref
    H = torch.from_numpy(tb.H.astype(np.float64)).cuda()
    Ad = torch.from_numpy(A[0:1]).cuda()
    chi, D, info = pkg.sp2_susceptibility(H, tb.nocc, Ad, "backward", diag_only=True, mode="fp64",
                                          want_density=True)
    eD = rel(D.cpu().numpy(), D_ex)
    eC = rel(chi[0].cpu().numpy(), chi_ex[0])
    vd = torch.from_numpy(v[0:2]).cuda()
    a_dual = pkg.response_contract(chi, vd, diag_only=True).cpu().numpy()[0]
    D1, _, _ = pkg.sp2_response(H, tb.nocc, vd, diag_only=True, mode="fp64",
                                sigma=info["sigma"], bounds=(info["eps_min"], info["eps_max"]))
    a_prim = pkg.response_contract(D1, Ad, diag_only=True).cpu().numpy()[:, 0]
    print(f"N=4096 fp64: M={info['M']} rel err D {eD:.2e} chi {eC:.2e} "
          f"a1 {rel(a_dual, a1_ex[0, :2]):.2e} primal/dual {rel(a_prim, a_dual):.2e}")
    assert eD < 1e-10 and eC < 1e-10
    assert rel(a_dual, a1_ex[0, :2]) < 1e-10
    assert rel(a_prim, a_dual) < 1e-10
