"""Finite-temperature path (Sec. V.B) on the GPU against the FP64 oracle.

Tolerances: FP64 1e-10 against the oracle's recursion with the same number
of doublings (D and every response); FP32 / split modes: D 1e-4 and
responses 1e-2 (the recursion halves nothing it starts from, so the
relative rounding of each product carries through all n doublings).
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import exact, fermi

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2409_17033_gb300 as p
    return p


@pytest.fixture(scope="module")
def metal():
    return workloads.metallic_spectrum(200, k=3, seed=2)


def cuda(x, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()


@pytest.mark.parametrize("canonical", [False, True])
def test_fp64_matches_oracle_recursion(pkg, metal, canonical):
    p = metal
    n, kT, mu = 14, 0.05, 0.05
    D1, D, info = pkg.sp2_fermi(cuda(p.H), mu, kT, cuda(p.H1), canonical=canonical,
                                n_doublings=n, mode="fp64")
    Dr, Rr = fermi.fermi_recursion(p.H, mu, kT, n, p.H1, canonical=canonical)
    assert info["M"] == n
    assert rel(D.cpu().numpy(), Dr) < 1e-10
    for k in range(3):
        assert rel(D1[k].cpu().numpy(), Rr[k]) < 1e-10
    if canonical:
        assert all(abs(float(torch.trace(D1[k]))) < 1e-9 for k in range(3))


def test_fp64_against_exact_fermi_dirac(pkg, metal):
    """n = 20 doublings: the exact Fermi-Dirac density and Daleckii-Krein response."""
    p = metal
    kT, mu = 0.05, 0.0
    D1, D, _ = pkg.sp2_fermi(cuda(p.H), mu, kT, cuda(p.H1[:2]), canonical=True, n_doublings=20,
                             mode="fp64")
    f = exact.fermi(p.e, mu, kT)
    assert rel(D.cpu().numpy(), (p.Q * f) @ p.Q.T) < 1e-9
    for k in range(2):
        ref = exact.response_fermi(p.e, p.Q, mu, kT, p.H1[k], canonical=True)
        assert rel(D1[k].cpu().numpy(), ref) < 1e-8


def test_finite_temperature_duality(pkg, metal):
    """Eq. Equivalence at finite T: Tr[A D1(H1_k)] = Tr[chi^A H1_k]."""
    p = metal
    kw = dict(canonical=True, n_doublings=16, mode="fp64", want_density=False)
    chi, _, _ = pkg.sp2_fermi(cuda(p.H), 0.0, 0.05, cuda(p.A[None]), **kw)
    D1, _, _ = pkg.sp2_fermi(cuda(p.H), 0.0, 0.05, cuda(p.H1), **kw)
    a_dual = pkg.response_contract(chi, cuda(p.H1)).cpu().numpy()[0]
    a_dir = pkg.response_contract(cuda(p.A[None]), D1).cpu().numpy()[0]
    assert np.allclose(a_dual, a_dir, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("mode", ["fp32", "bf16x2", "fp16x2"])
def test_low_precision_modes(pkg, metal, mode):
    p = metal
    n, kT = 14, 0.05
    D1, D, _ = pkg.sp2_fermi(cuda(p.H, torch.float32), 0.0, kT, cuda(p.H1, torch.float32),
                             canonical=True, n_doublings=n, mode=mode)
    Dr, Rr = fermi.fermi_recursion(p.H, 0.0, kT, n, p.H1, canonical=True)
    assert rel(D.double().cpu().numpy(), Dr) < 1e-4
    for k in range(3):
        assert rel(D1[k].double().cpu().numpy(), Rr[k]) < 1e-2


def test_diagonal_perturbations_ragged_and_empty(pkg):
    p = workloads.metallic_spectrum(77, k=0, seed=4)
    v = np.random.default_rng(0).uniform(-1, 1, (2, 77))
    D1, D, _ = pkg.sp2_fermi(cuda(p.H), 0.0, 0.1, cuda(v), diag_only=True, n_doublings=12,
                             mode="fp64")
    _, Rr = fermi.fermi_recursion(p.H, 0.0, 0.1, 12, np.stack([np.diag(x) for x in v]))
    for k in range(2):
        assert rel(D1[k].cpu().numpy(), Rr[k]) < 1e-10
    _, D0, _ = pkg.sp2_fermi(cuda(p.H), 0.0, 0.1, None, n_doublings=12, mode="fp64")
    assert rel(D0.cpu().numpy(), D.cpu().numpy()) < 1e-14


def test_too_few_doublings_rejected(pkg, metal):
    from paper_2409_17033_gb300 import _lib
    with pytest.raises(pkg.SP2Error) as e:
        pkg.sp2_fermi(cuda(metal.H), 0.0, 0.001, None, n_doublings=2, mode="fp64")
    assert e.value.code == _lib.EINVAL
