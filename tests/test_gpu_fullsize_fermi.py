"""Finite-temperature path (Sec. V.B) at its full size: N=8192 gapless
spectrum e ~ U[-1, 1] with Haar eigenvectors, kT = 0.02, mu = 0, 20 doublings,
canonical responses, in the FP16X2 mode the bench times.

The eigensystem is known by construction (H = Q diag(e) Q^T), so the oracle's
closed forms need no eigensolver: the Fermi-Dirac density Q f(e) Q^T and the
Daleckii-Krein responses with the canonical mu_1. Checked on the observable
A (its chi^A) and the first two perturbations H1_0, H1_1 of the seeded host
generator, plus Eq. Equivalence between the primal Tr[A D1_k] and the dual
Tr[chi^A H1_k] contractions.

Tolerances: measured errors times about 3 (printed with -s).
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import exact

pytestmark = pytest.mark.gpu

N, KT, NDBL = 8192, 0.02, 20


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
def prob():
    p = workloads.metallic_spectrum(N, k=2, seed=0)
    f = exact.fermi(p.e, 0.0, KT)
    D = (p.Q * f) @ p.Q.T
    R = [exact.response_fermi(p.e, p.Q, 0.0, KT, b, canonical=True) for b in (p.A, p.H1[0], p.H1[1])]
    return p, D, R


def test_fp16x2_against_exact(pkg, prob):
    p, D_ex, R_ex = prob
    H = torch.from_numpy(p.H.astype(np.float32)).cuda()
    B = torch.from_numpy(np.stack([p.A, p.H1[0], p.H1[1]]).astype(np.float32)).cuda()
    R, D, info = pkg.sp2_fermi(H, 0.0, KT, B, canonical=True, n_doublings=NDBL, mode="fp16x2")
    eD = rel(D.cpu().numpy(), D_ex)
    eR = [rel(R[i].cpu().numpy(), R_ex[i]) for i in range(3)]
    tr = [abs(float(torch.trace(R[i].double()))) for i in range(3)]
    # Eq. Equivalence: primal Tr[A D1_k] against dual Tr[chi^A H1_k], and both against exact
    a_ex = np.array([np.sum(p.A * R_ex[k]) for k in (1, 2)])
    a_dual = pkg.response_contract(R[0:1], B[1:3]).cpu().numpy()[0]
    a_prim = pkg.response_contract(R[1:3], B[0:1]).cpu().numpy()[:, 0]
    print(f"N=8192 finite T fp16x2: rel err D {eD:.2e} chi^A {eR[0]:.2e} D1_0 {eR[1]:.2e} "
          f"D1_1 {eR[2]:.2e}; |Tr| {max(tr):.1e}; a1 primal {rel(a_prim, a_ex):.2e} "
          f"dual {rel(a_dual, a_ex):.2e} primal/dual {rel(a_prim, a_dual):.2e}")
    assert info["M"] == NDBL
    # measured: D 1.1e-4, responses 3.0e-4, |Tr| 1e-7, a1 1.3e-4, primal/dual 3.0e-6
    assert eD < 4e-4
    assert max(eR) < 1e-3
    assert max(tr) < 1e-5 * max(float(R[i].norm()) for i in range(3))
    assert rel(a_dual, a_ex) < 5e-4 and rel(a_prim, a_ex) < 5e-4
    assert rel(a_prim, a_dual) < 3e-5
