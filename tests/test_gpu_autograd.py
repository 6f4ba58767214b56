"""Autograd wrapper: forward = SP2 density (Eq. DM0), backward = adjoint
susceptibility (Eq. DM2), checked by central finite differences at N=512 on
the tight-binding construction, and against the oracle."""
import numpy as np
import pytest
import torch

import workloads
from oracle import exact
from oracle import sp2 as osp2

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2409_17033_gb300 as p
    return p


@pytest.fixture(scope="module")
def tb512():
    tb = workloads.tight_binding(512, seed=0)
    A = np.diag(workloads.tb_dipole_observables(tb)[0])
    return tb, A


def test_gradient_is_susceptibility_fp64(pkg, tb512):
    tb, A = tb512
    H = torch.from_numpy(tb.H).cuda().requires_grad_(True)
    At = torch.from_numpy(A).cuda()
    D = pkg.sp2_density_autograd(H, tb.nocc, mode="fp64", ckpt_k=4)
    loss = (D * At).sum()
    loss.backward()
    g = H.grad.cpu().numpy()
    e, V = exact.eigh(tb.H)
    assert rel(g, exact.response_zero_T(e, V, tb.nocc, A)) < 1e-8
    # the oracle's backward recursion run with the GPU's branch sequence
    _, info = pkg.sp2_density(H.detach(), tb.nocc, mode="fp64")
    o = osp2.sp2_density(tb.H, tb.nocc, sigma=info["sigma"], keep=True)
    assert rel(g, osp2.susceptibility_backward(o.X, o.sigma, o.beta, A)) < 1e-10


def test_gradient_matches_central_differences(pkg, tb512):
    """d Tr[A D(H + h E)]/dh at h=0 along random symmetric directions E equals
    sum(grad * E); the differences use the forward pass with its branch
    sequence and spectral bounds frozen, so both follow one polynomial."""
    tb, A = tb512
    H = torch.from_numpy(tb.H).cuda().requires_grad_(True)
    At = torch.from_numpy(A).cuda()
    D = pkg.sp2_density_autograd(H, tb.nocc, mode="fp64", ckpt_k=3)
    (D * At).sum().backward()
    g = H.grad.cpu().numpy()
    _, info = pkg.sp2_density(H.detach(), tb.nocc, mode="fp64")
    sig, bounds = info["sigma"], (info["eps_min"], info["eps_max"])
    rng = np.random.default_rng(0)
    h = 1e-4
    for _ in range(3):
        E = workloads.sym_gaussian(rng, 512, 1.0 / np.sqrt(512))
        Et = torch.from_numpy(E).cuda()
        Dp, _ = pkg.sp2_density(H.detach() + h * Et, tb.nocc, mode="fp64", sigma=sig, bounds=bounds)
        Dm, _ = pkg.sp2_density(H.detach() - h * Et, tb.nocc, mode="fp64", sigma=sig, bounds=bounds)
        fd = float(((Dp - Dm) * At).sum().item()) / (2 * h)
        an = float(np.sum(g * E))
        assert fd == pytest.approx(an, rel=1e-6, abs=1e-9)


def test_gradient_split_precision(pkg, tb512):
    """FP16X2 forward + adjoint: the gradient against the exact susceptibility,
    within the split-precision tolerance, and equal to the backward
    sp2_susceptibility of the same observable."""
    tb, A = tb512
    H = torch.from_numpy(tb.H).float().cuda().requires_grad_(True)
    At = torch.from_numpy(A).float().cuda()
    D = pkg.sp2_density_autograd(H, tb.nocc, mode="fp16x2", ckpt_k=4)
    (D * At).sum().backward()
    g = H.grad.double().cpu().numpy()
    e, V = exact.eigh(tb.H)
    assert rel(g, exact.response_zero_T(e, V, tb.nocc, A)) < 1e-3
    chi, _, _ = pkg.sp2_susceptibility(H.detach(), tb.nocc, At[None], "backward", mode="fp16x2",
                                       ckpt_k=4)
    assert rel(g, chi[0].double().cpu().numpy()) < 1e-6
