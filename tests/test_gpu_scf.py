"""Self-consistent response (Eq. DM_CP_SCF with a site-charge G) and the MLP
preconditioner kernels on the GPU, against the FP64 oracle.

Tolerances: FP64 response path 1e-8 for the SCF solution and its residual
history; the MLP kernels run in FP32: loss and gradients 1e-5 relative to
the FP64 oracle."""
import numpy as np
import pytest
import torch

import workloads
from oracle import exact, scf

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
def small():
    tb = workloads.tight_binding(256, seed=0)
    e, V = exact.eigh(tb.H)
    chi0 = scf.chi0_sites(e, V, tb.nocc, tb.norb)
    K = workloads.site_kernel(tb, "regularised")
    Vx = workloads.site_fields(tb, 6, seed=3)
    return tb, chi0, K, Vx


@pytest.mark.parametrize("mixer", ["linear", "anderson"])
def test_scf_fp64_matches_oracle(pkg, small, mixer):
    tb, chi0, K, Vx = small
    H = torch.from_numpy(tb.H).cuda()
    q, res, its, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, Vx, mixer=mixer, alpha=0.3, history=8,
                                          tol=1e-9, max_iter=300, mode="fp64", idem_tol=1e-13)
    q_or, res_or = scf.scf_iterate(chi0, K, Vx, mixer=mixer, alpha=0.3, hist=8, tol=1e-9,
                                   max_iter=300)
    assert rel(q, scf.scf_exact(chi0, K, Vx)) < 1e-7
    assert abs(its - len(res_or)) <= 1
    k = min(its, len(res_or))
    # Anderson's coefficients amplify rounding differences late in the run
    assert np.allclose(res[:k], res_or[:k], rtol=1e-6 if mixer == "linear" else 1e-3, atol=1e-10)


@pytest.mark.parametrize("net", ["random", "exact_correction"])
def test_scf_mlp_mixer_matches_oracle_step_by_step(pkg, small, net):
    """The learned mixer q <- q + alpha r + ||r|| MLP(r/||r||) on the GPU (FP64
    responses, FP32 network, no bfloat16) against the oracle's MLP branch of
    scf_iterate with the same weights, residual by residual. "random": a small
    random network (the mixer stays contractive); "exact_correction": the ReLU
    pair that represents (I - chi0 K)^(-1) - alpha I exactly, so the residual
    drops to the FP32 network's rounding in one step."""
    tb, chi0, K, Vx = small
    ns = chi0.shape[0]
    alpha = 0.3
    if net == "random":
        rng = np.random.default_rng(4)
        W1 = rng.standard_normal((32, ns)) / np.sqrt(ns)
        W2 = 0.05 * rng.standard_normal((ns, 32)) / np.sqrt(32)
        tol, cap = 1e-8, 200
    else:
        C = np.linalg.inv(np.eye(ns) - chi0 @ K) - alpha * np.eye(ns)
        W1 = np.vstack([np.eye(ns), -np.eye(ns)])
        W2 = np.hstack([C, -C])
        tol, cap = 1e-5, 10
    W1 = W1.astype(np.float32)
    W2 = W2.astype(np.float32)
    H = torch.from_numpy(tb.H).cuda()
    q, res, its, _ = pkg.sp2_scf_response(
        H, tb.nocc, 4, K, Vx, mixer="mlp", alpha=alpha, tol=tol, max_iter=cap,
        W1=torch.from_numpy(W1).cuda(), W2=torch.from_numpy(W2).cuda(), bf16_infer=False,
        mode="fp64", idem_tol=1e-13)
    q_or, res_or = scf.scf_iterate(chi0, K, Vx, mixer="mlp", alpha=alpha, tol=tol, max_iter=cap,
                                   mlp=(W1.astype(np.float64), W2.astype(np.float64)))
    assert abs(its - len(res_or)) <= 1
    if net == "exact_correction":
        # one step to the solution on both sides; the remaining residual is each
        # side's rounding of the network (FP32 weights: ~1e-8 oracle, ~1e-7 GPU)
        assert its == 2 and len(res_or) == 2
        assert res[0] == pytest.approx(res_or[0], rel=1e-9)
        assert res[1] < 1e-6 and res_or[1] < 1e-6
    else:
        k = min(its, len(res_or))
        # the network runs in FP32 on the GPU: each step's correction carries ~1e-7
        assert np.allclose(res[:k], res_or[:k], rtol=1e-5, atol=1e-9)
    assert rel(q, q_or) < 1e-6


def test_scf_anderson_with_learned_step_matches_oracle(pkg, small):
    """Anderson with the learned step as its preconditioner on the GPU (FP64
    responses, FP32 network) against the oracle's anderson_mlp branch with the
    same weights, residual by residual; Anderson's coefficients amplify the
    FP32 network's rounding late in the run, as for plain Anderson."""
    tb, chi0, K, Vx = small
    ns = chi0.shape[0]
    rng = np.random.default_rng(6)
    W1 = (rng.standard_normal((32, ns)) / np.sqrt(ns)).astype(np.float32)
    W2 = (0.05 * rng.standard_normal((ns, 32)) / np.sqrt(32)).astype(np.float32)
    H = torch.from_numpy(tb.H).cuda()
    q, res, its, _ = pkg.sp2_scf_response(
        H, tb.nocc, 4, K, Vx, mixer="anderson_mlp", alpha=0.3, history=8, tol=1e-9, max_iter=200,
        W1=torch.from_numpy(W1).cuda(), W2=torch.from_numpy(W2).cuda(), bf16_infer=False,
        mode="fp64", idem_tol=1e-13)
    q_or, res_or = scf.scf_iterate(chi0, K, Vx, mixer="anderson_mlp", alpha=0.3, hist=8, tol=1e-9,
                                   max_iter=200, mlp=(W1.astype(np.float64), W2.astype(np.float64)))
    assert abs(its - len(res_or)) <= 1
    k = min(its, len(res_or))
    assert np.allclose(res[:k], res_or[:k], rtol=1e-3, atol=1e-10)
    assert rel(q, scf.scf_exact(chi0, K, Vx)) < 1e-7


def test_scf_split_precision(pkg, small):
    tb, chi0, K, Vx = small
    H = torch.from_numpy(tb.H).float().cuda()
    q, res, its, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, Vx, mixer="anderson", tol=1e-5,
                                          max_iter=200, mode="fp16x2")
    assert res[-1] <= 1e-5
    assert rel(q, scf.scf_exact(chi0, K, Vx)) < 1e-3


def test_scf_precision_refinement(pkg, small):
    """Split FP16X2 responses do the first iterations; below 1e-4 (or on a stall)
    the loop switches to FP64 responses, whose own SP2 polynomial is converged
    once and fixed, and reaches a residual the split arithmetic cannot (1e-10),
    at the exact solution."""
    tb, chi0, K, Vx = small
    H = torch.from_numpy(tb.H).cuda()
    q, res, its, _, info = pkg.sp2_scf_response(H, tb.nocc, 4, K, Vx, mixer="anderson", tol=1e-10,
                                                max_iter=100, mode="fp16x2", refine_mode="fp64",
                                                refine_below=1e-4, return_info=True)
    assert res[-1] <= 1e-10
    assert 0 < info["refine_iter"] < its
    assert rel(q, scf.scf_exact(chi0, K, Vx)) < 1e-8
    _, res16, _, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, Vx, mixer="anderson", tol=1e-10,
                                          max_iter=40, mode="fp16x2", allow_noconv=True)
    assert min(res16) > 1e-10                # the split arithmetic alone floors above it


def test_scf_dual_on_gpu(pkg, small):
    """Eq. CP_SCF on the GPU: the response of the x, y, z site dipoles to 6
    fields, primal (one SCF solve per field) against dual (one SCF solve per
    observable, the observable as the field, then dot products), FP64, and
    both against the oracle's exact solve."""
    tb, chi0, K, Vx = small
    H = torch.from_numpy(tb.H).cuda()
    obs = np.ascontiguousarray((tb.pos - 0.5 * tb.box).T)
    kw = dict(mixer="anderson", alpha=0.3, tol=1e-12, max_iter=300, mode="fp64", idem_tol=1e-13)
    q_f, _, _, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, Vx, **kw)
    q_a, _, _, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, obs, **kw)
    primal = obs @ q_f.T
    dual = q_a @ Vx.T
    exact_ = obs @ scf.scf_exact(chi0, K, Vx).T
    assert rel(dual, primal) < 1e-9
    assert rel(primal, exact_) < 1e-8 and rel(dual, exact_) < 1e-8


def test_scf_finite_temperature(pkg, small):
    """Self-consistent response at finite temperature (Sec. V.B responses with
    the canonical mu_1 inside Eq. DM_CP_SCF) against the oracle's exact linear
    solve with the finite-T site susceptibility, FP64; and Eq. CP_SCF at finite
    T: primal (per field) and dual (per observable) agree."""
    tb, chi0, K, Vx = small
    e, V = exact.eigh(tb.H)
    mu = 0.5 * (e[tb.nocc - 1] + e[tb.nocc])
    kT = 0.05
    c0 = scf.chi0_sites_fermi(e, V, mu, kT, tb.norb, canonical=True)
    H = torch.from_numpy(tb.H).cuda()
    kw = dict(mixer="anderson", alpha=0.3, tol=1e-11, max_iter=200, mode="fp64", kT=kT, mu=mu,
              n_doublings=24)
    q, res, its, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, Vx, **kw)
    assert res[-1] <= 1e-11
    assert rel(q, scf.scf_exact(c0, K, Vx)) < 1e-7
    obs = np.ascontiguousarray((tb.pos - 0.5 * tb.box).T)
    q_a, _, _, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, obs, **kw)
    assert rel(q_a @ Vx.T, obs @ q.T) < 1e-9
    q16, res16, _, _ = pkg.sp2_scf_response(H.float(), tb.nocc, 4, K, Vx, mixer="anderson",
                                            tol=1e-5, max_iter=100, mode="fp16x2", kT=kT, mu=mu,
                                            n_doublings=24)
    assert res16[-1] <= 1e-5
    assert rel(q16, scf.scf_exact(c0, K, Vx)) < 1e-3


def test_mlp_kernels_against_oracle(pkg):
    rng = np.random.default_rng(0)
    din, dh, P = 96, 40, 70
    W1 = rng.standard_normal((dh, din)) / np.sqrt(din)
    W2 = rng.standard_normal((din, dh)) / np.sqrt(dh)
    X = rng.standard_normal((P, din))
    T = rng.standard_normal((P, din))
    f = lambda a: torch.from_numpy(a.astype(np.float32)).cuda()  # noqa: E731
    Y = pkg.mlp_forward(f(W1), f(W2), f(X)).cpu().numpy()
    W1f, W2f, Xf, Tf = (a.astype(np.float32).astype(np.float64) for a in (W1, W2, X, T))
    assert rel(Y, scf.mlp_forward(W1f, W2f, Xf)) < 1e-5
    L, g1, g2 = pkg.mlp_loss_grad(f(W1), f(W2), f(X), f(T))
    Lr, g1r, g2r = scf.mlp_loss_grad(W1f, W2f, Xf, Tf)
    assert L == pytest.approx(Lr, rel=1e-5)
    assert rel(g1.cpu().numpy(), g1r) < 1e-5
    assert rel(g2.cpu().numpy(), g2r) < 1e-5
    Yb = pkg.mlp_forward(f(W1), f(W2), f(X), bf16=True).cpu().numpy()
    assert 1e-5 < rel(Yb, Y) < 2e-2          # bf16 operands: visibly rounded, still close


def test_mlp_training_matches_oracle_adam(pkg):
    """Five full-batch Adam steps on the GPU track the FP64 oracle's."""
    rng = np.random.default_rng(1)
    din, dh, P = 32, 16, 50
    W1 = rng.standard_normal((dh, din)) / np.sqrt(din)
    W2 = rng.standard_normal((din, dh)) / np.sqrt(dh)
    X = rng.standard_normal((P, din))
    T = X @ rng.standard_normal((din, din)).T * 0.3
    f = lambda a: torch.from_numpy(a.astype(np.float32)).cuda()  # noqa: E731
    W1g, W2g = f(W1), f(W2)
    hist = pkg.mlp_train(W1g, W2g, f(X), f(T), steps=5, lr=1e-2)
    w1, w2 = (a.astype(np.float32).astype(np.float64) for a in (W1, W2))
    Xf, Tf = (a.astype(np.float32).astype(np.float64) for a in (X, T))
    m1 = v1 = np.zeros_like(w1)
    m2 = v2 = np.zeros_like(w2)
    ref = []
    for t in range(1, 6):
        L, g1, g2 = scf.mlp_loss_grad(w1, w2, Xf, Tf)
        ref.append(L)
        w1, m1, v1 = scf.adam_step(w1, g1, m1, v1, t, 1e-2)
        w2, m2, v2 = scf.adam_step(w2, g2, m2, v2, t, 1e-2)
    assert np.allclose(hist, ref, rtol=1e-4)
    assert rel(W1g.cpu().numpy(), w1) < 1e-4
    assert rel(W2g.cpu().numpy(), w2) < 1e-4


@pytest.mark.parametrize("a_mlp", [0.3, 1.0])
def test_learned_preconditioner_reduces_iterations(pkg, small, a_mlp):
    """Train the MLP on residual -> (q* - q - a r) pairs from linear-mixing
    runs (step a) of training fields, then precondition held-out fields with
    q <- q + a r + |r| MLP(r/|r|): fewer SCF iterations than linear mixing at
    alpha = 0.3 to the same residual (judged by the plain method). a = 1 is the
    form used at scale: the correction beyond a unit step, A (I - A)^-1 r for
    A = chi0 K, lives on the few stiff modes of A."""
    tb, chi0, K, _ = small
    H = torch.from_numpy(tb.H).cuda()
    train = workloads.site_fields(tb, 96, seed=10)
    test = workloads.site_fields(tb, 4, seed=11)
    tol = 1e-6
    q_star, _, _, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, train, mixer="anderson", tol=1e-10,
                                           max_iter=300, mode="fp64")
    _, _, its, (tr, tq) = pkg.sp2_scf_response(H, tb.nocc, 4, K, train, mixer="linear", alpha=a_mlp,
                                               tol=tol, max_iter=60, record=True, mode="fp64",
                                               allow_noconv=True)
    R = tr.reshape(-1, tr.shape[-1]).cpu().numpy()
    Tt = (torch.from_numpy(q_star).cuda()[None] - tq - a_mlp * tr).reshape(-1, tq.shape[-1]).cpu().numpy()
    nr = np.linalg.norm(R, axis=1, keepdims=True)
    keep = nr[:, 0] > 0
    Xn, Tn = R[keep] / nr[keep], Tt[keep] / nr[keep]
    ns, dh = Xn.shape[1], 128     # width 2 n_sites: room for a full-rank linear map
    rng = np.random.default_rng(5)
    W1 = torch.from_numpy((rng.standard_normal((dh, ns)) / np.sqrt(ns)).astype(np.float32)).cuda()
    W2 = torch.from_numpy((0.1 * rng.standard_normal((ns, dh)) / np.sqrt(dh)).astype(np.float32)).cuda()
    f = lambda a: torch.from_numpy(a.astype(np.float32)).cuda()  # noqa: E731
    hist = pkg.mlp_train(W1, W2, f(Xn), f(Tn), steps=1500, lr=3e-3)
    assert hist[-1] < 0.2 * hist[0]
    _, res_lin, it_lin, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, test, mixer="linear", alpha=0.3,
                                                 tol=tol, max_iter=300, mode="fp64")
    q_mlp, res_mlp, it_mlp, _ = pkg.sp2_scf_response(H, tb.nocc, 4, K, test, mixer="mlp", W1=W1,
                                                     W2=W2, bf16_infer=True, tol=tol, alpha=a_mlp,
                                                     max_iter=300, mode="fp64")
    assert res_mlp[-1] <= tol
    assert it_mlp < it_lin
    assert rel(q_mlp, scf.scf_exact(chi0, K, test)) < 1e-4
