"""Products on CTA pairs (sp2_set_option SP2_OPTION_PAIR_TILES): one tcgen05
instruction stream of M = 256 over two SMs of a thread-block cluster, 256 x 256
output tiles, each SM holding half of both operands' rows and its half of the
accumulator. The arithmetic per output entry (split segments, K order, 256-wide
TMEM chunks, FP32 drains) is the one-SM kernel's, so both tile shapes must give
the same numbers. Checked: one emulated split step against the oracle, whole
recursions (square, response, adjoint, fused response) against the one-SM
kernel and the closed forms, ragged sizes, stacked batches, more tiles than
resident pairs, and the timed-out wait path."""
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


def f32(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


@pytest.fixture(scope="module")
def sp2():
    import __graft_entry__ as g
    g.build()
    import paper_2409_17033_gb300 as p
    return p


def handle(sp2, pair, fused=0):
    h = sp2.Handle()
    h.set_option("pair_tiles", pair)
    h.set_option("fused_response", fused)
    return h


@pytest.mark.parametrize("mode", ["bf16x2", "fp16x2", "bf16x3"])
def test_pair_single_response_step_matches_emulated_split(sp2, mode):
    """One response step Y1 X1 + X1 Y1 (both branches) on 256 x 256 pair tiles
    against the oracle's emulation of the split product on the same planes."""
    p = workloads.random_spectrum(300, nocc=150, k=1, seed=4)
    h = handle(sp2, 1)
    n = 300
    for s in (1, -1):
        chi, _, info = sp2.sp2_susceptibility(f32(p.H), p.nocc, f32(p.A[None]), "forward",
                                              mode=mode, sigma=[s], handle=h)
        a, b = info["alpha"], info["beta"]
        X1 = (a * np.eye(n) + b * p.H.astype(np.float32).astype(np.float64)).astype(np.float32)
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
@pytest.mark.parametrize("n", [300, 700])
def test_pair_recursions_equal_one_sm_kernel(sp2, mode, n):
    """Density (square epilogue), three stacked responses (plain product +
    transpose-add) and the adjoint susceptibility: the same bits as on one SM,
    and the closed forms within the split accuracy."""
    p = workloads.random_spectrum(n, nocc=n // 2, k=3, seed=5)
    H, H1, A = f32(p.H), f32(p.H1), f32(p.A[None])
    out = {}
    for pair in (0, 1):
        h = handle(sp2, pair)
        D, info = sp2.sp2_density(H, p.nocc, mode=mode, handle=h)
        D1, _, info1 = sp2.sp2_response(H, p.nocc, H1, mode=mode, handle=h)
        chi, _, _ = sp2.sp2_susceptibility(H, p.nocc, A, "backward", mode=mode, handle=h)
        torch.cuda.synchronize()
        out[pair] = (D.cpu().numpy(), D1.cpu().numpy(), chi.cpu().numpy(), info["M"],
                     info["sigma"], info1["M"])
    a, b = out[0], out[1]
    assert a[3:] == b[3:]
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    tolD, tolC = (1e-4, 1e-2) if mode == "bf16x2" else (3e-5, 2e-3)
    assert rel(b[0], exact.density_zero_T(p.e, p.Q, p.nocc)) < tolD
    for k in range(3):
        assert rel(b[1][k], exact.response_zero_T(p.e, p.Q, p.nocc, p.H1[k])) < tolC
    assert rel(b[2][0], exact.response_zero_T(p.e, p.Q, p.nocc, p.A)) < tolC


def test_pair_fused_response_equals_one_sm(sp2):
    p = workloads.random_spectrum(700, nocc=350, k=3, seed=6)
    H, H1 = f32(p.H), f32(p.H1)
    res = []
    for pair in (0, 1):
        h = handle(sp2, pair, fused=1)
        D1, _, _ = sp2.sp2_response(H, p.nocc, H1, mode="fp16x2", handle=h)
        res.append(D1.cpu().numpy())
    assert np.array_equal(res[0], res[1])
    for k in range(3):
        assert rel(res[1][k], exact.response_zero_T(p.e, p.Q, p.nocc, p.H1[k])) < 2e-3


def test_pair_more_tiles_than_resident_pairs(sp2):
    """N = 4096: 136 upper pair tiles for at most 76 resident pairs, so every
    pair walks several tiles and its ring and TMEM phases run on across them."""
    p = workloads.tight_binding(4096, seed=0, dtype=np.float32)
    H = f32(p.H)
    res = []
    for pair in (0, 1):
        h = handle(sp2, pair)
        D, info = sp2.sp2_density(H, p.nocc, mode="fp16x2", handle=h)
        res.append((D.cpu().numpy(), info["M"]))
    assert res[0][1] == res[1][1]
    assert np.array_equal(res[0][0], res[1][0])


def test_pair_timed_out_wait_is_reported_and_the_handle_recovers(sp2):
    from paper_2409_17033_gb300 import _lib
    p = workloads.random_spectrum(300, nocc=150, k=1, seed=3)
    H = f32(p.H)
    G = f32(p.A)
    h = handle(sp2, 1)
    D0, info0 = sp2.sp2_density(H, p.nocc, mode="fp16x2", handle=h, keep_history=True)
    g0 = sp2.sp2_adjoint(G, handle=h)
    torch.cuda.synchronize()
    h.set_option("wait_limit_ns", 20_000_000)
    h.set_option("withhold_load", 1)
    for fn in (lambda: sp2.sp2_adjoint(G, handle=h),
               lambda: sp2.sp2_density(H, p.nocc, mode="fp16x2", handle=h)):
        with pytest.raises(sp2.SP2Error) as ex:
            fn()
        assert ex.value.code == _lib.ETIMEOUT, str(ex.value)
    h.set_option("withhold_load", 0)
    h.set_option("wait_limit_ns", 2_000_000_000)
    D1, info1 = sp2.sp2_density(H, p.nocc, mode="fp16x2", handle=h, keep_history=True)
    g1 = sp2.sp2_adjoint(G, handle=h)
    torch.cuda.synchronize()
    assert info1["M"] == info0["M"]
    assert torch.equal(D1, D0)
    assert torch.equal(g1, g0)
