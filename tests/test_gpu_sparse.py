"""Block-sparse SP2 (sp2_opts.block_sparse / block_tau; Sec. II's thresholded
sparse algebra) against the oracle's thresholded recursion and the dense path.

* block_tau = 0 drops only exactly-zero blocks, and the sparse square walks the
  same TMEM chunks as the dense one: the result is the dense result bit for bit,
  on a dense H and on decoupled subsystems (whose coupling blocks stay zero and
  are skipped).
* block_tau > 0 on a gapped periodic rod: the same branches, M, formed-block
  share and D (to the split accuracy) as oracle.sparse at the same threshold.
  The threshold is picked where no block norm of the oracle's run lies within
  0.1 % of it, so both sides take every keep/drop decision the same way.
* the timed-out wait path and the argument checks."""
import numpy as np
import pytest
import torch

import workloads
from oracle import sparse

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


@pytest.mark.parametrize("mode", ["bf16x2", "fp16x2", "bf16x3"])
def test_tau_zero_is_the_dense_result(sp2, mode):
    p = workloads.random_spectrum(1000, nocc=500, k=1, seed=8)
    H = f32(p.H)
    Dd, infd = sp2.sp2_density(H, p.nocc, mode=mode)
    Ds, infs = sp2.sp2_density(H, p.nocc, mode=mode, block_tau=0.0)
    assert infs["M"] == infd["M"] and infs["sigma"] == infd["sigma"]
    assert torch.equal(Ds, Dd)
    assert infs["block_fill"] == 1.0


def test_decoupled_subsystems_skip_their_coupling_blocks(sp2):
    rng = np.random.default_rng(9)
    H = np.zeros((1024, 1024))
    H[:512, :512] = workloads.sym_gaussian(rng, 512, 1.0)
    H[512:, 512:] = workloads.sym_gaussian(rng, 512, 1.0) + 0.2 * np.eye(512)
    Ht = f32(H)
    Dd, infd = sp2.sp2_density(Ht, 500, mode="fp16x2")
    Ds, infs = sp2.sp2_density(Ht, 500, mode="fp16x2", block_tau=0.0)
    assert infs["M"] == infd["M"]
    assert torch.equal(Ds, Dd)
    assert not Ds[:512, 512:].any()
    # two 2 x 2 groups of 256-blocks out of 4 x 4: 6 of the 10 upper blocks
    assert infs["block_fill"] == pytest.approx(0.6)
    assert infs["executed_flops"] < 0.5 * infd["executed_flops"]


def _margin_tau(res_norms, cands, margin=1e-3):
    """The first candidate threshold with no off-diagonal block norm of the
    oracle's run (before thresholding) within `margin` of it, relatively."""
    offs = np.concatenate([n[~np.eye(n.shape[0], dtype=bool)] for n in res_norms])
    for tau in cands:
        if np.all(np.abs(offs - tau) > margin * tau):
            return tau
    return None


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3"])
def test_thresholded_rod_matches_the_oracle(sp2, mode):
    tb = workloads.tight_binding_rod(2000, seed=1, dtype=np.float32)
    H64 = tb.H.astype(np.float64)
    cands = [3e-4, 2e-4, 1.5e-4, 1e-4, 7e-5, 5e-5]
    tau, ref = None, None
    for c in cands:
        r = sparse.sp2_density_thresholded(H64, tb.nocc, c, block=256)
        if _margin_tau(r.norms, [c]) is not None:
            tau, ref = c, r
            break
    assert tau is not None, "no threshold with a decision margin"
    assert ref.converged
    D, info = sp2.sp2_density(f32(tb.H), tb.nocc, mode=mode, block_tau=tau)
    assert info["M"] == ref.M and info["sigma"] == ref.sigma
    assert info["block_fill"] == pytest.approx(sparse.block_fill(ref.masks), abs=1e-12)
    assert info["block_fill"] < 0.9
    assert rel(D.cpu().numpy(), ref.D) < 1e-5
    # the zero blocks of the result are the oracle's
    nz = sparse.block_norms(D.cpu().numpy().astype(np.float64), 256) > 0
    assert np.array_equal(nz, sparse.block_norms(ref.D, 256) > 0)


def test_sparse_timed_out_wait_is_reported_and_the_handle_recovers(sp2):
    from paper_2409_17033_gb300 import _lib
    tb = workloads.tight_binding_rod(1024, seed=2, dtype=np.float32)
    H = f32(tb.H)
    h = sp2.Handle()
    D0, i0 = sp2.sp2_density(H, tb.nocc, mode="fp16x2", block_tau=1e-4, handle=h)
    h.set_option("wait_limit_ns", 20_000_000)
    h.set_option("withhold_load", 1)
    with pytest.raises(sp2.SP2Error) as ex:
        sp2.sp2_density(H, tb.nocc, mode="fp16x2", block_tau=1e-4, handle=h)
    assert ex.value.code == _lib.ETIMEOUT, str(ex.value)
    h.set_option("withhold_load", 0)
    h.set_option("wait_limit_ns", 2_000_000_000)
    D1, i1 = sp2.sp2_density(H, tb.nocc, mode="fp16x2", block_tau=1e-4, handle=h)
    assert i1["M"] == i0["M"] and torch.equal(D1, D0)


def test_sparse_arguments_are_checked(sp2):
    p = workloads.random_spectrum(300, nocc=150, k=1, seed=3)
    H = f32(p.H)
    with pytest.raises(sp2.SP2Error):
        sp2.sp2_density(H, p.nocc, mode="fp32", block_tau=0.0)
    with pytest.raises(sp2.SP2Error):
        sp2.sp2_density(H, p.nocc, mode="fp16x2", block_tau=-1.0)
    with pytest.raises(sp2.SP2Error):
        sp2.sp2_density(H, p.nocc, mode="fp16x2", block_tau=0.0, keep_history=True)
    with pytest.raises(sp2.SP2Error):
        sp2.sp2_response(H, p.nocc, f32(p.H1), mode="fp16x2", block_tau=0.0)
    h = sp2.Handle()
    h.set_option("pair_tiles", 0)
    with pytest.raises(sp2.SP2Error):
        sp2.sp2_density(H, p.nocc, mode="fp16x2", block_tau=0.0, handle=h)
