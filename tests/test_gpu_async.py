"""Asynchronous calls and sp2_synchronize (C ABI): a call with info == NULL and
device buffers returns once its work is enqueued -- here a backward
susceptibility whose adjoint recursion (Eq. DM2) is still running -- and
sp2_synchronize then reports exactly what the synchronous call reports (branch
sequence, M, traces, idempotency errors, bounds), with bit-identical outputs.
Also: the status known only after the work ran (a timed-out wait in the
adjoint) comes from sp2_synchronize, and a host-buffer call completes before it
returns."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp2():
    import __graft_entry__ as g
    g.build()
    import paper_2409_17033_gb300 as p
    return p


@pytest.fixture(scope="module")
def tb():
    t = workloads.tight_binding(4096, seed=0, dtype=np.float32)
    A = workloads.tb_dipole_observables(t)[0:1].astype(np.float32)
    return t, A


KEYS = ("M", "converged", "alpha", "beta", "eps_min", "eps_max", "trace", "idem_err", "sigma",
        "errors", "idem_fro", "n_gemm_launches", "ckpt_k")


def test_call_returns_before_its_stream_completes(sp2, tb):
    t, A = tb
    H = torch.from_numpy(t.H).cuda()
    Ad = torch.from_numpy(A).cuda()
    h = sp2.Handle()
    kw = dict(direction="backward", diag_only=True, mode="fp16x2", want_density=True, handle=h)
    chi_s, D_s, info_s = sp2.sp2_susceptibility(H, t.nocc, Ad, **kw)   # synchronous
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    chi_a, D_a, none = sp2.sp2_susceptibility(H, t.nocc, Ad, sync=False, **kw)
    pending = not stream.query()         # the adjoint of ~50 products is still running
    info_a = sp2.synchronize(h)
    assert none is None
    assert pending, "the call waited for its stream"
    assert stream.query()
    for k in KEYS:
        assert info_a[k] == info_s[k], k
    assert torch.equal(chi_a, chi_s)
    assert torch.equal(D_a, D_s)


def test_synchronize_without_pending_call(sp2):
    h = sp2.Handle()
    info = sp2.synchronize(h)
    assert info["M"] == 0


def test_adjoint_timeout_reported_by_synchronize(sp2):
    """The forward recursion runs normally; the adjoint's product launches meet a
    withheld operand load (test hook, 20 ms wait limit): the asynchronous call
    returns SP2_OK, sp2_synchronize returns SP2_ETIMEOUT, and the handle works
    afterwards."""
    from paper_2409_17033_gb300 import _lib
    p = workloads.random_spectrum(256, nocc=128, k=1, seed=2)
    H = torch.from_numpy(p.H).float().cuda()
    G = torch.from_numpy(p.A).float().cuda()
    h = sp2.Handle()
    sp2.sp2_density(H, p.nocc, mode="fp16x2", handle=h, keep_history=True)
    g0 = sp2.sp2_adjoint(G, handle=h)
    h.set_option("wait_limit_ns", 20_000_000)
    h.set_option("withhold_load", 1)
    sp2.sp2_adjoint(G, handle=h, sync=False)
    with pytest.raises(sp2.SP2Error) as ex:
        sp2.synchronize(h)
    assert ex.value.code == _lib.ETIMEOUT
    h.set_option("withhold_load", 0)
    h.set_option("wait_limit_ns", 2_000_000_000)
    g1 = sp2.sp2_adjoint(G, handle=h)
    assert torch.equal(g1, g0)


def test_host_buffers_complete_before_return(sp2):
    p = workloads.random_spectrum(300, nocc=150, k=1, seed=4)
    h = sp2.Handle()
    Hh = p.H.astype(np.float32)
    lib = h.lib
    D = np.full((300, 300), np.nan, np.float32)
    opts, _k = sp2.make_opts("fp16x2")
    rc = lib.sp2_density(h.h, C.c_void_p(Hh.ctypes.data), 300, 1, float(p.nocc), C.byref(opts),
                         C.c_void_p(D.ctypes.data), None)
    assert rc == 0
    assert np.isfinite(D).all()          # complete on return although info was NULL
    Dd, _ = sp2.sp2_density(torch.from_numpy(Hh).cuda(), p.nocc, mode="fp16x2", handle=h)
    assert np.array_equal(D, Dd.cpu().numpy())
