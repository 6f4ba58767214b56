"""The bounded device waits of the tensor-core product kernel, made to run out
on purpose through the library's test hook (sp2_set_option
SP2_OPTION_WITHHOLD_LOAD): the first operand load of the first CTA is never
issued, so that CTA's wait for it ends at the wait limit (20 ms here). The
kernel then raises its abort flag, drains its own copies and tensor-core work,
frees its tensor memory and returns; the call must report SP2_ETIMEOUT, and the
next call on the same handle must succeed with the same result as before.
Covered: the forward recursion (sp2_density) and the adjoint recursion
(sp2_adjoint, Eq. DM2), whose product launches keep their own device state.
No GPU fault is involved: every wait is bounded and nothing is left running."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2409_17033_gb300 as p
    return p


def _expect_timeout(pkg, fn):
    from paper_2409_17033_gb300 import _lib
    with pytest.raises(pkg.SP2Error) as ex:
        fn()
    assert ex.value.code == _lib.ETIMEOUT, str(ex.value)


@pytest.mark.parametrize("mode", ["fp16x2", "bf16x3"])
def test_timed_out_wait_is_reported_and_the_handle_recovers(pkg, mode):
    p = workloads.random_spectrum(300, nocc=150, k=1, seed=3)
    H = torch.from_numpy(p.H).float().cuda()
    G = torch.from_numpy(p.A).float().cuda()
    h = pkg.Handle()
    D0, info0 = pkg.sp2_density(H, p.nocc, mode=mode, handle=h, keep_history=True)
    g0 = pkg.sp2_adjoint(G, handle=h)
    torch.cuda.synchronize()

    h.set_option("wait_limit_ns", 20_000_000)
    h.set_option("withhold_load", 1)
    # the adjoint over the kept history: its product launches time out
    _expect_timeout(pkg, lambda: pkg.sp2_adjoint(G, handle=h))
    # the forward recursion
    _expect_timeout(pkg, lambda: pkg.sp2_density(H, p.nocc, mode=mode, handle=h))
    h.set_option("withhold_load", 0)
    h.set_option("wait_limit_ns", 2_000_000_000)

    D1, info1 = pkg.sp2_density(H, p.nocc, mode=mode, handle=h, keep_history=True)
    g1 = pkg.sp2_adjoint(G, handle=h)
    torch.cuda.synchronize()
    assert info1["M"] == info0["M"] and info1["sigma"] == info0["sigma"]
    assert torch.equal(D1, D0)
    assert torch.equal(g1, g0)
    assert np.isfinite(g1.cpu().numpy()).all()


def test_option_arguments_are_checked(pkg):
    h = pkg.Handle()
    with pytest.raises(pkg.SP2Error):
        h.set_option("wait_limit_ns", 10)        # below 1 us
    from paper_2409_17033_gb300 import _lib
    assert h.lib.sp2_set_option(h.h, 99, 0) == _lib.EINVAL
