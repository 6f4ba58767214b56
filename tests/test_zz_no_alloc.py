"""response_contract_noalloc (the allocation-free contraction) against
response_contract, called through the C ABI.

Some callers cannot allocate device memory, so they cannot create a handle;
this entry point serves them with a fixed device array for its partial sums.
Two calls in a row must both agree with the handle-based entry point: the
second one shows that what the first left in the shared array does not leak
into the next result. This file is collected last so that a failure here
comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2409_17033_gb300 import _lib
    assert torch.cuda.is_available()
    return _lib.load()


def _noalloc(lib, P, Q, diag):
    from paper_2409_17033_gb300 import _lib
    L, K, n = P.shape[0], Q.shape[0], P.shape[-1]
    out = torch.full((L, K), float("nan"), dtype=torch.float64, device=P.device)
    dt = _lib.F64 if P.dtype == torch.float64 else _lib.F32
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.response_contract_noalloc(C.c_void_p(P.data_ptr()), L, C.c_void_p(Q.data_ptr()), K,
                                       n, dt, 1 if diag else 0, C.c_void_p(out.data_ptr()),
                                       C.c_void_p(stream))
    assert rc == _lib.OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("diag", [False, True])
def test_noalloc_matches_handle_entry_point_twice(lib, dtype, diag):
    import paper_2409_17033_gb300 as sp2
    rng = np.random.default_rng(7)
    for call, (L, K, n) in enumerate([(2, 5, 300), (3, 4, 257)]):
        P = torch.from_numpy(rng.standard_normal((L, n, n))).to(dtype).cuda()
        Q = torch.from_numpy(rng.standard_normal((K, n) if diag else (K, n, n))).to(dtype).cuda()
        got = _noalloc(lib, P, Q, diag)
        ref = sp2.response_contract(P, Q, diag_only=diag).cpu().numpy()
        assert np.isfinite(got).all(), f"call {call}"
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-10), f"call {call}"


@pytest.mark.parametrize("case", ["clamped_partials", "most_pairs"])
def test_noalloc_at_its_limits(lib, case):
    """The two ends of the fixed partial-sum array: a dense FP32 case whose usual
    partial count (256 per pair at N=1024) times its 32 x 32 pairs exceeds the
    array, so every pair gets fewer partials; and the largest pair count the
    entry point accepts (L * K = 65535) with diagonal perturbations. Both twice
    in a row against the handle-based entry point."""
    import paper_2409_17033_gb300 as sp2
    rng = np.random.default_rng(11)
    if case == "clamped_partials":
        L, K, n, diag, dt = 32, 32, 1024, False, torch.float32
    else:
        L, K, n, diag, dt = 5, 13107, 64, True, torch.float64
    P = torch.from_numpy(rng.standard_normal((L, n, n))).to(dt).cuda()
    Q = torch.from_numpy(rng.standard_normal((K, n) if diag else (K, n, n))).to(dt).cuda()
    ref = sp2.response_contract(P, Q, diag_only=diag).cpu().numpy()
    for call in range(2):
        got = _noalloc(lib, P, Q, diag)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-10), f"call {call}"


def test_noalloc_rejects_bad_arguments(lib):
    from paper_2409_17033_gb300 import _lib
    P = torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    host = np.zeros((1, 4, 4))
    rc = lib.response_contract_noalloc(C.c_void_p(host.ctypes.data), 1, C.c_void_p(P.data_ptr()),
                                       1, 4, _lib.F64, 0, C.c_void_p(out.data_ptr()), None)
    assert rc == _lib.EINVAL
    rc = lib.response_contract_noalloc(C.c_void_p(P.data_ptr()), 300, C.c_void_p(P.data_ptr()),
                                       300, 4, _lib.F64, 0, C.c_void_p(out.data_ptr()), None)
    assert rc == _lib.EINVAL
