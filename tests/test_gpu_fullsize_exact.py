"""The benchmark solve at full size (N=16384 tight-binding, FP16X2, forward SP2
and backward chi of the x-dipole, X_n checkpointed every 4 steps) against the
oracle's exact closed forms: D = theta(mu I - H) from LAPACK's dsyevd and
chi^A by Daleckii-Krein (Sec. II, Appendix), in FP64 on the host.

The eigendecomposition of a 16384 x 16384 matrix takes minutes of host time,
so this test runs only when SP2_FULLSIZE_EXACT=1 is set; the N=4096 accuracy
test covers the same comparison by default. FP16X2 and BF16X3 are compared
with plain FP32 CUDA-core products on the same solve: the density to 5e-5, and
chi no less accurate than FP32's (chi carries the 1/gap sensitivity of this
workload, gap 6.0e-3 against a spectral width of about 32).
"""
import os
import time

import numpy as np
import pytest
import torch

import workloads
from oracle import exact

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("SP2_FULLSIZE_EXACT") != "1",
                                 reason="set SP2_FULLSIZE_EXACT=1 (minutes of host LAPACK)")]

N = 16384


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_fullsize_against_exact():
    import __graft_entry__ as g
    g.build()
    import paper_2409_17033_gb300 as sp2
    tb = workloads.tight_binding(N, seed=0, dtype=np.float32)
    A = workloads.tb_dipole_observables(tb)[0].astype(np.float32)
    H = torch.from_numpy(tb.H).cuda()
    Ad = torch.from_numpy(A[None]).cuda()
    out = {}
    for mode in ("fp16x2", "bf16x3", "fp32"):
        chi, D, info = sp2.sp2_susceptibility(H, tb.nocc, Ad, "backward", diag_only=True,
                                              mode=mode, want_density=True, ckpt_k=4)
        out[mode] = (D.cpu().numpy(), chi[0].cpu().numpy(), info["M"])
        del chi, D
    t0 = time.time()
    e, V = exact.eigh(tb.H.astype(np.float64))
    t_eigh = time.time() - t0
    D_ex = exact.density_zero_T(e, V, tb.nocc)
    chi_ex = exact.response_zero_T(e, V, tb.nocc, np.diag(A.astype(np.float64)))
    err = {}
    for mode, (D, chi, M) in out.items():
        err[mode] = (rel(D, D_ex), rel(chi, chi_ex))
        print(f"N=16384 {mode} vs exact: M={M} gap={e[tb.nocc] - e[tb.nocc - 1]:.2e} "
              f"rel err D {err[mode][0]:.2e} chi {err[mode][1]:.2e} (host eigh {t_eigh:.0f} s)")
    print(f"N=16384 chi fp16x2 vs bf16x3 {rel(out['fp16x2'][1], out['bf16x3'][1]):.2e}, "
          f"fp16x2 vs fp32 {rel(out['fp16x2'][1], out['fp32'][1]):.2e}")
    # measured: fp16x2 D 7.8e-6 chi 1.15e-2; bf16x3 9.7e-6, 1.2e-2; fp32 2.8e-4, 2.0
    assert err["fp16x2"][0] < 3e-5 and err["bf16x3"][0] < 3e-5
    assert err["fp16x2"][1] < 4e-2 and err["bf16x3"][1] < 4e-2
    # the split tensor-core paths are no less accurate than plain FP32 CUDA-core products
    assert err["fp16x2"][1] <= 1.5 * err["fp32"][1]
