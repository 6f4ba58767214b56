"""The benchmark solve at full size (N=16384 tight-binding, forward SP2 and
backward chi of the x-dipole, X_n checkpointed every 4 steps, the bench's
launch configuration) against the oracle's exact closed forms: D = theta(mu I - H)
from LAPACK's dsyevd and chi^A by Daleckii-Krein (Sec. II, Appendix), in FP64 on
the host (the eigendecomposition takes one to two minutes of host time).

Bars: the per-mode constants of tests/tolerances.py times the conditioning
measure (kappa = spectral width / HOMO-LUMO gap, here about 5.3e3). The split
tensor-core paths must also be no less accurate in chi than plain FP32
CUDA-core products on the same solve.
"""
import time

import numpy as np
import pytest
import torch

import tolerances
import workloads
from oracle import exact

pytestmark = [pytest.mark.gpu]

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
    h = sp2.Handle()
    for mode in ("fp16x2", "bf16x3", "fp32"):
        chi, D, info = sp2.sp2_susceptibility(H, tb.nocc, Ad, "backward", diag_only=True,
                                              mode=mode, want_density=True, ckpt_k=4, handle=h)
        out[mode] = (D.cpu().numpy(), chi[0].cpu().numpy(), info["M"])
        del chi, D
    h.close()
    del H
    torch.cuda.empty_cache()
    t0 = time.time()
    e, V = exact.eigh(tb.H.astype(np.float64))
    t_eigh = time.time() - t0
    D_ex = exact.density_zero_T(e, V, tb.nocc)
    chi_ex = exact.response_zero_T(e, V, tb.nocc, np.diag(A.astype(np.float64)))
    kap = tolerances.kappa(e, tb.nocc)
    err = {}
    for mode, (D, chi, M) in out.items():
        err[mode] = (rel(D, D_ex), rel(chi, chi_ex))
        bD, bC = tolerances.tol_d(mode, kap), tolerances.tol_chi(mode, kap, N)
        print(f"N=16384 {mode} vs exact: M={M} gap={e[tb.nocc] - e[tb.nocc - 1]:.2e} "
              f"kappa={kap:.3g} rel err D {err[mode][0]:.2e} (bar {bD:.2e}) chi "
              f"{err[mode][1]:.2e} (bar {bC:.2e}); host eigh {t_eigh:.0f} s")
        assert err[mode][0] < bD, mode
        assert err[mode][1] < bC, mode
    print(f"N=16384 chi fp16x2 vs bf16x3 {rel(out['fp16x2'][1], out['bf16x3'][1]):.2e}, "
          f"fp16x2 vs fp32 {rel(out['fp16x2'][1], out['fp32'][1]):.2e}")
    # the split tensor-core paths are no less accurate than plain FP32 CUDA-core products
    assert err["fp16x2"][1] <= 1.5 * err["fp32"][1]
    assert err["bf16x3"][1] <= 1.5 * err["fp32"][1]
