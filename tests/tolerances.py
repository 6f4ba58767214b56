"""Accuracy bars of the arithmetic modes on gapped problems, as stated numbers
times a conditioning measure the tests compute from the oracle's eigenvalues.

kappa = (e_max - e_min) / (e_LUMO - e_HOMO) is the SP2 condition number: the
recursion needs about 2 log2(kappa) steps, and a perturbation of relative size
u in X_1 moves a near-gap eigenvalue by about u * kappa gaps. The measured
errors of the split tensor-core modes and of plain FP32 follow

    rel err D    <= C_D[mode]   * u[mode] * kappa
    rel err chi  <= C_CHI[mode] * u[mode] * kappa * N      (also a1 = Tr[chi H1])

with u the unit roundoff the mode carries through its products: 2^-24 for the
FP32 accumulation of FP16X2 and BF16X3 and for plain FP32, 2^-16 for the
two bfloat16 planes of BF16X2. The chi bound grows with N because chi sums
N near-gap pair terms (the Loewner form), each carrying the u * kappa error.

The constants are fixed from the tight-binding workloads at N = 4096 and
N = 16384 (same construction, kappa 5.7e3 and 5.3e3), with a margin of about
4: measured chi / (u kappa N) = 2.1e-3 and 2.2e-3 for FP16X2, 2.9e-3 for
BF16X2, 0.34 and 0.38 for plain FP32 (whose run stops at its higher rounding
floor a few steps earlier); D / (u kappa) = 0.023 (FP16X2), 0.22 (BF16X2),
0.19 and 0.88 (FP32). When a bound exceeds 1 the mode cannot resolve the
problem at that size (BF16X2 at N = 4096: 3.6) and the test says so.
"""
import numpy as np

U = {"fp16x2": 2.0 ** -24, "bf16x3": 2.0 ** -24, "fp32": 2.0 ** -24, "bf16x2": 2.0 ** -16}
C_D = {"fp16x2": 0.1, "bf16x3": 0.1, "bf16x2": 1.0, "fp32": 3.0}
C_CHI = {"fp16x2": 1e-2, "bf16x3": 1e-2, "bf16x2": 1e-2, "fp32": 1.5}


def kappa(e: np.ndarray, nocc: int) -> float:
    """Spectral width over the HOMO-LUMO gap (ascending eigenvalues e)."""
    return float((e[-1] - e[0]) / (e[nocc] - e[nocc - 1]))


def tol_d(mode: str, kap: float) -> float:
    return C_D[mode] * U[mode] * kap


def tol_chi(mode: str, kap: float, n: int) -> float:
    return C_CHI[mode] * U[mode] * kap * n
