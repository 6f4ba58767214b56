"""Split-precision products of Sec. VI.B (oracle; test infrastructure only).

Eq. doubleHalf: X = X^(h) + X^(l) with X^(h) = half[X] and
X^(l) = half[X - single[X^(h)]]. "half" is FP16 in the paper; the BF16 form is
the same construction with bfloat16 as the narrow type.

Eq. MixPrecMult / Eq. mults: X Y ~ X^(h) Y^(h) + X^(h) Y^(l) + X^(l) Y^(h),
the X^(l) Y^(l) term dropped. Here the three products are formed in FP64 from
the exactly represented narrow operands, so the only difference from a
tensor-core evaluation with FP32 accumulation is the accumulation rounding.
"""
from __future__ import annotations

import numpy as np


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16 (round to nearest, ties to even), returned
    as float32 holding the bfloat16 value. Written from the format's
    definition: bfloat16 keeps the top 16 bits of the IEEE binary32 pattern.
    NaN inputs are not expected here."""
    x32 = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = x32.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = (b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    out = (r << np.uint64(16)).astype(np.uint32)
    return out.view(np.float32).reshape(x32.shape)


def round_fp16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to IEEE binary16 (numpy's RNE cast), as float32."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def pow2_scale(bound: float) -> float:
    """Power-of-two matrix scale for FP16 planes: 2^(14 - e) where
    bound = m 2^e with m in [0.5, 1), so every scaled entry is at most 2^14
    (below the FP16 maximum 65504); 1 for a zero or non-finite bound."""
    import math
    if not (bound > 0.0) or not math.isfinite(bound):
        return 1.0
    _, e = math.frexp(float(np.float32(bound)))
    k = min(120, max(-120, 14 - e))
    return math.ldexp(1.0, k)


def split_hi_lo(x: np.ndarray, kind: str = "bf16", lo_scale: float = 1.0, scale: float = 1.0):
    """Eq. doubleHalf on scale * x. Returns (hi, lo) as float32 arrays holding
    narrow values. ``scale`` and ``lo_scale`` are powers of two; lo_scale
    multiplies the residual before it is rounded (FP16 range handling) and the
    returned lo is the scaled one."""
    rnd = round_bf16 if kind == "bf16" else round_fp16
    x32 = np.asarray(x, dtype=np.float32) * np.float32(scale)
    hi = rnd(x32)
    lo = rnd((x32 - hi) * np.float32(lo_scale))
    return hi, lo


def mixed_product(X: np.ndarray, Y: np.ndarray, kind: str = "bf16",
                  lo_scale: float = 1.0, sx: float = 1.0, sy: float = 1.0) -> np.ndarray:
    """Eq. MixPrecMult without the lo*lo term, in FP64 on the split operands
    of sx X and sy Y, with the scales divided out."""
    xh, xl = split_hi_lo(X, kind, lo_scale, sx)
    yh, yl = split_hi_lo(Y, kind, lo_scale, sy)
    xh, xl, yh, yl = (a.astype(np.float64) for a in (xh, xl, yh, yl))
    return (xh @ yh + (xh @ yl + xl @ yh) / lo_scale) / (sx * sy)


def split_hi_mid_lo(x: np.ndarray):
    """Three bfloat16 planes of an FP32 value (the multi-split extension the
    paper's Sec. VI.C points to for tunable accuracy): hi = bf16(x),
    mid = bf16(x - hi), lo = bf16(x - hi - mid). Each residual is exact in
    FP32 and each plane carries the next 8 significand bits, so
    hi + mid + lo = x exactly for normal FP32 x (bfloat16 shares FP32's
    exponent range; only residuals below the smallest normal lose bits)."""
    x32 = np.asarray(x, dtype=np.float32)
    hi = round_bf16(x32)
    r1 = x32 - hi
    mid = round_bf16(r1)
    lo = round_bf16(r1 - mid)
    return hi, mid, lo


def mixed_product3(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Product of the three-plane splits keeping every term down to 2^-16
    relative (hi.hi; hi.mid, mid.hi; hi.lo, mid.mid, lo.hi) and dropping the
    2^-24 and 2^-32 ones (mid.lo, lo.mid, lo.lo), in FP64."""
    xh, xm, xl = (a.astype(np.float64) for a in split_hi_mid_lo(X))
    yh, ym, yl = (a.astype(np.float64) for a in split_hi_mid_lo(Y))
    return xh @ yh + (xh @ ym + xm @ yh) + (xh @ yl + xm @ ym + xl @ yh)
