// Element-wise and reduction kernels of the SP2 path: spectral bounds, the
// initial scaling X_1 = alpha I + beta H, the device-side branch/stop decision,
// the symmetrised response update, output copies and the response contraction.
// All reductions accumulate in FP64 in a fixed order (deterministic).
#include <math.h>

#include "sp2_internal.h"
#include "decide.cuh"

namespace sp2 {

namespace {

constexpr int kRedThreads = 256;

template <typename T>
__device__ __forceinline__ double ld_as_double(const void* p, int64_t idx) {
  return (double)(static_cast<const T*>(p)[idx]);
}

__device__ __forceinline__ double ld_any(const void* p, int64_t idx, int dtype) {
  return dtype == SP2_F64 ? ld_as_double<double>(p, idx) : ld_as_double<float>(p, idx);
}

// block-wide sum of a double (blockDim.x multiple of 32, <= 1024)
// NaN-propagating min / max
__device__ __forceinline__ double nmin(double a, double b) { return (isnan(a) || isnan(b)) ? NAN : fmin(a, b); }
__device__ __forceinline__ double nmax(double a, double b) { return (isnan(a) || isnan(b)) ? NAN : fmax(a, b); }

__device__ double2 block_minmax(double lo, double hi) {
  __shared__ double rlo[32], rhi[32];
  for (int o = 16; o > 0; o >>= 1) {
    lo = nmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = nmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { rlo[w] = lo; rhi[w] = hi; }
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  lo = (threadIdx.x < nw) ? rlo[threadIdx.x] : INFINITY;
  hi = (threadIdx.x < nw) ? rhi[threadIdx.x] : -INFINITY;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) {
      lo = nmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = nmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
  return make_double2(lo, hi);
}

// ------------------------------------------------------------ Gershgorin
// Row i contributes H_ii -/+ sum_{j != i} |H_ij| (Sec. II: spectral bound
// estimates eps_min, eps_max, read as Gershgorin discs).
__global__ void k_bounds(const void* H, int64_t n, int dtype, double2* part) {
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    double r = 0.0, d = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      double v = ld_any(H, i * n + j, dtype);
      if (j == i) d = v; else r += fabs(v);
    }
    r = block_sum(r);
    d = block_sum(d);
    if (threadIdx.x == 0) { lo = nmin(lo, d - r); hi = nmax(hi, d + r); }
  }
  double2 mm = block_minmax(lo, hi);
  if (threadIdx.x == 0) part[blockIdx.x] = mm;
}

// Sec. II: X_1 = alpha I + beta H maps [eps_min, eps_max] onto [1, 0] in reverse
// order, alpha = eps_max / (eps_max - eps_min), beta = -1 / (eps_max - eps_min); a
// point spectrum is widened to [eps - 1/2, eps + 1/2].
__device__ void set_coefficients(DevState* st, double lo, double hi) {
  if (!isfinite(lo) || !isfinite(hi)) {
    st->bounds[0] = lo;
    st->bounds[1] = hi;
    st->nonfinite = 1;
    st->stop_at = -1;   // every step kernel is a no-op
    return;
  }
  if (!(hi > lo)) {
    lo -= 0.5;
    hi += 0.5;
  }
  st->bounds[0] = lo;
  st->bounds[1] = hi;
  const double w = hi - lo;
  st->alpha = hi / w;
  st->beta = -1.0 / w;
}

__global__ void k_bounds_final(const double2* part, int nparts, DevState* st) {
  double lo = INFINITY, hi = -INFINITY;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    lo = nmin(lo, part[i].x);
    hi = nmax(hi, part[i].y);
  }
  double2 mm = block_minmax(lo, hi);
  if (threadIdx.x == 0) set_coefficients(st, mm.x, mm.y);
}

__global__ void k_set_bounds(DevState* st, double lo, double hi) { set_coefficients(st, lo, hi); }

struct SigmaArg {
  int8_t s[SP2_MAX_ITER];
};

__global__ void k_set_sigma(DevState* st, SigmaArg a, int m) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) st->sigma[i + 1] = a.s[i];
}

// an adjoint recursion runs every step it is given and keeps no floor candidate
__global__ void k_adjoint_state(DevState* st) {
  st->stop_at = 0;
  st->keep_step = 0;
  st->abort_flag = 0;
  st->nonfinite = 0;
}

// ------------------------------------------------------------ init
// Writes one element in the mode's layout; split modes also write the planes
// (fp16 planes with scale 1) unless planes == false.
__device__ __forceinline__ void store_elem(MatBuf d, int mode, int64_t idx, double v, bool planes) {
  if (mode == SP2_MODE_FP64) {
    static_cast<double*>(d.master)[idx] = v;
    return;
  }
  const float f = (float)v;
  static_cast<float*>(d.master)[idx] = f;
  if (!planes) return;
  uint16_t h, l;
  if (mode == SP2_MODE_BF16X2) {
    split_bf16(f, h, l);
    d.hi[idx] = h;
    d.lo[idx] = l;
  } else if (mode == SP2_MODE_FP16X2) {
    split_fp16(f, 1.0f, h, l);
    d.hi[idx] = h;
    d.lo[idx] = l;
  } else if (mode == SP2_MODE_BF16X3) {
    uint16_t m;
    split_bf16x3(f, h, m, l);
    d.hi[idx] = h;
    d.mid[idx] = m;
    d.lo[idx] = l;
  }
}

__device__ __forceinline__ double stored_value(int mode, double v) {
  return mode == SP2_MODE_FP64 ? v : (double)(float)v;
}

// atomic max of non-negative floats through their (monotone) bit patterns
__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
  atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
}

__global__ void k_init(const void* src, int64_t n, int64_t np, int64_t batch, int dtype,
                       int diag_only, int symmetrize, double alpha, double beta, int mode,
                       MatBuf dst, Part3* part, float* ymax, int coef, const DevState* st) {
  if (coef == INIT_STATE) {
    alpha = st->alpha;
    beta = st->beta;
  } else if (coef == INIT_STATE_BETA) {
    alpha = 0.0;
    beta = st->beta;
  }
  double t1 = 0.0, t2 = 0.0;
  const bool planes = !(mode == SP2_MODE_FP16X2 && ymax != nullptr);
  const int64_t rows = batch * np;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const int64_t b = r / np, i = r % np;
    float rmax = 0.0f;
    for (int64_t j = threadIdx.x; j < np; j += blockDim.x) {
      double v = 0.0;
      if (i < n && j < n) {
        if (diag_only) {
          if (i == j) v = beta * ld_any(src, b * n + i, dtype);
        } else if (symmetrize) {
          v = beta * (0.5 * (ld_any(src, (b * n + i) * n + j, dtype) +
                             ld_any(src, (b * n + j) * n + i, dtype)));
        } else {
          v = beta * ld_any(src, (b * n + i) * n + j, dtype);
        }
        if (i == j) v += alpha;
      }
      store_elem(dst, mode, r * np + j, v, planes);
      double s = stored_value(mode, v);
      if (i == j) t1 += s;
      t2 += s * s;
      rmax = fmaxf(rmax, fabsf((float)v));
    }
    if (!planes) {
      for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
      if ((threadIdx.x & 31) == 0 && rmax > 0.0f) atomic_max_nonneg(&ymax[b], rmax);
    }
  }
  if (part) {
    t1 = block_sum(t1);
    __syncthreads();
    t2 = block_sum(t2);
    if (threadIdx.x == 0) part[blockIdx.x] = Part3{t1, t2, 0.0};
  }
}

// ------------------------------------------------------------ decide
__global__ void k_decide(const Part3* part, DevState* st, DecideParams p) {
  decide_block(part, st, p);
}

template <typename T>
__global__ void k_keep_best(const T* __restrict__ src, T* __restrict__ dst, int64_t count,
                            const DevState* st, int step) {
  if (*((volatile const int*)&st->keep_step) != step) return;
  const int64_t n4 = count / 4;   // count is a multiple of np^2, np % 256 == 0
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4;
       t += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 4) {
      reinterpret_cast<float4*>(dst)[t] = reinterpret_cast<const float4*>(src)[t];
    } else {
      reinterpret_cast<double2*>(dst)[2 * t] = reinterpret_cast<const double2*>(src)[2 * t];
      reinterpret_cast<double2*>(dst)[2 * t + 1] = reinterpret_cast<const double2*>(src)[2 * t + 1];
    }
  }
}

__device__ __forceinline__ bool halted(const DevState* st, int step) {
  const int m = *((volatile const int*)&st->stop_at);
  return m != 0 && step > m;
}

// ------------------------------------------------------------ symmetrised update
// Y_{n+1} = (1 - sigma) Y_n + sigma (Z + Z^T), Z = Y_n X_n (Eqs. DM1-DM3: X_n Y_n = (Y_n X_n)^T
// for symmetric X_n, Y_n). One block per tile pair (I <= J) of the upper triangle, taken from
// a linear block index (no idle blocks for the lower triangle); Z tiles (I,J) and (J,I) are
// read once with 16-byte loads, Y_{n+1}(I,J) is written and mirrored into (J,I).
template <typename T>
__device__ __forceinline__ void ld4_stream(const T* p, T (&v)[4]);
template <>
__device__ __forceinline__ void ld4_stream<float>(const float* p, float (&v)[4]) {
  const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
  v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
template <>
__device__ __forceinline__ void ld4_stream<double>(const double* p, double (&v)[4]) {
  const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
  const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}

// four consecutive entries of Y_{n+1} (idx a multiple of 4): master and, in the split
// modes, the hi/lo planes as one 8-byte store each
template <typename ZT, int MODE>
__device__ __forceinline__ void store_y4(MatBuf y, int64_t idx, const ZT (&v)[4], float s) {
  if constexpr (sizeof(ZT) == 4) {
    *reinterpret_cast<float4*>(static_cast<float*>(y.master) + idx) =
        make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  } else {
    double2* d = reinterpret_cast<double2*>(static_cast<double*>(y.master) + idx);
    d[0] = make_double2((double)v[0], (double)v[1]);
    d[1] = make_double2((double)v[2], (double)v[3]);
  }
  if (MODE == SP2_MODE_BF16X3) {
    uint16_t h[4], m[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) split_bf16x3((float)v[j], h[j], m[j], l[j]);
    *reinterpret_cast<uint2*>(y.hi + idx) =
        make_uint2(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16));
    *reinterpret_cast<uint2*>(y.mid + idx) =
        make_uint2(m[0] | ((uint32_t)m[1] << 16), m[2] | ((uint32_t)m[3] << 16));
    *reinterpret_cast<uint2*>(y.lo + idx) =
        make_uint2(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16));
  }
  if (MODE == SP2_MODE_BF16X2 || MODE == SP2_MODE_FP16X2) {
    uint16_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (MODE == SP2_MODE_BF16X2) split_bf16((float)v[j], h[j], l[j]);
      else split_fp16((float)v[j], s, h[j], l[j]);
    }
    *reinterpret_cast<uint2*>(y.hi + idx) =
        make_uint2(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16));
    *reinterpret_cast<uint2*>(y.lo + idx) =
        make_uint2(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16));
  }
}

constexpr int kSymThreads = 256;
template <typename ZT>
constexpr int sym_tile() { return sizeof(ZT) == 4 ? 64 : 32; }   // 33 / 17 KB of shared memory

template <typename ZT, int MODE>
__global__ void __launch_bounds__(kSymThreads)
    k_symm_update(const ZT* __restrict__ Z, MatBuf yin, MatBuf yout, int64_t np,
                  const DevState* st, int step, ScaleBuf sc, int slot_in, int slot_out) {
  if (halted(st, step)) return;
  constexpr int TE = sym_tile<ZT>();
  constexpr int V = TE / 4;                // 4-entry vectors per tile row
  constexpr int R = kSymThreads / V;       // rows covered by one pass of the block
  constexpr int P = TE / R;
  // column J of the upper triangle holds tiles I = 0..J: t = J (J + 1) / 2 + I
  const int64_t t = blockIdx.x;
  int64_t J = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (J * (J + 1) / 2 > t) --J;
  while ((J + 1) * (J + 2) / 2 <= t) ++J;
  const int64_t I = t - J * (J + 1) / 2;
  const int64_t base = (int64_t)blockIdx.y * np * np;
  const int64_t b = blockIdx.y;
  __shared__ ZT za[TE][TE + 1];   // Z tile (I,J), overwritten in place by Y_{n+1}(I,J)
  __shared__ ZT zb[TE][TE + 1];   // Z tile (J,I)
  const int c4 = (threadIdx.x % V) * 4, r0 = threadIdx.x / V;
  const int sg = st->sigma[step];
  float s = 1.0f;
  if (MODE == SP2_MODE_FP16X2) {
    // |Y_{n+1}| <= |Z_ij| + |Z_ji| (+ 2 |Y_n| for sigma<0), elementwise
    float bound = 2.0f * sc.zmax[b];
    if (sg < 0) bound += 2.0f * sc.ymax[slot_in * sc.B + b];
    s = pow2_scale(bound);
    if (t == 0 && threadIdx.x == 0) sc.yscale[slot_out * sc.B + b] = s;
  }
  const int64_t rI = I * TE, rJ = J * TE;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int r = r0 + p * R;
    ZT a[4], c[4];
    ld4_stream(Z + base + (rI + r) * np + rJ + c4, a);
    ld4_stream(Z + base + (rJ + r) * np + rI + c4, c);
#pragma unroll
    for (int j = 0; j < 4; ++j) za[r][c4 + j] = a[j], zb[r][c4 + j] = c[j];
  }
  __syncthreads();
  float amax = 0.0f;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int r = r0 + p * R;
    const int64_t idx = base + (rI + r) * np + rJ + c4;
    ZT y[4], yo[4];
    if (sg < 0) ld4_stream(static_cast<const ZT*>(yin.master) + idx, yo);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const ZT sum = za[r][c4 + j] + zb[c4 + j][r];
      y[j] = sg > 0 ? sum : (ZT)2 * yo[j] - sum;
      amax = fmaxf(amax, fabsf((float)y[j]));
      za[r][c4 + j] = y[j];   // only this thread touches za[r][c4..c4+3] in this phase
    }
    store_y4<ZT, MODE>(yout, idx, y, s);
  }
  if (MODE == SP2_MODE_FP16X2) {
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && amax > 0.0f) atomic_max_nonneg(&sc.ymax[slot_out * sc.B + b], amax);
  }
  if (I == J) return;
  __syncthreads();
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int r = r0 + p * R;
    ZT y[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) y[j] = za[c4 + j][r];
    store_y4<ZT, MODE>(yout, base + (rJ + r) * np + rI + c4, y, s);
  }
}

// ------------------------------------------------------------ output copy
__global__ void k_copy_out(MatBuf src, int64_t n, int64_t np, int64_t batch, int mode,
                           double scale, void* dst, int dtype, const DevState* beta_state) {
  if (beta_state) scale *= beta_state->beta;
  const int64_t total = batch * n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / (n * n), rem = t % (n * n), i = rem / n, j = rem % n;
    const int64_t s = (b * np + i) * np + j;
    double v = mode == SP2_MODE_FP64 ? static_cast<const double*>(src.master)[s]
                                     : (double)static_cast<const float*>(src.master)[s];
    v *= scale;
    if (dtype == SP2_F64) static_cast<double*>(dst)[t] = v;
    else static_cast<float*>(dst)[t] = (float)v;
  }
}

// planes of four consecutive entries (8-byte stores per plane)
__device__ __forceinline__ uint2 pack4(const uint16_t (&v)[4]) {
  return make_uint2(v[0] | ((uint32_t)v[1] << 16), v[2] | ((uint32_t)v[3] << 16));
}

// ---- vectorised forms of the O(N^2) passes for an FP32 input with N % 4 == 0:
// four consecutive entries per thread step, FP64 only where the values need it
// (GB300 runs FP64 at a small fraction of its FP32 rate)

// planes of four stored entries in the mode's split (fp16 planes with scale 1)
__device__ __forceinline__ void store_planes4(MatBuf d, int mode, int64_t t, const float (&f)[4]) {
  uint16_t h[4], l[4], md[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (mode == SP2_MODE_BF16X3) split_bf16x3(f[k], h[k], md[k], l[k]);
    else if (mode == SP2_MODE_BF16X2) split_bf16(f[k], h[k], l[k]);
    else split_fp16(f[k], 1.0f, h[k], l[k]);
  }
  reinterpret_cast<uint2*>(d.hi)[t] = pack4(h);
  reinterpret_cast<uint2*>(d.lo)[t] = pack4(l);
  if (mode == SP2_MODE_BF16X3) reinterpret_cast<uint2*>(d.mid)[t] = pack4(md);
}

// FP32 forms of FP64 arithmetic for the O(N^2) passes (GB300's FP64 pipe, and
// its conversions, run at a small fraction of the FP32 rate and bounded these
// passes well below the HBM bandwidth):
// - TwoSum (Knuth) and the fmaf product residual give an addition's and a
//   product's rounding error exactly; the _rn intrinsics keep the compiler from
//   contracting the steps into fused operations, which would lose them;
// - an FP64 coefficient c is carried as hi + lo, hi = fl32(c), lo = fl32(c - hi),
//   and x c is formed as fl32(p + (e + x lo)) with p = fl32(x hi) and e its
//   residual: within one rounding of the exact x c (the FP64 form rounds twice).
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 split_coef(double c) {
  const float hi = (float)c;
  return F2{hi, (float)(c - (double)hi)};
}
__device__ __forceinline__ float mul_coef(float x, F2 c) {
  const float p = __fmul_rn(x, c.hi);
  const float e = fmaf(x, c.hi, -p);
  return __fadd_rn(p, fmaf(x, c.lo, e));
}
// s + c += x with the rounding error of the addition carried in c
__device__ __forceinline__ void two_sum_add(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float bp = __fsub_rn(t, s);
  c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
  s = t;
}
// s + c += x^2 exactly up to the rounding of c
__device__ __forceinline__ void two_sum_add_sq(float& s, float& c, float x) {
  const float p = __fmul_rn(x, x);
  two_sum_add(s, c, p);
  c = __fadd_rn(c, fmaf(x, x, -p));
}

// X_1 = alpha I + beta H (coefficients from st) with its planes. Off the diagonal
// an entry is beta h formed in FP32 from beta = hi + lo (mul_coef); a diagonal
// entry, one per row, is beta h + alpha in FP64, rounded once. The trace partials
// take Tr exactly (the diagonal entries) and ||X_1||_F^2 as an exact FP32 sum of
// squares per row segment, added in FP64.
__global__ void k_init_x4(const float* __restrict__ src, int64_t n, int64_t np, int mode,
                          MatBuf dst, Part3* part, const DevState* st) {
  const double alpha = st->alpha, beta = st->beta;
  const F2 bc = split_coef(beta);
  double t1 = 0.0, t2 = 0.0;
  const int64_t q = np / 4;
  for (int64_t r = blockIdx.x; r < np; r += gridDim.x) {
    float ss = 0.0f, sc = 0.0f;   // this thread's sum of squares of the row segment
    for (int64_t c = threadIdx.x; c < q; c += blockDim.x) {
      const int64_t j = 4 * c;
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      if (r < n && j < n) {   // n % 4 == 0: the whole group is inside
        const float4 h = *reinterpret_cast<const float4*>(src + r * n + j);
        x[0] = h.x;
        x[1] = h.y;
        x[2] = h.z;
        x[3] = h.w;
      }
      float f[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) f[k] = mul_coef(x[k], bc);
      if (r < n && r >= j && r < j + 4) {
        f[r - j] = (float)(beta * (double)x[r - j] + alpha);
        t1 += (double)f[r - j];
      }
      reinterpret_cast<float4*>(dst.master)[r * q + c] = make_float4(f[0], f[1], f[2], f[3]);
      store_planes4(dst, mode, r * q + c, f);
#pragma unroll
      for (int k = 0; k < 4; ++k) two_sum_add_sq(ss, sc, f[k]);
    }
    t2 += (double)ss + (double)sc;
  }
  t1 = block_sum(t1);
  __syncthreads();
  t2 = block_sum(t2);
  if (threadIdx.x == 0) part[blockIdx.x] = Part3{t1, t2, 0.0};
}

// Gershgorin discs of an FP32 H, one warp per row: each lane sums |h| of its
// part of the row with TwoSum in FP32, four 16-byte loads in flight, and moves
// the sum and its error to FP64 after each group of 16 entries; lanes add in FP64.
__global__ void k_bounds_x4(const float* __restrict__ H, int64_t n, double2* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t q = n / 4;
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < n; i += (int64_t)gridDim.x * nw) {
    const float4* row = reinterpret_cast<const float4*>(H + i * n);
    const int64_t cd = i >> 2;   // the group holding the diagonal entry
    double r = 0.0, d = 0.0;
    for (int64_t c0 = lane; c0 < q; c0 += 4 * 32) {
      float4 h[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t c = c0 + 32 * u;
        h[u] = c < q ? row[c] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      float s = 0.0f, e = 0.0f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float x[4] = {h[u].x, h[u].y, h[u].z, h[u].w};
        if (c0 + 32 * u == cd) {   // take the diagonal entry out of the row sum
          d = x[i & 3];
          x[i & 3] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) two_sum_add(s, e, fabsf(x[k]));
      }
      r += (double)s + (double)e;
    }
    for (int o = 16; o > 0; o >>= 1) {
      r += __shfl_xor_sync(0xffffffffu, r, o);
      d += __shfl_xor_sync(0xffffffffu, d, o);
    }
    if (lane == 0) {
      lo = nmin(lo, d - r);
      hi = nmax(hi, d + r);
    }
  }
  double2 mm = block_minmax(lo, hi);
  if (threadIdx.x == 0) part[blockIdx.x] = mm;
}

// caller-layout copy of an FP32 master, four entries per step, one row per block
// step (no per-entry division); a scale (times beta from the state, when given)
// is applied as an FP32 product with the split coefficient (mul_coef)
__global__ void k_copy_out_x4(const float* __restrict__ src, int64_t n, int64_t np, int64_t batch,
                              double scale, float* __restrict__ dst, const DevState* beta_state) {
  if (beta_state) scale *= beta_state->beta;
  const bool scaled = scale != 1.0;
  const F2 sc = split_coef(scale);
  const int64_t q = n / 4, rows = batch * n;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int64_t b = row / n, i = row - b * n;
    const float4* s4 = reinterpret_cast<const float4*>(src + (b * np + i) * np);
    float4* d4 = reinterpret_cast<float4*>(dst) + row * q;
    for (int64_t c = threadIdx.x; c < q; c += blockDim.x) {
      float4 v = s4[c];
      if (scaled) {
        v.x = mul_coef(v.x, sc);
        v.y = mul_coef(v.y, sc);
        v.z = mul_coef(v.z, sc);
        v.w = mul_coef(v.w, sc);
      }
      d4[c] = v;
    }
  }
}

// hi/lo (and BF16X3 mid) planes from the FP32 master; total is a multiple of 4
__global__ void k_split(MatBuf m, int64_t total, int mode) {
  const int64_t total4 = total / 4;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total4;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float4 f = reinterpret_cast<const float4*>(m.master)[t];
    const float x[4] = {f.x, f.y, f.z, f.w};
    uint16_t h[4], l[4], md[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (mode == SP2_MODE_BF16X3) split_bf16x3(x[j], h[j], md[j], l[j]);
      else if (mode == SP2_MODE_BF16X2) split_bf16(x[j], h[j], l[j]);
      else split_fp16(x[j], 1.0f, h[j], l[j]);
    }
    reinterpret_cast<uint2*>(m.hi)[t] = pack4(h);
    reinterpret_cast<uint2*>(m.lo)[t] = pack4(l);
    if (mode == SP2_MODE_BF16X3) reinterpret_cast<uint2*>(m.mid)[t] = pack4(md);
  }
}

__global__ void k_scales_from_max(ScaleBuf sc, int slot) {
  for (int64_t b = threadIdx.x; b < sc.B; b += blockDim.x)
    sc.yscale[slot * sc.B + b] = pow2_scale(sc.ymax[slot * sc.B + b]);
}

// FP16X2 planes of a batch of sc.B matrices of `per` entries each (per % 4 == 0),
// each with its slot's power-of-two scale
__global__ void k_split_scaled(MatBuf m, int64_t per, ScaleBuf sc, int slot) {
  const int64_t total4 = per * sc.B / 4;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total4;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float4 f = reinterpret_cast<const float4*>(m.master)[t];
    const float x[4] = {f.x, f.y, f.z, f.w};
    const float scale = sc.yscale[slot * sc.B + (4 * t) / per];
    uint16_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) split_fp16(x[j], scale, h[j], l[j]);
    reinterpret_cast<uint2*>(m.hi)[t] = pack4(h);
    reinterpret_cast<uint2*>(m.lo)[t] = pack4(l);
  }
}

// ------------------------------------------------------------ FP16X2 response scales
// The symmetric response update maps Y to Y X + X Y or Y (I - X) + (I - X) Y,
// with the spectrum of X in [0, 1]; either way ||Y_{n+1}||_2 <= 2 ||Y_n||_2,
// and |entry| <= 2-norm <= Frobenius norm. The plane scale of Y_{n+2} is
// therefore fixed by ||Y_{n+1}||_F before the step that writes it.
__global__ void k_sym_scale(const Part3* part, int ppt, const Tile* tiles, int ntiles, int64_t np,
                            const DevState* st, int step, float* scale_out) {
  if (st) {
    const int m = st->stop_at;
    if ((m != 0 && step > m) || st->abort_flag) return;
  }
  const int64_t b = blockIdx.x;
  double acc = 0.0;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
    if (tiles[t].row0 / np == b)
      for (int j = 0; j < ppt; ++j) acc += part[t * ppt + j].t2;
  acc = block_sum(acc);
  if (threadIdx.x == 0) scale_out[b] = pow2_scale((float)(2.0 * sqrt(fmax(acc, 0.0))));
}

__global__ void k_fro_part(const float* __restrict__ m, int64_t per, double* part) {
  const float* x = m + blockIdx.y * per;
  double acc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < per;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[t];
    acc += v * v;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

__global__ void k_fro_final(const double* part, int nparts, float* scale_out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[blockIdx.x * nparts + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) scale_out[blockIdx.x] = pow2_scale((float)(2.0 * sqrt(acc)));
}

// ------------------------------------------------------------ contraction
// out[l,k] = sum_ij P_l[i,j] Q_k[i,j] (Eqs. expectation, direct, dual), FP64
// accumulation, per-block partials then a fixed-order second pass.
template <typename T>
__global__ void k_contract_dense(const T* __restrict__ P, const T* __restrict__ Q, int64_t K,
                                 int64_t nn, double* part, int nparts, int64_t y0) {
  const int64_t pair = y0 + blockIdx.y;
  const int64_t l = pair / K, k = pair % K;
  const T* p = P + l * nn;
  const T* q = Q + k * nn;
  double acc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn;
       t += (int64_t)gridDim.x * blockDim.x)
    acc += (double)p[t] * (double)q[t];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[pair * nparts + blockIdx.x] = acc;
}

// FP32 inputs: exact products and sums at FP32 cost. TwoProduct splits a*b into
// p + e exactly (e = fma(a, b, -p)); TwoSum adds p to the running pair (s, c)
// without loss; the small terms e and c are summed in FP32, their rounding far
// below 2^-40 of the magnitudes involved. Each thread converts once to FP64 at
// the end. A block covers one slice of the N^2 entries for up to kCtrKT
// perturbations Q_k, so the shared left factor P_l is read once per kCtrKT.
constexpr int kCtrKT = 8;

// (the _rn intrinsics are never contracted into FMAs, which would break both
// error-free transformations)
__device__ __forceinline__ void acc_exact(float& s, float& c, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  c = __fadd_rn(c, __fadd_rn(err, e));
  s = t;
}

template <int VEC>
__global__ void __launch_bounds__(256) k_contract_dense_f32(const float* __restrict__ P,
                                                           const float* __restrict__ Q, int64_t K,
                                                           int64_t nn, double* part, int nparts,
                                                           int64_t y0) {
  const int64_t ktiles = (K + kCtrKT - 1) / kCtrKT;
  const int64_t y = y0 + blockIdx.y;
  const int64_t l = y / ktiles, k0 = (y % ktiles) * kCtrKT;
  const int kn = (int)((K - k0) < kCtrKT ? (K - k0) : kCtrKT);
  const float* p = P + l * nn;
  float s[kCtrKT], c[kCtrKT];
#pragma unroll
  for (int kk = 0; kk < kCtrKT; ++kk) s[kk] = c[kk] = 0.0f;
  const int64_t nv = nn / VEC;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nv;
       t += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (VEC == 4) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p) + t);
#pragma unroll
      for (int kk = 0; kk < kCtrKT; ++kk) {
        if (kk < kn) {
          const float4 b = __ldcs(reinterpret_cast<const float4*>(Q + (k0 + kk) * nn) + t);
          acc_exact(s[kk], c[kk], a.x, b.x);
          acc_exact(s[kk], c[kk], a.y, b.y);
          acc_exact(s[kk], c[kk], a.z, b.z);
          acc_exact(s[kk], c[kk], a.w, b.w);
        }
      }
    } else {
      const float a = p[t];
#pragma unroll
      for (int kk = 0; kk < kCtrKT; ++kk)
        if (kk < kn) acc_exact(s[kk], c[kk], a, Q[(k0 + kk) * nn + t]);
    }
  }
#pragma unroll
  for (int kk = 0; kk < kCtrKT; ++kk) {
    if (kk >= kn) break;   // uniform across the block
    const double v = block_sum((double)s[kk] + (double)c[kk]);
    if (threadIdx.x == 0) part[(l * K + k0 + kk) * nparts + blockIdx.x] = v;
  }
}

template <typename T>
__global__ void k_contract_diag(const T* __restrict__ P, const T* __restrict__ Q, int64_t K,
                                int64_t n, double* part, int nparts, int64_t y0) {
  const int64_t pair = y0 + blockIdx.y;
  const int64_t l = pair / K, k = pair % K;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)P[l * n * n + i * n + i] * (double)Q[k * n + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[pair * nparts + blockIdx.x] = acc;
}

__global__ void k_contract_final(const double* part, int nparts, double* out) {
  const int64_t pair = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[pair * nparts + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[pair] = acc;
}

inline int grid_for(int64_t total, int threads, int cap) {
  int64_t g = (total + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

// ------------------------------------------------------------ launchers
int bounds_nparts(int64_t n) { return (int)(n < 1024 ? (n < 1 ? 1 : n) : 1024); }

cudaError_t launch_bounds(const void* H, int64_t n, int dtype, double2* part, int nparts,
                          DevState* st, cudaStream_t s) {
  if (dtype == SP2_F32 && n % 4 == 0 && (reinterpret_cast<uintptr_t>(H) & 15u) == 0)
    k_bounds_x4<<<nparts, kRedThreads, 0, s>>>(static_cast<const float*>(H), n, part);
  else
    k_bounds<<<nparts, kRedThreads, 0, s>>>(H, n, dtype, part);
  k_bounds_final<<<1, 1024, 0, s>>>(part, nparts, st);
  return cudaGetLastError();
}

int init_nparts(int64_t np) { return (int)(np < 1024 ? np : 1024); }

cudaError_t launch_init(const void* src, int64_t n, int64_t np, int64_t batch, int dtype,
                        int diag_only, int symmetrize, double alpha, double beta, int mode,
                        MatBuf dst, Part3* part, int nparts, float* ymax, cudaStream_t s,
                        int coef, const DevState* st) {
  if (coef == INIT_STATE && part && batch == 1 && dtype == SP2_F32 && !diag_only && !symmetrize &&
      !ymax && split_mode(mode) && n % 4 == 0 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
    k_init_x4<<<nparts, kRedThreads, 0, s>>>(static_cast<const float*>(src), n, np, mode, dst, part,
                                             st);
    return cudaGetLastError();
  }
  int grid = part ? nparts : grid_for(batch * np, 1, 4096);
  k_init<<<grid, kRedThreads, 0, s>>>(src, n, np, batch, dtype, diag_only, symmetrize, alpha,
                                      beta, mode, dst, part, ymax, coef, st);
  return cudaGetLastError();
}

cudaError_t launch_set_bounds(DevState* st, double eps_min, double eps_max, cudaStream_t s) {
  k_set_bounds<<<1, 1, 0, s>>>(st, eps_min, eps_max);
  return cudaGetLastError();
}

cudaError_t launch_set_sigma(DevState* st, const int8_t* sigma, int m, cudaStream_t s) {
  if (m < 0 || m > SP2_MAX_ITER) return cudaErrorInvalidValue;
  SigmaArg a;
  for (int i = 0; i < SP2_MAX_ITER; ++i) a.s[i] = i < m ? sigma[i] : 0;
  k_set_sigma<<<1, 256, 0, s>>>(st, a, m);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_state(DevState* st, cudaStream_t s) {
  k_adjoint_state<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_keep_best(const void* src, void* dst, int64_t count, int mode, const DevState* st,
                             int step, cudaStream_t s) {
  const int grid = 2 * 152 * 4;
  if (mode == SP2_MODE_FP64)
    k_keep_best<double><<<grid, 256, 0, s>>>(static_cast<const double*>(src),
                                             static_cast<double*>(dst), count, st, step);
  else
    k_keep_best<float><<<grid, 256, 0, s>>>(static_cast<const float*>(src), static_cast<float*>(dst),
                                            count, st, step);
  return cudaGetLastError();
}

cudaError_t launch_decide(const Part3* part, DevState* st, DecideParams p, cudaStream_t s) {
  k_decide<<<1, kRedThreads, 0, s>>>(part, st, p);
  return cudaGetLastError();
}

cudaError_t launch_symm_update(const void* Z, MatBuf y_in, MatBuf y_out, int64_t np, int64_t batch,
                               int mode, const DevState* st, int step, ScaleBuf sc, int slot_in,
                               int slot_out, cudaStream_t s) {
  // np is a multiple of 256, so both tile edges divide it
  const int64_t nb = np / (mode == SP2_MODE_FP64 ? sym_tile<double>() : sym_tile<float>());
  dim3 grid((unsigned)(nb * (nb + 1) / 2), (unsigned)batch), block(kSymThreads);
  if (mode == SP2_MODE_FP64)
    k_symm_update<double, SP2_MODE_FP64><<<grid, block, 0, s>>>(
        static_cast<const double*>(Z), y_in, y_out, np, st, step, sc, slot_in, slot_out);
  else if (mode == SP2_MODE_FP32)
    k_symm_update<float, SP2_MODE_FP32><<<grid, block, 0, s>>>(
        static_cast<const float*>(Z), y_in, y_out, np, st, step, sc, slot_in, slot_out);
  else if (mode == SP2_MODE_BF16X2)
    k_symm_update<float, SP2_MODE_BF16X2><<<grid, block, 0, s>>>(
        static_cast<const float*>(Z), y_in, y_out, np, st, step, sc, slot_in, slot_out);
  else if (mode == SP2_MODE_BF16X3)
    k_symm_update<float, SP2_MODE_BF16X3><<<grid, block, 0, s>>>(
        static_cast<const float*>(Z), y_in, y_out, np, st, step, sc, slot_in, slot_out);
  else
    k_symm_update<float, SP2_MODE_FP16X2><<<grid, block, 0, s>>>(
        static_cast<const float*>(Z), y_in, y_out, np, st, step, sc, slot_in, slot_out);
  return cudaGetLastError();
}

cudaError_t launch_copy_out(MatBuf src, int64_t n, int64_t np, int64_t batch, int mode,
                            double scale, void* dst, int dtype, cudaStream_t s,
                            const DevState* beta_state) {
  if (mode != SP2_MODE_FP64 && dtype == SP2_F32 && n % 4 == 0 &&
      (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
    k_copy_out_x4<<<grid_for(batch * n, 1, 8192), 256, 0, s>>>(
        static_cast<const float*>(src.master), n, np, batch, scale, static_cast<float*>(dst),
        beta_state);
    return cudaGetLastError();
  }
  k_copy_out<<<grid_for(batch * n * n, 256, 8192), 256, 0, s>>>(src, n, np, batch, mode, scale,
                                                                 dst, dtype, beta_state);
  return cudaGetLastError();
}

cudaError_t launch_split(MatBuf m, int64_t rows, int64_t np, int mode, cudaStream_t s) {
  k_split<<<grid_for(rows * np / 4, 256, 8192), 256, 0, s>>>(m, rows * np, mode);
  return cudaGetLastError();
}

cudaError_t launch_split_scaled(MatBuf m, int64_t np, ScaleBuf sc, int slot, cudaStream_t s) {
  k_scales_from_max<<<1, 256, 0, s>>>(sc, slot);
  k_split_scaled<<<grid_for(sc.B * np * np / 4, 256, 8192), 256, 0, s>>>(m, np * np, sc, slot);
  return cudaGetLastError();
}

cudaError_t launch_sym_scale(const Part3* part, int ppt, const Tile* tiles, int ntiles, int64_t np,
                             int64_t batch, const DevState* st, int step, float* scale_out,
                             cudaStream_t s) {
  k_sym_scale<<<(unsigned)batch, kRedThreads, 0, s>>>(part, ppt, tiles, ntiles, np, st, step,
                                                        scale_out);
  return cudaGetLastError();
}

int fro_nparts() { return 256; }

cudaError_t launch_fro_scale(const float* master, int64_t np, int64_t batch, double* part,
                             int nparts, float* scale_out, cudaStream_t s) {
  dim3 grid((unsigned)nparts, (unsigned)batch);
  k_fro_part<<<grid, kRedThreads, 0, s>>>(master, np * np, part);
  k_fro_final<<<(unsigned)batch, kRedThreads, 0, s>>>(part, nparts, scale_out);
  return cudaGetLastError();
}

// blocks per (l, k) pair: one per 4096 entries, at most 1216 (8 blocks of 256
// threads per SM on 152 SMs, enough loads in flight for HBM with one pair)
int contract_nparts(int64_t n, int q_diag) {
  int64_t work = q_diag ? n : n * n;
  int64_t g = (work + 256 * 16 - 1) / (256 * 16);
  if (g < 1) g = 1;
  if (g > 1216) g = 1216;
  return (int)g;
}

cudaError_t launch_contract(const void* P, int64_t L, const void* Q, int64_t K, int64_t n,
                            int dtype, int q_diag, double* part, int nparts, double* out,
                            cudaStream_t s) {
  // grid rows (one per pair, or per observable and group of kCtrKT perturbations)
  // go out in launches of at most 65535, the limit of gridDim.y
  constexpr int64_t kMaxY = 65535;
  const int64_t nn = n * n;
  const bool f32_dense = dtype != SP2_F64 && !q_diag;
  const int64_t ktiles = (K + kCtrKT - 1) / kCtrKT;
  const int64_t rows = f32_dense ? L * ktiles : L * K;
  // float4 path when every matrix starts on a 16-byte boundary
  const bool v4 = nn % 4 == 0 && ((reinterpret_cast<uintptr_t>(P) |
                                   reinterpret_cast<uintptr_t>(Q)) & 15u) == 0;
  for (int64_t y0 = 0; y0 < rows; y0 += kMaxY) {
    const int64_t ny = (rows - y0) < kMaxY ? (rows - y0) : kMaxY;
    dim3 grid((unsigned)nparts, (unsigned)ny);
    if (dtype == SP2_F64) {
      if (q_diag)
        k_contract_diag<double><<<grid, 256, 0, s>>>(static_cast<const double*>(P),
                                                     static_cast<const double*>(Q), K, n, part,
                                                     nparts, y0);
      else
        k_contract_dense<double><<<grid, 256, 0, s>>>(static_cast<const double*>(P),
                                                      static_cast<const double*>(Q), K, nn, part,
                                                      nparts, y0);
    } else if (q_diag) {
      k_contract_diag<float><<<grid, 256, 0, s>>>(static_cast<const float*>(P),
                                                  static_cast<const float*>(Q), K, n, part, nparts,
                                                  y0);
    } else if (v4) {
      k_contract_dense_f32<4><<<grid, 256, 0, s>>>(static_cast<const float*>(P),
                                                   static_cast<const float*>(Q), K, nn, part,
                                                   nparts, y0);
    } else {
      k_contract_dense_f32<1><<<grid, 256, 0, s>>>(static_cast<const float*>(P),
                                                   static_cast<const float*>(Q), K, nn, part,
                                                   nparts, y0);
    }
  }
  k_contract_final<<<(unsigned)(L * K), 256, 0, s>>>(part, nparts, out);
  return cudaGetLastError();
}

}  // namespace sp2
