// CUDA-core product kernels for the plain FP64 and FP32 forms of the SP2 path
// (the "GPU FP32" arithmetic of Sec. VI.C and an FP64 form for 1e-10 parity).
//
// C = A * X with A a stack of row-major (np x np) matrices and X symmetric, so
// X is read row-major as the B operand. Epilogues:
//   EPI_SQUARE  X_{n+1} = sigma>0 ? X_n^2 : 2 X_n - X_n^2 (Eq. DM0) on the tiles
//               meeting the upper triangle; element (i,j), i<j, is written to
//               both (i,j) and (j,i), i>j is skipped, so the result is exactly
//               symmetric. Per-block FP64 partials of Tr[X] and ||X||_F^2.
//   EPI_PLAIN   Z = A X for the response update of Eqs. DM1-DM3.
#include "sp2_internal.h"
#include "decide.cuh"

namespace sp2 {

namespace {

__device__ __forceinline__ bool halted_simt(const DevState* st, int step) {
  const int m = *((volatile const int*)&st->stop_at);
  return m != 0 && step > m;
}

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(256)
k_gemm_simt(const T* __restrict__ A, const T* __restrict__ X, int64_t np, int epi,
            T* __restrict__ out, const T* __restrict__ xprev, Part3* __restrict__ part,
            const Tile* __restrict__ tiles, const DevState* st, int step, SimtDecide dec) {
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  static_assert(BM * BK == 256 * VN && BN * BK == 256 * VN, "one vector per thread per tile");
  if (halted_simt(st, step)) return;

  __shared__ __align__(16) T As[BK][BM];
  __shared__ __align__(16) T Bs[BK][BN];
  const Tile t = tiles[blockIdx.x];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);

  // global -> register staging indices
  const int a_r = tid / (BK / VN), a_k = (tid % (BK / VN)) * VN;
  const int b_k = tid / (BN / VN), b_c = (tid % (BN / VN)) * VN;
  const T* a_ptr = A + (int64_t)(t.row0 + a_r) * np + a_k;
  const T* b_ptr = X + (int64_t)b_k * np + t.col0 + b_c;

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = (T)0;

  V ra = *reinterpret_cast<const V*>(a_ptr);
  V rb = *reinterpret_cast<const V*>(b_ptr);
  for (int64_t k0 = 0; k0 < np; k0 += BK) {
    {
      const T* pa = reinterpret_cast<const T*>(&ra);
#pragma unroll
      for (int v = 0; v < VN; ++v) As[a_k + v][a_r] = pa[v];
      *reinterpret_cast<V*>(&Bs[b_k][b_c]) = rb;
    }
    __syncthreads();
    if (k0 + BK < np) {  // prefetch the next K slice while this one is consumed
      ra = *reinterpret_cast<const V*>(a_ptr + k0 + BK);
      rb = *reinterpret_cast<const V*>(b_ptr + (k0 + BK) * np);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  if (epi == EPI_PLAIN) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t gi = t.row0 + ty + i * (BM / TM), gj = t.col0 + tx + j * (BN / TN);
        out[gi * np + gj] = acc[i][j];
      }
    return;
  }

  const int sg = st->sigma[step];
  double t1 = 0.0, t2 = 0.0, f = 0.0;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gi = t.row0 + ty + i * (BM / TM), gj = t.col0 + tx + j * (BN / TN);
      if (gi > gj) continue;
      const T c = acc[i][j];
      const T x = xprev[gi * np + gj];
      const T v = sg > 0 ? c : (T)2 * x - c;
      out[gi * np + gj] = v;
      const double d = (double)v;
      const double r = (double)x - (double)c;  // (X_n - X_n^2)_ij
      if (gi == gj) {
        t1 += d;
        t2 += d * d;
        f += r * r;
      } else {
        out[gj * np + gi] = v;
        t2 += 2.0 * d * d;
        f += 2.0 * r * r;
      }
    }
  // block reduction of the partials (fixed order)
  __shared__ double r1[8], r2[8], r3[8];
  for (int o = 16; o > 0; o >>= 1) {
    t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    t2 += __shfl_xor_sync(0xffffffffu, t2, o);
    f += __shfl_xor_sync(0xffffffffu, f, o);
  }
  if ((tid & 31) == 0) { r1[tid >> 5] = t1; r2[tid >> 5] = t2; r3[tid >> 5] = f; }
  __syncthreads();
  if (tid == 0) {
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int w = 0; w < 8; ++w) { s1 += r1[w]; s2 += r2[w]; s3 += r3[w]; }
    part[blockIdx.x] = Part3{s1, s2, s3};
  }
  if (dec.done) {
    // the last block to finish reduces every block's partials (fixed order, as the
    // decision kernel does) and takes the step decision
    __shared__ int last;
    if (tid == 0) {
      __threadfence();
      last = atomicAdd(dec.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      decide_block(part, dec.st, dec.p);
      if (tid == 0) *dec.done = 0u;
    }
  }
}

}  // namespace

// FP64 runs at a small fraction of the FP32 rate on GB300, so an FP64 product
// takes as long as its busiest SM: up to np = 1024 it uses 16 x 16 tiles (136
// upper tiles at np = 256, where 64 x 64 tiles would keep 10 SMs busy and leave
// the rest idle), above that 64 x 64.
void simt_tile_shape(int mode, int64_t np, int* bm, int* bn) {
  if (mode == SP2_MODE_FP64) {
    const int t = np <= 1024 ? 16 : 64;
    *bm = t;
    *bn = t;
  } else {
    *bm = 128;
    *bn = 128;
  }
}

cudaError_t launch_gemm_simt(int mode, int epi, const void* A, int64_t a_rows, const void* X,
                             int64_t np, void* out, const void* x_prev, Part3* part,
                             const Tile* tiles, int ntiles, const DevState* st, int step,
                             cudaStream_t s, const SimtDecide* dec) {
  (void)a_rows;
  if (ntiles <= 0) return cudaSuccess;
  int bm, bn;
  simt_tile_shape(mode, np, &bm, &bn);
  SimtDecide sd;
  if (dec && epi == EPI_SQUARE) sd = *dec;
  if (mode == SP2_MODE_FP64 && bm == 16) {
    k_gemm_simt<double, 16, 16, 32, 1, 1><<<ntiles, 256, 0, s>>>(
        static_cast<const double*>(A), static_cast<const double*>(X), np, epi,
        static_cast<double*>(out), static_cast<const double*>(x_prev), part, tiles, st, step, sd);
  } else if (mode == SP2_MODE_FP64) {
    k_gemm_simt<double, 64, 64, 8, 4, 4><<<ntiles, 256, 0, s>>>(
        static_cast<const double*>(A), static_cast<const double*>(X), np, epi,
        static_cast<double*>(out), static_cast<const double*>(x_prev), part, tiles, st, step, sd);
  } else {
    k_gemm_simt<float, 128, 128, 8, 8, 8><<<ntiles, 256, 0, s>>>(
        static_cast<const float*>(A), static_cast<const float*>(X), np, epi,
        static_cast<float*>(out), static_cast<const float*>(x_prev), part, tiles, st, step, sd);
  }
  return cudaGetLastError();
}

}  // namespace sp2
