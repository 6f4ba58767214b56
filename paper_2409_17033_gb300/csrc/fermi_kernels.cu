// Element-wise kernels of the finite-temperature recursion (Sec. V.B): a
// symmetrising linear combination of padded matrices and an FP64 trace.
#include "sp2_internal.h"

namespace sp2 {

namespace {

__device__ __forceinline__ void atomic_max_nonneg_f(float* addr, float v) {
  atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
}

// out = z1 (Z1 + Z1^T) + z2 (Z2 + Z2^T) + a A + id I (I restricted to the
// caller's n x n block). Null operands are skipped. One block per 32 x 32
// tile pair (I <= J); both tiles written, each element from its own inputs.
template <typename T>
__global__ void k_combine(T* __restrict__ out, int64_t np, int64_t n, const T* __restrict__ Z1,
                          T z1, const T* __restrict__ Z2, T z2, const T* __restrict__ A, T a,
                          T id, float* amax) {
  const int I = blockIdx.y, J = blockIdx.x;
  if (I > J) return;
  __shared__ T s1a[32][33], s1b[32][33], s2a[32][33], s2b[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = 0; k < 32; k += 8) {
    const int r = ty + k;
    const int64_t ij = (int64_t)(I * 32 + r) * np + J * 32 + tx;
    const int64_t ji = (int64_t)(J * 32 + r) * np + I * 32 + tx;
    if (Z1) {
      s1a[r][tx] = Z1[ij];
      s1b[r][tx] = Z1[ji];
    }
    if (Z2) {
      s2a[r][tx] = Z2[ij];
      s2b[r][tx] = Z2[ji];
    }
  }
  __syncthreads();
  float m = 0.0f;
  for (int pass = 0; pass < (I == J ? 1 : 2); ++pass) {
    const int R0 = pass == 0 ? I : J, C0 = pass == 0 ? J : I;
    for (int k = 0; k < 32; k += 8) {
      const int r = ty + k, c = tx;
      const int64_t gi = (int64_t)R0 * 32 + r, gj = (int64_t)C0 * 32 + c;
      const int64_t idx = gi * np + gj;
      T v = (T)0;
      if (Z1) v += z1 * (pass == 0 ? s1a[r][c] + s1b[c][r] : s1b[r][c] + s1a[c][r]);
      if (Z2) v += z2 * (pass == 0 ? s2a[r][c] + s2b[c][r] : s2b[r][c] + s2a[c][r]);
      if (A) v += a * A[idx];
      if (gi == gj && gi < n) v += id;
      out[idx] = v;
      m = fmaxf(m, fabsf((float)v));
    }
  }
  if (amax) {
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (tx == 0 && m > 0.0f) atomic_max_nonneg_f(amax, m);
  }
}

// out[0] = sum_{i < n} M[i, i] in FP64 (one block, fixed order)
template <typename T>
__global__ void k_trace(const T* __restrict__ M, int64_t np, int64_t n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)M[i * np + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[0] = t;
  }
}

}  // namespace

cudaError_t launch_combine(int mode, void* out, int64_t np, int64_t n, const void* Z1, double z1,
                           const void* Z2, double z2, const void* A, double a, double id,
                           float* amax, cudaStream_t s) {
  dim3 grid((unsigned)(np / 32), (unsigned)(np / 32)), block(32, 8);
  if (mode == SP2_MODE_FP64)
    k_combine<double><<<grid, block, 0, s>>>(
        static_cast<double*>(out), np, n, static_cast<const double*>(Z1), z1,
        static_cast<const double*>(Z2), z2, static_cast<const double*>(A), a, id, amax);
  else
    k_combine<float><<<grid, block, 0, s>>>(
        static_cast<float*>(out), np, n, static_cast<const float*>(Z1), (float)z1,
        static_cast<const float*>(Z2), (float)z2, static_cast<const float*>(A), (float)a,
        (float)id, amax);
  return cudaGetLastError();
}

cudaError_t launch_trace(int mode, const void* M, int64_t np, int64_t n, double* out,
                         cudaStream_t s) {
  if (mode == SP2_MODE_FP64)
    k_trace<double><<<1, 1024, 0, s>>>(static_cast<const double*>(M), np, n, out);
  else
    k_trace<float><<<1, 1024, 0, s>>>(static_cast<const float*>(M), np, n, out);
  return cudaGetLastError();
}

}  // namespace sp2
