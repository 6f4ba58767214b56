// Element-wise kernels of the finite-temperature recursion (Sec. V.B): a
// symmetrising linear combination of padded matrices and an FP64 trace.
#include "sp2_internal.h"

namespace sp2 {

namespace {

__device__ __forceinline__ void atomic_max_nonneg_f(float* addr, float v) {
  atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
}

// out = z1 (Z1 + Z1^T) + z2 (Z2 + Z2^T) + a A + id I (I restricted to the
// caller's n x n block). Null operands are skipped. One block of 256 threads per
// upper-triangle tile pair (I <= J) of TE x TE tiles, from a linear block index;
// both tiles written with 16-byte accesses, each element from its own inputs.
template <typename T>
constexpr int comb_tile() { return sizeof(T) == 4 ? 64 : 32; }

template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_combine(T* __restrict__ out, int64_t np, int64_t n, const T* __restrict__ Z1, T z1,
              const T* __restrict__ Z2, T z2, const T* __restrict__ A, T a, T id, float* amax) {
  constexpr int TE = comb_tile<T>();
  constexpr int V = TE / 4, R = 256 / V, P = TE / R;
  const int64_t t = blockIdx.x;
  int64_t J = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (J * (J + 1) / 2 > t) --J;
  while ((J + 1) * (J + 2) / 2 <= t) ++J;
  const int64_t I = t - J * (J + 1) / 2;
  const bool diag = I == J;
  __shared__ T sa[TE][TE + 1], sb[TE][TE + 1];
  const int c4 = (threadIdx.x % V) * 4, r0 = threadIdx.x / V;
  const int64_t rI = I * TE, rJ = J * TE;
  T v[P][4], w[P][4];   // out tile (I,J) and, off the diagonal, tile (J,I)
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int j = 0; j < 4; ++j) v[p][j] = w[p][j] = (T)0;
  for (int op = 0; op < 2; ++op) {
    const T* Z = op == 0 ? Z1 : Z2;
    const T zc = op == 0 ? z1 : z2;
    if (!Z) continue;   // uniform across the block
    __syncthreads();    // the previous operand's tiles are no longer read
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int r = r0 + p * R;
      T x[4], y[4];
      ld4(Z + (rI + r) * np + rJ + c4, x);
      ld4(Z + (rJ + r) * np + rI + c4, y);
#pragma unroll
      for (int j = 0; j < 4; ++j) sa[r][c4 + j] = x[j], sb[r][c4 + j] = y[j];
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int r = r0 + p * R;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        v[p][j] += zc * (sa[r][c4 + j] + sb[c4 + j][r]);
        w[p][j] += zc * (sb[r][c4 + j] + sa[c4 + j][r]);
      }
    }
  }
  float m = 0.0f;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int r = r0 + p * R;
    for (int pass = 0; pass < (diag ? 1 : 2); ++pass) {
      const int64_t gi = (pass == 0 ? rI : rJ) + r, gj0 = (pass == 0 ? rJ : rI) + c4;
      T o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = pass == 0 ? v[p][j] : w[p][j];
      if (A) {
        T x[4];
        ld4(A + gi * np + gj0, x);
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] += a * x[j];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (gi == gj0 + j && gi < n) o[j] += id;
        m = fmaxf(m, fabsf((float)o[j]));
      }
      st4(out + gi * np + gj0, o);
    }
  }
  if (amax) {
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomic_max_nonneg_f(amax, m);
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
  // np is a multiple of 256, so both tile edges divide it
  const int64_t nb = np / (mode == SP2_MODE_FP64 ? comb_tile<double>() : comb_tile<float>());
  const dim3 grid((unsigned)(nb * (nb + 1) / 2)), block(256);
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
