// Kernels of the self-consistent response loop (Appendix, Eq. DM_CP_SCF with
// a site-charge G) and of the learned MLP preconditioner: small dense
// products, site-charge gathering, mixing updates, MLP training steps.
#include "sp2_internal.h"

namespace sp2 {

namespace {

// C = alpha op(A) op(B) + beta C, FP32, row-major; op(A) is M x K (A stored
// [M][K], or [K][M] when ta), op(B) is K x N (B stored [K][N], or [N][K] when
// tb). relu != 0 applies max(., 0) to the result. bf16 != 0 rounds every
// operand element to bfloat16 on load (bf16 inference, FP32 accumulation).
constexpr int SG_T = 64, SG_K = 16;

__device__ __forceinline__ float ld_op(const float* P, int64_t ld, bool t, int64_t r, int64_t c,
                                       int64_t R, int64_t Cc, bool bf16) {
  if (r >= R || c >= Cc) return 0.0f;
  float v = t ? P[c * ld + r] : P[r * ld + c];
  if (bf16) v = __bfloat162float(__float2bfloat16_rn(v));
  return v;
}

__global__ void __launch_bounds__(256)
k_sgemm(int64_t M, int64_t N, int64_t K, float alpha, const float* __restrict__ A, int64_t lda,
        int ta, const float* __restrict__ B, int64_t ldb, int tb, float beta,
        float* __restrict__ C, int64_t ldc, int relu, int bf16) {
  __shared__ float As[SG_K][SG_T + 1];
  __shared__ float Bs[SG_K][SG_T + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * SG_T, n0 = (int64_t)blockIdx.x * SG_T;
  float acc[4][4] = {};
  for (int64_t k0 = 0; k0 < K; k0 += SG_K) {
    for (int e = threadIdx.x; e < SG_T * SG_K; e += 256) {
      const int mm = e / SG_K, kk = e % SG_K;
      As[kk][mm] = ld_op(A, lda, ta, m0 + mm, k0 + kk, M, K, bf16);
      const int nn = e / SG_K;
      const int64_t kb = k0 + kk, nb = n0 + nn;
      float bv = 0.0f;
      if (kb < K && nb < N) bv = tb ? B[nb * ldb + kb] : B[kb * ldb + nb];
      if (bf16) bv = __bfloat162float(__float2bfloat16_rn(bv));
      Bs[kk][nn] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SG_K; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m >= M || n >= N) continue;
      float v = alpha * acc[i][j];
      if (beta != 0.0f) v += beta * C[m * ldc + n];
      if (relu) v = fmaxf(v, 0.0f);
      C[m * ldc + n] = v;
    }
}

// u[f][a] = V[f][a] + sum_b K[a][b] q[f][b]   (FP64, one thread per (f, a))
__global__ void k_site_potential(const double* __restrict__ V, const double* __restrict__ K,
                                 const double* __restrict__ q, int64_t F, int64_t ns,
                                 double* __restrict__ u) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * ns) return;
  const int64_t f = t / ns, a = t % ns;
  double s = V[t];
  const double* qf = q + f * ns;
  const double* Ka = K + a * ns;
  for (int64_t b = 0; b < ns; ++b) s += Ka[b] * qf[b];
  u[t] = s;
}

// per-orbital diagonal perturbation from site potentials: out[f][a*norb+o] = u[f][a]
template <typename T>
__global__ void k_expand_sites(const double* __restrict__ u, int64_t F, int64_t ns, int norb,
                               T* __restrict__ out) {
  const int64_t n = ns * norb;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * n) return;
  const int64_t f = t / n, i = t % n;
  out[t] = (T)u[f * ns + i / norb];
}

// q[f][a] = sum_{mu in a} Y_f[mu][mu] over the padded response masters
template <typename T>
__global__ void k_site_charges(const T* __restrict__ Y, int64_t F, int64_t ns, int norb,
                               int64_t np, double* __restrict__ q) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * ns) return;
  const int64_t f = t / ns, a = t % ns;
  const T* Yf = Y + f * np * np;
  double s = 0.0;
  for (int o = 0; o < norb; ++o) {
    const int64_t mu = a * norb + o;
    s += (double)Yf[mu * np + mu];
  }
  q[t] = s;
}

// r = qout - q; out[0] += sum r^2, out[1] += sum qout^2 (FP64 atomics over blocks)
__global__ void k_residual(const double* __restrict__ qout, const double* __restrict__ q,
                           int64_t total, double* __restrict__ r, double* __restrict__ out) {
  double s1 = 0.0, s2 = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double d = qout[t] - q[t];
    r[t] = d;
    s1 += d * d;
    s2 += qout[t] * qout[t];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], s1);
    atomicAdd(&out[1], s2);
  }
}

__global__ void k_axpy_d(double* __restrict__ y, double a, const double* __restrict__ x,
                         int64_t total) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x)
    y[t] += a * x[t];
}

// Anderson Gram matrices: G[f][i][j] = <R_i[f], R_j[f]> over the m stored residuals
__global__ void k_gram(const double* __restrict__ R, int m, int64_t F, int64_t ns, int64_t stride,
                       double* __restrict__ G) {
  const int64_t f = blockIdx.x;
  const int i = blockIdx.y / m, j = blockIdx.y % m;
  const double* a = R + i * stride + f * ns;
  const double* b = R + j * stride + f * ns;
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < ns; t += blockDim.x) s += a[t] * b[t];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t2 += red[w];
    G[(f * m + i) * m + j] = t2;
  }
}

// q[f] = sum_i c[f][i] (Q_i[f] + alpha R_i[f])
__global__ void k_anderson_combine(const double* __restrict__ Qh, const double* __restrict__ Rh,
                                   const double* __restrict__ c, int m, int64_t F, int64_t ns,
                                   int64_t stride, double alpha, double* __restrict__ q) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * ns) return;
  const int64_t f = t / ns;
  double s = 0.0;
  for (int i = 0; i < m; ++i) s += c[f * m + i] * (Qh[i * stride + t] + alpha * Rh[i * stride + t]);
  q[t] = s;
}

// MLP input: x[f] = r[f] / ||r[f]|| (float), nr[f] = ||r[f]||
__global__ void k_normalise_rows(const double* __restrict__ r, int64_t F, int64_t ns,
                                 float* __restrict__ x, double* __restrict__ nr) {
  const int64_t f = blockIdx.x;
  const double* rf = r + f * ns;
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < ns; t += blockDim.x) s += rf[t] * rf[t];
  __shared__ double red[32];
  __shared__ double tot;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t2 += red[w];
    tot = sqrt(t2);
    nr[f] = tot;
  }
  __syncthreads();
  const double inv = tot > 0.0 ? 1.0 / tot : 0.0;
  for (int64_t t = threadIdx.x; t < ns; t += blockDim.x) x[f * ns + t] = (float)(rf[t] * inv);
}

// q[f] += nr[f] * y[f]
__global__ void k_apply_update(double* __restrict__ q, const float* __restrict__ y,
                               const double* __restrict__ nr, int64_t F, int64_t ns) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * ns) return;
  q[t] += nr[t / ns] * (double)y[t];
}

// --- MLP training: E = Y - T, dY = 2 E / P, loss partials
__global__ void k_mse_grad(const float* __restrict__ Y, const float* __restrict__ T, int64_t total,
                           float scale, float* __restrict__ dY, double* __restrict__ loss) {
  double s = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float e = Y[t] - T[t];
    dY[t] = 2.0f * e * scale;
    s += (double)e * e;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * scale);
}

// dH *= (Hpre > 0)
__global__ void k_relu_mask(float* __restrict__ dH, const float* __restrict__ Hr, int64_t total) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x)
    if (!(Hr[t] > 0.0f)) dH[t] = 0.0f;
}

// Adam (Kingma & Ba): m, v moments, bias-corrected step
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t total, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float mt = b1 * m[t] + (1.0f - b1) * g[t];
    const float vt = b2 * v[t] + (1.0f - b2) * g[t] * g[t];
    m[t] = mt;
    v[t] = vt;
    w[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  }
}

inline unsigned grid_of(int64_t total, int threads, int cap = 65535) {
  int64_t g = (total + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

cudaError_t launch_sgemm(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                         int ta, const float* B, int64_t ldb, int tb, float beta, float* C,
                         int64_t ldc, int relu, int bf16, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((unsigned)((N + SG_T - 1) / SG_T), (unsigned)((M + SG_T - 1) / SG_T));
  k_sgemm<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, relu, bf16);
  return cudaGetLastError();
}

cudaError_t launch_site_potential(const double* V, const double* K, const double* q, int64_t F,
                                  int64_t ns, double* u, cudaStream_t s) {
  k_site_potential<<<grid_of(F * ns, 128), 128, 0, s>>>(V, K, q, F, ns, u);
  return cudaGetLastError();
}

cudaError_t launch_expand_sites(const double* u, int64_t F, int64_t ns, int norb, void* out,
                                int dtype, cudaStream_t s) {
  const int64_t total = F * ns * norb;
  if (dtype == SP2_F64)
    k_expand_sites<double><<<grid_of(total, 256), 256, 0, s>>>(u, F, ns, norb,
                                                               static_cast<double*>(out));
  else
    k_expand_sites<float><<<grid_of(total, 256), 256, 0, s>>>(u, F, ns, norb,
                                                              static_cast<float*>(out));
  return cudaGetLastError();
}

cudaError_t launch_site_charges(const void* Y, int mode, int64_t F, int64_t ns, int norb,
                                int64_t np, double* q, cudaStream_t s) {
  if (mode == SP2_MODE_FP64)
    k_site_charges<double><<<grid_of(F * ns, 128), 128, 0, s>>>(static_cast<const double*>(Y), F,
                                                                ns, norb, np, q);
  else
    k_site_charges<float><<<grid_of(F * ns, 128), 128, 0, s>>>(static_cast<const float*>(Y), F,
                                                               ns, norb, np, q);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* qout, const double* q, int64_t total, double* r,
                            double* out2, cudaStream_t s) {
  k_residual<<<grid_of(total, 256, 1024), 256, 0, s>>>(qout, q, total, r, out2);
  return cudaGetLastError();
}

cudaError_t launch_axpy_d(double* y, double a, const double* x, int64_t total, cudaStream_t s) {
  k_axpy_d<<<grid_of(total, 256, 4096), 256, 0, s>>>(y, a, x, total);
  return cudaGetLastError();
}

cudaError_t launch_gram(const double* R, int m, int64_t F, int64_t ns, int64_t stride, double* G,
                        cudaStream_t s) {
  dim3 grid((unsigned)F, (unsigned)(m * m));
  k_gram<<<grid, 256, 0, s>>>(R, m, F, ns, stride, G);
  return cudaGetLastError();
}

cudaError_t launch_anderson_combine(const double* Qh, const double* Rh, const double* c, int m,
                                    int64_t F, int64_t ns, int64_t stride, double alpha, double* q,
                                    cudaStream_t s) {
  k_anderson_combine<<<grid_of(F * ns, 256), 256, 0, s>>>(Qh, Rh, c, m, F, ns, stride, alpha, q);
  return cudaGetLastError();
}

cudaError_t launch_normalise_rows(const double* r, int64_t F, int64_t ns, float* x, double* nr,
                                  cudaStream_t s) {
  k_normalise_rows<<<(unsigned)F, 256, 0, s>>>(r, F, ns, x, nr);
  return cudaGetLastError();
}

cudaError_t launch_apply_update(double* q, const float* y, const double* nr, int64_t F, int64_t ns,
                                cudaStream_t s) {
  k_apply_update<<<grid_of(F * ns, 256), 256, 0, s>>>(q, y, nr, F, ns);
  return cudaGetLastError();
}

cudaError_t launch_mse_grad(const float* Y, const float* T, int64_t total, float scale, float* dY,
                            double* loss, cudaStream_t s) {
  k_mse_grad<<<grid_of(total, 256, 1024), 256, 0, s>>>(Y, T, total, scale, dY, loss);
  return cudaGetLastError();
}

cudaError_t launch_relu_mask(float* dH, const float* Hr, int64_t total, cudaStream_t s) {
  k_relu_mask<<<grid_of(total, 256, 4096), 256, 0, s>>>(dH, Hr, total);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int64_t total, float lr,
                        float b1, float b2, float eps, int t, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  k_adam<<<grid_of(total, 256, 4096), 256, 0, s>>>(w, g, m, v, total, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace sp2
