// Block-sparse SP2 (Sec. II: the products of Eq. DM0 in thresholded sparse
// algebra): 256 x 256 blocks, the tile of a CTA pair. Every iterate keeps dense
// storage; what changes is which blocks exist and which products run.
//
//   X~_1 = T_tau(alpha I + beta H),  X~_{n+1} = T_tau(F_sigma_n(X~_n)),
//
// where T_tau zeroes every off-diagonal block whose Frobenius norm is <= tau
// (diagonal blocks always stay). A square then only forms the upper blocks
// (I, J) for which some K has both (I, K) and (K, J) in X~_n, and each of them
// only over those K blocks; everything else of X_{n+1} is zero.
//
// After each square, one plan kernel (one CTA) turns the tile partials into
// block norms, thresholds, lists the blocks to zero (dropped now, or stale from
// the buffer's previous content), reduces the traces of X~_{n+1} for the branch
// and stop decisions, and writes the next square's tile list with every tile's
// K blocks, in the grouped order the dense tile lists use. A zeroing kernel then
// clears the listed blocks of master and planes (and their mirrors).
#include "sp2_internal.h"

namespace sp2 {

namespace {

constexpr int kBlk = 256;        // block edge = the pair tile
constexpr int kPlanThreads = 1024;
constexpr int kWords = kMaxSparseBlocks / 64;   // 64-bit words of one mask row

__device__ __forceinline__ bool halted_at(const DevState* st, int step) {
  const int m = *((volatile const int*)&st->stop_at);
  return (m != 0 && step > m) || *((volatile const int*)&st->abort_flag);
}

// ||block (I, J)||_F^2 of the master, upper blocks only; one CTA per block
__global__ void k_block_norms(const float* __restrict__ x, int64_t np, int nb, double* nrm2) {
  int I = 0, rem = blockIdx.x;
  while (rem >= nb - I) {   // blockIdx.x enumerates I <= J row by row
    rem -= nb - I;
    ++I;
  }
  const int J = I + rem;
  double acc = 0.0;
  for (int t = threadIdx.x; t < kBlk * kBlk / 4; t += blockDim.x) {
    const int r = t / (kBlk / 4), c4 = t % (kBlk / 4);
    const float4 v = *reinterpret_cast<const float4*>(x + ((int64_t)I * kBlk + r) * np +
                                                      (int64_t)J * kBlk + 4 * c4);
    acc += (double)(v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);   // four in FP32, then FP64
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    nrm2[I * nb + J] = s;
  }
}

struct PlanArgs {
  int nb;
  double tau2;
  int init;                // 1: X~_1 from nrm2 and the init partials; 0: after a square
  const Part3* part;       // init: the init partials; step: two per tile of the square
  int nparts_init;
  const Tile* tiles_in;    // the square's tiles, their count and K-block counts
  const int* ntiles_in;
  const int* kcnt_in;
  uint8_t* mask;           // content mask of the buffer just written (in: stale; out: new)
  double* nrm2;
  uint32_t* zero;          // (I << 16) | J, I <= J
  int* nzero;
  Tile* tiles_out;         // the next square's tiles and K lists
  int* ntiles_out;
  int* kcnt_out;
  uint16_t* klist_out;
  Part3* psum;             // traces of X~ (and f) for the decision
  DevState* st;
  int step;
};

__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kPlanThreads / 32; ++w) s += red[w];
  return s;   // in every thread
}

// candidate x of the grouped tile order (groups of 8 block rows sweep the block
// columns): its block row I and column J
__device__ __forceinline__ void order_ij(int x, int nb, int& I, int& J) {
  const int g0 = (x / (8 * nb)) * 8;
  const int gs = nb - g0 < 8 ? nb - g0 : 8;
  const int rem = x - g0 * nb;
  J = rem / gs;
  I = g0 + rem % gs;
}

__global__ void __launch_bounds__(kPlanThreads, 1) k_sparse_plan(PlanArgs a) {
  if (!a.init && halted_at(a.st, a.step)) return;
  const int nb = a.nb;
  const int tid = threadIdx.x;
  __shared__ unsigned long long bits[kMaxSparseBlocks][kWords];   // mask rows of X~_{n+1}
  __shared__ double red[kPlanThreads / 32];
  __shared__ int scan[kPlanThreads];
  __shared__ int nz;
  const int ntin = a.init ? 0 : *a.ntiles_in;

  // block norms^2 of the new iterate; -1 marks a block the square did not form
  if (!a.init) {
    for (int i = tid; i < nb * nb; i += kPlanThreads) a.nrm2[i] = -1.0;
    __syncthreads();
    for (int t = tid; t < ntin; t += kPlanThreads) {
      const int I = a.tiles_in[t].row0 / kBlk, J = a.tiles_in[t].col0 / kBlk;
      // off-diagonal tiles count every entry twice (the mirror) in their t2
      a.nrm2[I * nb + J] = (a.part[2 * t].t2 + a.part[2 * t + 1].t2) * (I == J ? 1.0 : 0.5);
    }
  }
  for (int i = tid; i < kMaxSparseBlocks * kWords; i += kPlanThreads) (&bits[0][0])[i] = 0ull;
  if (tid == 0) nz = 0;
  __syncthreads();

  // keep / drop / zero, and the traces of X~_{n+1}
  double t1 = 0.0, t2 = 0.0, f = 0.0, drop2 = 0.0;
  if (a.init) {
    for (int i = tid; i < a.nparts_init; i += kPlanThreads) {
      t1 += a.part[i].t1;
      t2 += a.part[i].t2;
    }
  } else {
    for (int i = tid; i < 2 * ntin; i += kPlanThreads) {
      t1 += a.part[i].t1;
      f += a.part[i].f;
    }
  }
  for (int i = tid; i < nb * nb; i += kPlanThreads) {
    const int I = i / nb, J = i % nb;
    if (I > J) continue;
    const double v = a.nrm2[i];
    const bool formed = v >= 0.0;
    const bool keep = formed && (I == J || v > a.tau2);
    const bool stale = !a.init && a.mask[i];
    a.mask[i] = keep;
    a.mask[J * nb + I] = keep;
    if (keep) {
      atomicOr(&bits[I][J >> 6], 1ull << (J & 63));
      atomicOr(&bits[J][I >> 6], 1ull << (I & 63));
      if (!a.init) t2 += v * (I == J ? 1.0 : 2.0);
    } else if (formed && a.init) {
      drop2 += 2.0 * v;
    }
    if ((formed && !keep) || (!formed && stale)) {
      const int z = atomicAdd(&nz, 1);
      a.zero[z] = ((uint32_t)I << 16) | (uint32_t)J;
    }
  }
  t1 = cta_sum(t1, red);
  t2 = cta_sum(t2, red);
  f = cta_sum(f, red);
  drop2 = cta_sum(drop2, red);
  // (cta_sum's barriers also order the mask bits before the listing below)

  // the next square: upper tiles with at least one K block, in grouped order;
  // each thread takes a contiguous range of candidates, counts, then writes
  const int ncand = nb * nb;
  const int per = (ncand + kPlanThreads - 1) / kPlanThreads;
  const int x0 = tid * per, x1 = x0 + per < ncand ? x0 + per : ncand;
  int mine = 0;
  for (int x = x0; x < x1; ++x) {
    int I, J;
    order_ij(x, nb, I, J);
    if (I > J) continue;
    int kc = 0;
    for (int w = 0; w < kWords; ++w) kc += __popcll(bits[I][w] & bits[J][w]);
    mine += kc > 0;
  }
  scan[tid] = mine;
  __syncthreads();
  for (int o = 1; o < kPlanThreads; o <<= 1) {   // inclusive scan
    const int v = tid >= o ? scan[tid - o] : 0;
    __syncthreads();
    scan[tid] += v;
    __syncthreads();
  }
  int pos = scan[tid] - mine;
  double work = 0.0;
  for (int x = x0; x < x1; ++x) {
    int I, J;
    order_ij(x, nb, I, J);
    if (I > J) continue;
    int kc = 0;
    uint16_t* kl = a.klist_out + (int64_t)pos * nb;
    for (int w = 0; w < kWords; ++w) {
      unsigned long long m = bits[I][w] & bits[J][w];
      while (m) {
        const int b = __ffsll((long long)m) - 1;
        m &= m - 1;
        kl[kc++] = (uint16_t)(64 * w + b);
      }
    }
    if (kc > 0) {
      a.tiles_out[pos] = Tile{I * kBlk, J * kBlk};
      a.kcnt_out[pos] = kc;
      ++pos;
    }
  }
  if (!a.init)
    for (int t = tid; t < ntin; t += kPlanThreads) work += a.kcnt_in[t];
  work = cta_sum(work, red);
  if (tid == 0) {
    *a.ntiles_out = scan[kPlanThreads - 1];
    *a.nzero = nz;
    a.psum[0] = Part3{t1, a.init ? t2 - drop2 : t2, f};
    if (!a.init) {
      // the square just done: its share of the upper blocks and its 256-wide K blocks
      if (a.step <= SP2_MAX_ITER) a.st->fill[a.step] = (double)ntin / (0.5 * nb * (nb + 1));
      a.st->work_kblocks += work;
    }
  }
}

// zero the listed blocks (and their mirrors) of master and planes
__global__ void k_zero_blocks(const uint32_t* zero, const int* nzero, MatBuf x, int64_t np,
                              int mode, const DevState* st, int step, int init) {
  if (!init && halted_at(st, step)) return;
  const int n = *nzero;
  const bool x3 = mode == SP2_MODE_BF16X3;
  for (int z = blockIdx.x; z < 2 * n; z += gridDim.x) {
    const uint32_t e = zero[z >> 1];
    int I = (int)(e >> 16), J = (int)(e & 0xffffu);
    if (z & 1) {   // the mirror block
      if (I == J) continue;
      const int t = I;
      I = J;
      J = t;
    }
    for (int t = threadIdx.x; t < kBlk * kBlk / 8; t += blockDim.x) {
      const int r = t / (kBlk / 8), c8 = t % (kBlk / 8);
      const int64_t o = ((int64_t)I * kBlk + r) * np + (int64_t)J * kBlk + 8 * c8;
      float* m = static_cast<float*>(x.master) + o;
      reinterpret_cast<float4*>(m)[0] = make_float4(0.f, 0.f, 0.f, 0.f);
      reinterpret_cast<float4*>(m)[1] = make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<uint4*>(x.hi + o) = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(x.lo + o) = make_uint4(0u, 0u, 0u, 0u);
      if (x3) *reinterpret_cast<uint4*>(x.mid + o) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

}  // namespace

cudaError_t launch_block_norms(const float* master, int64_t np, int nb, double* nrm2,
                               cudaStream_t s) {
  k_block_norms<<<nb * (nb + 1) / 2, 256, 0, s>>>(master, np, nb, nrm2);
  return cudaGetLastError();
}

cudaError_t launch_sparse_plan(const SparseBufs& B, int init, int xo, int tl_in, int tl_out,
                               const Part3* part, int nparts_init, DevState* st, int step,
                               cudaStream_t s) {
  PlanArgs a;
  a.nb = B.nb;
  a.tau2 = B.tau2;
  a.init = init;
  a.part = part;
  a.nparts_init = nparts_init;
  a.tiles_in = B.tiles[tl_in];
  a.ntiles_in = B.ntiles[tl_in];
  a.kcnt_in = B.kcnt[tl_in];
  a.mask = B.mask[xo];
  a.nrm2 = B.nrm2;
  a.zero = B.zero;
  a.nzero = B.nzero;
  a.tiles_out = B.tiles[tl_out];
  a.ntiles_out = B.ntiles[tl_out];
  a.kcnt_out = B.kcnt[tl_out];
  a.klist_out = B.klist[tl_out];
  a.psum = B.psum;
  a.st = st;
  a.step = step;
  k_sparse_plan<<<1, kPlanThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_zero_blocks(const SparseBufs& B, MatBuf x, int64_t np, int mode,
                               const DevState* st, int step, int init, cudaStream_t s) {
  k_zero_blocks<<<2 * 152, 256, 0, s>>>(B.zero, B.nzero, x, np, mode, st, step, init);
  return cudaGetLastError();
}

}  // namespace sp2
