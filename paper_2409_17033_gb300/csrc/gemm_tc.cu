// Split-precision tensor-core product kernel for sm_103a (tcgen05 + TMEM + TMA).
//
// Computes C = A X for the SP2 path with the hi/lo splitting of Eq. doubleHalf
// and the three-product form of Eq. MixPrecMult / Eq. mults (lo*lo dropped):
//     A X ~ A_hi X_hi + A_hi X_lo + A_lo X_hi,
// evaluated over a concatenated K axis of length 3 np,
//     [A_hi | A_hi | A_lo] . [X_hi ; X_lo ; X_hi],
// into FP32 accumulators in tensor memory. X is symmetric, so the row-major
// X planes are directly the K-major B operand.
//   BF16X2: one accumulator for all three segments.
//   BF16X3: three bfloat16 planes (hi + mid + lo = the FP32 value) and six
//           segments [A_h|A_h|A_m|A_h|A_m|A_l] . [X_h;X_m;X_h;X_l;X_m;X_h]: every
//           term down to 2^-16 relative, K = 6 np, no scaling.
//   FP16X2: the lo planes hold residuals times 2^11, so segment 0 (hi*hi) and
//           segments 1-2 (hi*lo, lo*hi) go to two accumulators (512 TMEM
//           columns) combined as acc0 + 2^-11 acc1; A may carry a per-matrix
//           power-of-two scale that the epilogue divides out.
//
// CTA tile 128 x 256, K step 64 (one 128-byte swizzle row of 16-bit values),
// 4-stage TMA -> shared-memory ring guarded by mbarriers. Persistent: one CTA
// per SM walks a static list of tiles; the K axis is accumulated in 256-wide
// chunks, alternately in two TMEM buffers, and each chunk is added into FP32
// registers by the epilogue warps (the tensor core's own FP32 accumulation
// truncates). Warp roles:
//   warp 0  (one thread)  TMA producer
//   warp 1  (one thread)  tcgen05.mma issuer; the whole warp owns the TMEM allocation
//   warps 2-9             epilogue: tcgen05.ld of each chunk (warp w reads TMEM
//                         lanes 32*(w%4) .. +31, columns of half (w-2)/4), then the
//                         fused SP2 branch update (EPI_SQUARE: sigma>0 ? C : 2X - C,
//                         FP32 master and planes written for (i,j) and mirrored to
//                         (j,i), trace / idempotency partials in FP32 per thread and
//                         FP64 across) or a plain FP32 store (EPI_PLAIN).
// Every mbarrier wait is bounded in time; on expiry the CTA raises the
// state's abort flag, waits (bounded) for its own copies in flight and
// returns after freeing its TMEM, and later CTAs exit at once.
#include <cuda.h>

#include <stdio.h>
#include <string.h>

#include "sp2_internal.h"

namespace sp2 {

namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 8;                     // two warps per TMEM lane quarter
constexpr int NUM_THREADS = 64 + 32 * EPI_WARPS;  // TMA warp, MMA warp, epilogue warps
constexpr uint32_t ACC_COLS = 256;               // one 128 x 256 FP32 accumulator
constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;     // two chunk buffers
constexpr int HALF_COLS = BN / 2;                // columns per epilogue thread
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align slack*/ + 256 /*barriers*/;
constexpr unsigned long long TIMEOUT_NS = 2000000000ull;

// Instruction descriptor, kind::f16: D=F32 (bits 4-5 = 1), A and B format at
// bits 7-9 / 10-12 (BF16 = 1, F16 = 0; always the same for A and B), both
// K-major (bits 15,16 = 0), N>>3 at bit 17, M>>4 at bit 24.
constexpr uint32_t idesc_for(bool f16) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of parity `parity` to complete. Gives up (returning
// false) when the abort flag is raised or after TIMEOUT_NS, raising the flag.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* abort_flag) {
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*((volatile int*)abort_flag)) return false;
      if (globaltimer() - t0 > TIMEOUT_NS) {
        atomicExch(abort_flag, 1);
        return false;
      }
    }
  }
}

// Same, ignoring the abort flag (drain of copies in flight), with its own limit.
__device__ void mbar_wait_drain(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > limit_ns) return;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major tile written by TMA with
// 128-byte swizzling: rows of 128 B, 8-row atoms of 1024 B (SBO = 1024),
// LBO unused for this layout (1), descriptor version 1, layout SWIZZLE_128B (2).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// plane kinds of the product kernel
constexpr int KIND_BF16X2 = 0, KIND_FP16X2 = 1, KIND_BF16X3 = 2;

template <int KIND>
__device__ __forceinline__ void split_store(uint16_t* hi, uint16_t* mid, uint16_t* lo, int64_t idx,
                                            float v) {
  uint16_t h, l;
  if constexpr (KIND == KIND_FP16X2) {
    split_fp16(v, 1.0f, h, l);
  } else if constexpr (KIND == KIND_BF16X3) {
    uint16_t m;
    split_bf16x3(v, h, m, l);
    mid[idx] = m;
  } else {
    split_bf16(v, h, l);
  }
  hi[idx] = h;
  lo[idx] = l;
}

template <int KIND>
__device__ __forceinline__ void store_split(float* m, uint16_t* hi, uint16_t* mid, uint16_t* lo,
                                            int64_t idx, float v) {
  m[idx] = v;
  split_store<KIND>(hi, mid, lo, idx, v);
}

template <int KIND>
__global__ void __launch_bounds__(NUM_THREADS, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap mA_hi, const __grid_constant__ CUtensorMap mA_lo,
          const __grid_constant__ CUtensorMap mB_hi, const __grid_constant__ CUtensorMap mB_lo,
          const __grid_constant__ CUtensorMap mA_mid, const __grid_constant__ CUtensorMap mB_mid,
          int nkb, int ch, int epi, int64_t np, float* __restrict__ out,
          uint16_t* __restrict__ out_hi, uint16_t* __restrict__ out_lo,
          uint16_t* __restrict__ out_mid,
          const float* __restrict__ xprev, Part3* __restrict__ part,
          const Tile* __restrict__ tiles, int ntiles, DevState* st, int step,
          const float* __restrict__ a_scale, const float* __restrict__ b_scale,
          float* __restrict__ zmax) {
  constexpr bool F16 = KIND == KIND_FP16X2;
  constexpr bool X3 = KIND == KIND_BF16X3;
  constexpr int NSEG = X3 ? 6 : 3;
  constexpr uint32_t kIdesc = idesc_for(F16);
  {
    const int m = *((volatile const int*)&st->stop_at);
    if ((m != 0 && step > m) || *((volatile const int*)&st->abort_flag)) return;
  }
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;   // [2] chunk accumulated in TMEM buffer b
  uint64_t* tempty = tfull + 2;       // [2] TMEM buffer b drained by the epilogue warps
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  __shared__ double red[2][3][EPI_WARPS];   // per-tile partials, double-buffered by tile parity

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* abortf = &st->abort_flag;
  const int total_kb = NSEG * nkb;
  const int nchunks = total_kb / ch;
  // persistent static schedule: this CTA handles tiles blockIdx.x, +gridDim.x, ...
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mA_hi)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mB_hi)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // k-block counter g runs on across tiles: stage g % STAGES, phase (g / STAGES) & 1
      int64_t issued = 0;
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it) {
        const Tile t = tiles[blockIdx.x + (int64_t)it * gridDim.x];
        for (int kb = 0; kb < total_kb; ++kb) {
          const int64_t g = (int64_t)it * total_kb + kb;
          const int s = (int)(g % STAGES);
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abortf)) {
            ok = false;
            break;
          }
          const int seg = kb / nkb;
          const int kx = (kb - seg * nkb) * BK;
          const CUtensorMap* ma;
          const CUtensorMap* mb;
          if constexpr (X3) {
            // segments hh, hm, mh, hl, mm, lh
            ma = (seg == 2 || seg == 4) ? &mA_mid : (seg == 5 ? &mA_lo : &mA_hi);
            mb = (seg == 1 || seg == 4) ? &mB_mid : (seg == 3 ? &mB_lo : &mB_hi);
          } else {
            ma = seg < 2 ? &mA_hi : &mA_lo;
            mb = seg == 1 ? &mB_lo : &mB_hi;
          }
          uint8_t* sa = smem + s * STAGE_BYTES;
          mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
          tma_load_2d(ma, &full[s], sa, kx, t.row0);
          tma_load_2d(mb, &full[s], sa + A_BYTES, kx, t.col0);
          issued = g + 1;
        }
      }
      if (!ok) {
        // aborted: let the copies already issued land before the CTA exits
        const int64_t first = issued > STAGES ? issued - STAGES : 0;
        for (int64_t g = first; g < issued; ++g)
          mbar_wait_drain(&full[g % STAGES], (uint32_t)(g / STAGES) & 1u, 200000000ull);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it) {
        for (int c = 0; c < nchunks && ok; ++c) {
          const int64_t gc = (int64_t)it * nchunks + c;  // chunk counter across tiles
          const int b = (int)(gc & 1);
          // the epilogue has drained buffer b (chunk gc-2)
          if (!mbar_wait(&tempty[b], ((uint32_t)(gc >> 1) & 1u) ^ 1u, abortf)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dtm = tmem + (uint32_t)b * ACC_COLS;
          for (int kb = c * ch; kb < (c + 1) * ch; ++kb) {
            const int64_t g = (int64_t)it * total_kb + kb;
            const int s = (int)(g % STAGES);
            const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
            if (!mbar_wait(&full[s], ph, abortf)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(smem + s * STAGE_BYTES);
            const uint64_t adesc = sdesc_sw128(a_addr);
            const uint64_t bdesc = sdesc_sw128(a_addr + A_BYTES);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              // advance 16 elements = 32 bytes along K inside the swizzled row: +2 in 16-byte units
              umma_bf16(dtm, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), kIdesc,
                        (kb > c * ch || k > 0) ? 1u : 0u);
            }
            umma_commit(&empty[s]);
          }
          umma_commit(&tfull[b]);
        }
      }
    }
  } else {
    // epilogue warps 2 .. 2+EPI_WARPS-1: warp w reads TMEM lanes 32*(w%4) .. +31 and
    // columns [half*128, half*128+128). Each K chunk is drained from TMEM into
    // FP32 registers with round-to-nearest adds (FP16X2: chunks of the hi*lo
    // segments weighted by 2^-11); the tile's stores follow while the MMA warp
    // already fills the freed TMEM buffers with the next tile's chunks.
    const int e = warp - 2;
    const int q = warp & 3;
    const int half = e >> 2;
    const int r = q * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * HALF_COLS);
    bool ok = true;
    for (int it = 0; it < my_tiles && ok; ++it) {
      const int tix = blockIdx.x + it * gridDim.x;
      const Tile t = tiles[tix];
      const int64_t gi = t.row0 + r;
      float acc[HALF_COLS];
#pragma unroll
      for (int j = 0; j < HALF_COLS; ++j) acc[j] = 0.0f;
      for (int c = 0; c < nchunks; ++c) {
        const int64_t gc = (int64_t)it * nchunks + c;
        const int b = (int)(gc & 1);
        bool w = mbar_wait(&tfull[b], (uint32_t)(gc >> 1) & 1u, abortf);
        w = __all_sync(0xffffffffu, w);
        if (!w) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (epi == EPI_SQUARE && c == nchunks - 2) {
          // the X_n entries the tile-end epilogue reads (512 B of this thread's row):
          // pulled into L2 two chunks ahead, while the MMA warp can run only one
          // chunk ahead of the epilogue
          const float* xr = xprev + gi * np + t.col0 + half * HALF_COLS;
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(xr),
                       "r"((uint32_t)(HALF_COLS * sizeof(float)))
                       : "memory");
        }
        const float wgt = (F16 && (c * ch) >= nkb) ? (1.0f / kLoScale) : 1.0f;
#pragma unroll
        for (int c0 = 0; c0 < HALF_COLS; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(trow + (uint32_t)b * ACC_COLS + (uint32_t)c0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[c0 + j] = fmaf(wgt, __uint_as_float(v[j]), acc[c0 + j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
      if (!ok || *((volatile int*)abortf)) break;
      // per-thread partials over at most 128 entries of one row in FP32 (GB300's FP64
      // rate is a small fraction of its FP32 rate); lanes, warps and tiles add in FP64
      float t1 = 0.0f, t2 = 0.0f, f = 0.0f;
      const int sg = (epi == EPI_SQUARE) ? st->sigma[step] : 1;
      const int64_t bat = gi / np;  // batch entry of this row (stacked A)
      float inv_s = (F16 && a_scale) ? 1.0f / a_scale[bat] : 1.0f;
      if (F16 && b_scale) inv_s /= b_scale[0];
      float zm = 0.0f;
#pragma unroll
      for (int c0 = 0; c0 < HALF_COLS; c0 += 16) {
        float val[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) val[j] = acc[c0 + j] * inv_s;
        const int64_t gj0 = t.col0 + half * HALF_COLS + c0;
        if (epi == EPI_PLAIN) {
          float4* dst = reinterpret_cast<float4*>(out + gi * np + gj0);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            dst[j] = make_float4(val[4 * j], val[4 * j + 1], val[4 * j + 2], val[4 * j + 3]);
#pragma unroll
          for (int j = 0; j < 16; ++j) zm = fmaxf(zm, fabsf(val[j]));
          continue;
        }
        if (gj0 + 15 < gi) continue;  // whole chunk below the diagonal
        float xin[16];  // X_n: the 2X - X^2 branch and the Frobenius idempotency error
        {
          const float4* xp = reinterpret_cast<const float4*>(xprev + gi * np + gj0);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float4 x = xp[j];
            xin[4 * j + 0] = x.x;
            xin[4 * j + 1] = x.y;
            xin[4 * j + 2] = x.z;
            xin[4 * j + 3] = x.w;
          }
        }
        float res[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          res[j] = xin[j] - val[j];
          if (sg < 0) val[j] = 2.0f * xin[j] - val[j];
        }
        if (gj0 >= gi) {
          // whole chunk on or above the diagonal: vector stores
          float4* dm = reinterpret_cast<float4*>(out + gi * np + gj0);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            dm[j] = make_float4(val[4 * j], val[4 * j + 1], val[4 * j + 2], val[4 * j + 3]);
          __align__(16) uint16_t hh[16], ll[16];
          if constexpr (X3) {
            __align__(16) uint16_t mm[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) split_bf16x3(val[j], hh[j], mm[j], ll[j]);
            uint4* dmid = reinterpret_cast<uint4*>(out_mid + gi * np + gj0);
            dmid[0] = reinterpret_cast<const uint4*>(mm)[0];
            dmid[1] = reinterpret_cast<const uint4*>(mm)[1];
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if (F16) split_fp16(val[j], 1.0f, hh[j], ll[j]);
              else split_bf16(val[j], hh[j], ll[j]);
            }
          }
          uint4* dh = reinterpret_cast<uint4*>(out_hi + gi * np + gj0);
          uint4* dl = reinterpret_cast<uint4*>(out_lo + gi * np + gj0);
          dh[0] = reinterpret_cast<const uint4*>(hh)[0];
          dh[1] = reinterpret_cast<const uint4*>(hh)[1];
          dl[0] = reinterpret_cast<const uint4*>(ll)[0];
          dl[1] = reinterpret_cast<const uint4*>(ll)[1];
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (gj0 + j >= gi)
              store_split<KIND>(out, out_hi, out_mid, out_lo, gi * np + gj0 + j, val[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int64_t gj = gj0 + j;
          if (gj < gi) continue;
          const float d = val[j], rr = res[j];
          if (gj == gi) {
            t1 += d;
            t2 = fmaf(d, d, t2);
            f = fmaf(rr, rr, f);
          } else {
            store_split<KIND>(out, out_hi, out_mid, out_lo, gj * np + gi, val[j]);  // mirror (coalesced over lanes)
            t2 = fmaf(2.0f * d, d, t2);
            f = fmaf(2.0f * rr, rr, f);
          }
        }
      }
      if (epi == EPI_PLAIN && zmax) {
        for (int o = 16; o > 0; o >>= 1) zm = fmaxf(zm, __shfl_xor_sync(0xffffffffu, zm, o));
        if (lane == 0 && zm > 0.0f)
          atomicMax(reinterpret_cast<int*>(&zmax[bat]), __float_as_int(zm));
      }
      if (epi == EPI_SQUARE) {
        double d1 = t1, d2 = t2, d3 = f;
        for (int o = 16; o > 0; o >>= 1) {
          d1 += __shfl_xor_sync(0xffffffffu, d1, o);
          d2 += __shfl_xor_sync(0xffffffffu, d2, o);
          d3 += __shfl_xor_sync(0xffffffffu, d3, o);
        }
        const int pb = it & 1;
        if (lane == 0) {
          red[pb][0][e] = d1;
          red[pb][1][e] = d2;
          red[pb][2][e] = d3;
        }
        // epilogue warps only (named barrier 1): one thread writes the tile's partials
        asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
        if (e == 0 && lane == 0) {
          double s1 = 0.0, s2 = 0.0, s3 = 0.0;
          for (int w = 0; w < EPI_WARPS; ++w) {
            s1 += red[pb][0][w];
            s2 += red[pb][1][w];
            s3 += red[pb][2][w];
          }
          part[tix] = Part3{s1, s2, s3};
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2D map over a row-major 16-bit plane (rows x np), box = 64 columns x box_rows rows.
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t np, int box_rows, bool f16) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)np * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

void tc_tile_shape(int* bm, int* bn) {
  *bm = BM;
  *bn = BN;
}

cudaError_t launch_gemm_tc(int mode, int epi, TcOperand A, TcOperand B, int64_t np, MatBuf out,
                           const float* x_prev, Part3* part, const Tile* tiles, int ntiles,
                           DevState* st, int step, const float* a_scale, float* zmax,
                           cudaStream_t s, char* errbuf, size_t errlen, const float* b_scale) {
  if (ntiles <= 0) return cudaSuccess;
  const int kind = mode == SP2_MODE_FP16X2 ? KIND_FP16X2
                                           : (mode == SP2_MODE_BF16X3 ? KIND_BF16X3 : KIND_BF16X2);
  const bool f16 = kind == KIND_FP16X2, x3 = kind == KIND_BF16X3;
  static bool attr_done[3] = {false, false, false};
  if (!attr_done[kind]) {
    cudaError_t e = kind == KIND_FP16X2
                        ? cudaFuncSetAttribute(k_gemm_tc<KIND_FP16X2>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)
                    : kind == KIND_BF16X3
                        ? cudaFuncSetAttribute(k_gemm_tc<KIND_BF16X3>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)
                        : cudaFuncSetAttribute(k_gemm_tc<KIND_BF16X2>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_done[kind] = true;
  }
  // the middle planes exist only in BF16X3; elsewhere the hi maps stand in (never read)
  const uint16_t* a_mid = x3 ? A.mid : A.hi;
  const uint16_t* b_mid = x3 ? B.mid : B.hi;
  if (x3 && (!a_mid || !b_mid || (epi == EPI_SQUARE && !out.mid))) {
    snprintf(errbuf, errlen, "tcgen05 product: BF16X3 operand without its middle plane");
    return cudaErrorInvalidValue;
  }
  // TMA box/stride rules: 16-byte aligned bases, np*2-byte row pitch (np % 256 == 0),
  // every x coordinate a multiple of 64 elements.
  if ((reinterpret_cast<uintptr_t>(A.hi) | reinterpret_cast<uintptr_t>(A.lo) |
       reinterpret_cast<uintptr_t>(B.hi) | reinterpret_cast<uintptr_t>(B.lo) |
       reinterpret_cast<uintptr_t>(a_mid) | reinterpret_cast<uintptr_t>(b_mid)) & 15u ||
      np % 256 != 0 || A.rows % BM != 0 || B.rows % BN != 0) {
    snprintf(errbuf, errlen, "tcgen05 product: operand alignment/shape violates the TMA rules");
    return cudaErrorInvalidValue;
  }
  CUtensorMap ma_hi, ma_lo, mb_hi, mb_lo, ma_mid, mb_mid;
  if (!make_map(&ma_hi, A.hi, A.rows, np, BM, f16) || !make_map(&ma_lo, A.lo, A.rows, np, BM, f16) ||
      !make_map(&mb_hi, B.hi, B.rows, np, BN, f16) || !make_map(&mb_lo, B.lo, B.rows, np, BN, f16) ||
      !make_map(&ma_mid, a_mid, A.rows, np, BM, f16) ||
      !make_map(&mb_mid, b_mid, B.rows, np, BN, f16)) {
    snprintf(errbuf, errlen, "cuTensorMapEncodeTiled failed (driver entry point unavailable?)");
    return cudaErrorInvalidValue;
  }
  const int nkb = (int)(np / BK);
  // K chunk drained from TMEM into FP32 registers: 4 k-blocks (256 products per
  // accumulator pass). np is a multiple of 256, so 4 divides every segment and
  // the lo-plane weight changes only at a chunk boundary. The tensor core's
  // FP32 accumulation truncates, and its bias grows with the chunk length: at
  // N=4096 (FP16X2) 256-wide chunks give a 1.0e-5 density error against the
  // exact form, 512-wide 2.5e-5 and 2048-wide 7.6e-4, for 3% more time per
  // product than 512-wide chunks.
  const int ch = 4;
  // persistent: one CTA per SM (the shared-memory ring allows no second one)
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 1;
  }
  const int grid = ntiles < nsm ? ntiles : nsm;
  float* om = static_cast<float*>(out.master);
  if (kind == KIND_FP16X2)
    k_gemm_tc<KIND_FP16X2><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(
        ma_hi, ma_lo, mb_hi, mb_lo, ma_mid, mb_mid, nkb, ch, epi, np, om, out.hi, out.lo, out.mid,
        x_prev, part, tiles, ntiles, st, step, a_scale, b_scale, zmax);
  else if (kind == KIND_BF16X3)
    k_gemm_tc<KIND_BF16X3><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(
        ma_hi, ma_lo, mb_hi, mb_lo, ma_mid, mb_mid, nkb, ch, epi, np, om, out.hi, out.lo, out.mid,
        x_prev, part, tiles, ntiles, st, step, nullptr, nullptr, nullptr);
  else
    k_gemm_tc<KIND_BF16X2><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(
        ma_hi, ma_lo, mb_hi, mb_lo, ma_mid, mb_mid, nkb, ch, epi, np, om, out.hi, out.lo, out.mid,
        x_prev, part, tiles, ntiles, st, step, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace sp2
