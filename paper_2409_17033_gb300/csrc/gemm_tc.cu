// Split-precision tensor-core product kernel for sm_103a (tcgen05 + TMEM + TMA).
//
// Computes the products of the SP2 path with the hi/lo splitting of Eq.
// doubleHalf and the three-product form of Eq. MixPrecMult / Eq. mults (lo*lo
// dropped):
//     P Q ~ P_hi Q_lo + P_lo Q_hi + P_hi Q_hi,
// evaluated over a concatenated K axis, [P_hi | P_lo | P_hi] . [Q_lo ; Q_hi ; Q_hi],
// into FP32 accumulators in tensor memory: the smaller terms first, hi*hi last.
// Every right factor Q is symmetric, so its row-major planes are directly the
// K-major B operand.
//   BF16X2: bfloat16 planes, one weight for all segments.
//   BF16X3: three bfloat16 planes (hi + mid + lo = the FP32 value) and six
//           segments [P_l|P_m|P_h|P_m|P_h|P_h] . [Q_h;Q_m;Q_l;Q_h;Q_m;Q_h]: every
//           term down to 2^-16 relative, no scaling.
//   FP16X2: the lo planes hold residuals times 2^11; chunks of the hi*lo and
//           lo*hi segments are weighted by 2^-11 when they are drained from
//           TMEM. P may carry a per-matrix power-of-two scale that the epilogue
//           divides out.
// Epilogues:
//   EPI_SQUARE  X_{n+1} = sigma_n > 0 ? X_n^2 : 2 X_n - X_n^2 (Eq. DM0), upper
//               tiles only, mirrored; partials of Tr X_{n+1}, ||X_{n+1}||_F^2 and
//               ||X_n - X_n^2||_F^2 for the branch and stop decisions.
//   EPI_PLAIN   C = P Q stored as it is (FP32).
//   EPI_SYMM    Y_{n+1} = sigma_n > 0 ? Y_n X_n + X_n Y_n : 2 Y_n - (Y_n X_n + X_n Y_n)
//               (Eqs. DM1, DM2, DM3) for a stacked batch of symmetric Y. With X
//               and Y symmetric, (X Y)(I, J) = X(I, :) Y(:, J), so each upper tile
//               of Y X + X Y is ONE accumulation over the doubled K axis
//               [P | Q] . [Q ; P] (P = Y, Q = X): no Z buffer and no transpose
//               pass. Partials of ||Y_{n+1}||_F^2 per tile (FP16X2 plane scales).
//
// CTA tile 128 x 256, K step 64 (one 128-byte swizzle row of 16-bit values),
// 4-stage TMA -> shared-memory ring guarded by mbarriers. Persistent: one CTA
// per SM walks tiles b, b+G, b+2G, ... of a static list. The K axis is
// accumulated in chunks, alternately in two TMEM buffers, and each chunk is
// added into FP32 registers by the epilogue warps (the tensor core's own FP32
// accumulation truncates, with a bias that grows with the chunk): 256-wide for
// hi*hi, up to 16384-wide (FP16X2, weight 2^-11) or 2048-wide (bfloat16 modes,
// 2^-8) for the cross terms. A tile starts with the long chunks, so the spare
// TMEM buffer covers the previous tile's stores.
//
// CTA pairs (CG = 2, a cluster of two): a 256 x 256 tile per pair, one
// tcgen05.mma.cta_group::2 stream of M = 256 issued by rank 0. Each CTA loads
// its own 128 rows of the A tile and 128 rows of the B tile into a 6-stage ring
// of 32 KB stages and drains its own 128 accumulator rows; rank 1's warp 1
// passes each landed stage on to rank 0's barrier, and rank 1's epilogue warps
// report drained TMEM buffers there. Same arithmetic and order as one SM.
//
// Warp roles:
//   warp 0  (one thread)  TMA producer
//   warp 1  (one thread)  tcgen05.mma issuer (pair: rank 1's relays stages); the
//                         whole warp owns the TMEM allocation
//   warps 2-17            epilogue: tcgen05.ld of each chunk (warp w reads TMEM lanes
//                         32*(w%4) .. +31, the 64 columns of group (w-2)/4), then
//                         the epilogue above. With 64 columns per thread the chunk
//                         drain (the tensor pipe's critical path: the MMA warp runs
//                         at most one chunk ahead) and the tile-end stores are spread
//                         over twice as many warps as with 128.
// Every mbarrier wait is bounded in time (a launch parameter, default 2 s); on
// expiry the CTA raises the state's abort flag, waits (bounded) for its own
// copies and tensor-core operations in flight, frees its TMEM and returns, and
// later CTAs exit at once.
#include <cuda.h>

#include <stdio.h>
#include <string.h>

#include <mutex>

#include "sp2_internal.h"

namespace sp2 {

namespace {

constexpr int BM = 128;        // output rows per CTA (a CTA pair's tile has 2 BM)
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int A_BYTES = BM * BK * 2;
// Per-CTA ring geometry for CG CTAs per tile: a CTA of a pair holds half of the
// right factor's rows, so its stage is 32 KB and six stages fit.
template <int CG>
struct Ring {
  static constexpr int B_ROWS = BN / CG;
  static constexpr int B_BYTES = B_ROWS * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = CG == 1 ? 4 : 6;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align slack*/ + 256 /*barriers*/;
};
constexpr int EPI_WARPS = 16;                    // four warps per TMEM lane quarter
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int NUM_THREADS = 64 + EPI_THREADS;    // TMA warp, MMA warp, epilogue warps
constexpr uint32_t ACC_COLS = 256;               // one 128 x 256 FP32 accumulator
constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;     // two chunk buffers
constexpr int COL_GROUPS = EPI_WARPS / 4;        // column groups of a tile
constexpr int TCOLS = BN / COL_GROUPS;            // columns per epilogue thread
constexpr unsigned long long DRAIN_NS = 200000000ull;

// Instruction descriptor, kind::f16: D=F32 (bits 4-5 = 1), A and B format at
// bits 7-9 / 10-12 (BF16 = 1, F16 = 0; always the same for A and B), both
// K-major (bits 15,16 = 0), N>>3 at bit 17, M>>4 at bit 24. M is the rows of
// one instruction: BM, or 2 BM for a CTA pair.
constexpr uint32_t idesc_for(bool f16, int m) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
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

// CL: acquire at cluster scope, for barriers that the peer CTA of a pair arrives
// on (or that its tensor-core operations signal)
template <bool CL = false>
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  if constexpr (CL) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return ok != 0;
}

// Wait for the phase of parity `parity` to complete. Gives up (returning
// false) when the abort flag is raised or after limit_ns, raising the flag.
template <bool CL = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* abort_flag,
                                          unsigned long long limit_ns) {
  if (mbar_try_wait<CL>(bar, parity)) return true;   // no clock read when it is ready
  const unsigned long long t0 = globaltimer();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait<CL>(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*((volatile int*)abort_flag)) return false;
      if (globaltimer() - t0 > limit_ns) {
        atomicExch(abort_flag, 1);
        return false;
      }
    }
  }
}

// Same, ignoring the abort flag (drain of work in flight), with its own limit.
__device__ void mbar_wait_drain(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > limit_ns) return;
}

// ---- CTA pairs (cluster of two; rank 0 issues the copies and the MMAs)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(uint32_t addr, uint32_t rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(addr), "r"(rank));
  return d;
}

// every thread of both CTAs (barrier initialisation and TMEM ownership before,
// shared-memory and TMEM lifetime after the work)
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// Arrive on a barrier of the peer CTA. Relaxed for the drained-TMEM signal: the
// waiter relies only on this thread's TMEM reads being done, which
// tcgen05.wait::ld already guarantees in program order (a release would first
// wait for every global store of the tile-end epilogue to become visible
// cluster-wide). Release for the relayed stage-ready signal, which passes on the
// visibility of the TMA writes this thread has just observed.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster_release(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar)
               : "memory");
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

// Stage and phase parity of a running k-block counter in a ring of STAGES
// stages, advanced by one per k-block without a division: the loops of the
// copy issuer and the MMA issuer (one thread each) are on the tensor pipe's
// critical path, and a 64-bit division by the stage count per k-block
// measurably delayed the MMA issue.
template <int STAGES>
struct RingPos {
  int s = 0;
  uint32_t ph = 0;
  __device__ __forceinline__ void next() {
    if (++s == STAGES) {
      s = 0;
      ph ^= 1u;
    }
  }
};

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

// CG = 2: one instruction of M = 256 over the CTA pair. A's rows 0-127 and B's
// columns 0-127 come from this CTA's shared memory, A's rows 128-255 and B's
// columns 128-255 from the same offsets in the peer's; D rows 0-127 land in this
// CTA's TMEM, rows 128-255 in the peer's, at the same address.
template <int CG>
__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  if constexpr (CG == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  }
}

// arrive on `bar` of this CTA once the tensor-core operations issued so far are done
template <int CG>
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  if constexpr (CG == 2)
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
  else
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// the same, arriving on the barrier at this offset in both CTAs of the pair
__device__ __forceinline__ void umma_commit_both(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"((uint16_t)3)
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

// 256-bit global accesses (sm_100 and later; 32-byte aligned addresses): one lane
// moves a full 32-byte sector, where 128-bit accesses by lanes on different rows
// would each fill half a sector.
__device__ __forceinline__ void st256(void* p, const uint32_t (&v)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

__device__ __forceinline__ void st256f(float* p, const float* v) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]),
               "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}

__device__ __forceinline__ void ld256f(const float* p, float* v) {
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                 "=f"(v[6]), "=f"(v[7])
               : "l"(p)
               : "memory");
}

// A sum of FP32 terms w x^2 (w a power of two) kept to about 2^-45 of its value
// before it goes to FP64, at FP32 rates (GB300's FP64 rate is a small fraction
// of its FP32 rate): each square enters as its rounded value plus its fmaf
// residual (exact), each addition as TwoSum (Knuth) with its rounding error
// carried in c. The _rn intrinsics keep the compiler from contracting the steps
// into fused operations, which would lose the error terms.
struct ExactSqSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add_sq(float w, float x) {
    const float wx = w * x;                 // exact: w is 1 or 2
    const float p = __fmul_rn(wx, x);
    const float e = fmaf(wx, x, -p);        // wx x - p exactly
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));   // s + p - t
    c = __fadd_rn(c, __fadd_rn(err, e));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// plane kinds of the product kernel
constexpr int KIND_BF16X2 = 0, KIND_FP16X2 = 1, KIND_BF16X3 = 2;
// plane indices of an operand: 0 = hi, 1 = lo, 2 = mid (BF16X3)
constexpr int PL_HI = 0, PL_LO = 1, PL_MID = 2;

// Planes of the left and right factor in base segment `seg` of a split product
// of nbase segments (K-concatenated), smallest terms first and hi*hi last: the
// FP32 register sum then adds terms in increasing size, and a tile starts with
// the long cross-term chunks, which is what the spare TMEM buffer overlaps with
// the previous tile's stores. nbase == 1 (split-tail bulk): hi*hi alone.
template <int KIND>
__device__ __forceinline__ void seg_planes(int seg, int nbase, int& pa, int& pb) {
  if (seg == nbase - 1) {
    pa = pb = PL_HI;
  } else if constexpr (KIND == KIND_BF16X3) {
    // lh, mm, hl (2^-16 of hh), mh, hm (2^-8), then hh
    pa = seg == 0 ? PL_LO : ((seg == 1 || seg == 3) ? PL_MID : PL_HI);
    pb = seg == 2 ? PL_LO : ((seg == 1 || seg == 4) ? PL_MID : PL_HI);
  } else {
    // hl, lh, then hh
    pa = seg == 1 ? PL_LO : PL_HI;
    pb = seg == 0 ? PL_LO : PL_HI;
  }
}

template <int KIND>
__device__ __forceinline__ void split_store(uint16_t* hi, uint16_t* mid, uint16_t* lo, int64_t idx,
                                            float v, float scale) {
  uint16_t h, l;
  if constexpr (KIND == KIND_FP16X2) {
    split_fp16(v, scale, h, l);
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
                                            int64_t idx, float v, float scale) {
  m[idx] = v;
  split_store<KIND>(hi, mid, lo, idx, v, scale);
}

struct KParams {
  int nkb;                 // k-blocks (of BK) per segment: np / BK
  int ch;                  // k-blocks per TMEM chunk of a product's leading (hi x hi) segment
  int ch_lo;               // k-blocks per TMEM chunk of its other segments
  int nbase;               // segments of one split product (3, or 6 for BF16X3)
  int nseg;                // segments on the K axis (nbase, or 2 nbase for EPI_SYMM)
  int64_t np;
  float* out;
  uint16_t* out_hi;
  uint16_t* out_lo;
  uint16_t* out_mid;
  const float* prev;       // EPI_SQUARE: X_n; EPI_SYMM: Y_n (stacked like out)
  Part3* part;             // per-tile partials
  const Tile* tiles;
  int ntiles;
  DevState* st;
  int step;
  const float* p_scale;    // FP16X2: per batch entry of P, the plane scale to divide out
  const float* q_scale;    // FP16X2: the plane scale of Q (nullable)
  const float* o_scale;    // FP16X2 EPI_SYMM: per batch entry, scale of the output planes
  float* zmax;             // FP16X2 EPI_PLAIN: per batch entry, receives max |C|
  unsigned long long wait_ns;
  int withhold;            // test hook: CTA 0 never issues its first load
  int tail;                // split-tail mode: st->plane1[step] selects the hi planes alone
  // block-sparse square (SPARSE kernels): the tile count, and per tile its listed
  // 256-wide K blocks klist[tix * nbk .. + kcnt[tix]], all written on the device
  const int* dyn_ntiles;
  const int* kcnt;
  const uint16_t* klist;
  int nbk;
};

// Tensor maps of one launch: the left factor's planes with 128-row boxes (A role)
// and the right factor's with 256-row boxes (B role; 128 rows for a CTA pair,
// which loads each half separately); EPI_SYMM also reads X in
// the A role and Y in the B role (its second half, [X | .] . [. ; Y]).
struct KMaps {
  CUtensorMap pa[3];   // P planes (hi, lo, mid), A role
  CUtensorMap qb[3];   // Q planes, B role
  CUtensorMap qa[3];   // Q planes, A role (EPI_SYMM)
  CUtensorMap pb[3];   // P planes, B role (EPI_SYMM)
};

// The stores and partials of one finished tile: row r of the tile, columns
// [grp * 64, grp * 64 + 64); acc holds this thread's FP32 sums; the tile's
// partials (of this CTA's rows) go to p.part[pidx]. The epilogue
// is a template parameter, so that each kernel carries only its own code (a
// smaller kernel keeps the producer's and the MMA issuer's loops in the
// instruction cache).
template <int KIND, int EPI>
__device__ __forceinline__ void tile_end(const KParams& p, float (&acc)[TCOLS], int tix, int pidx,
                                         int it, int e, int lane, int grp, int r, int sg,
                                         double (*red)[3][EPI_WARPS]) {
  constexpr bool F16 = KIND == KIND_FP16X2;
  constexpr bool X3 = KIND == KIND_BF16X3;
  const int64_t np = p.np;
  const Tile t = p.tiles[tix];
  const int64_t bat = EPI == EPI_SQUARE ? 0 : t.row0 / np;   // batch entry (stacked P)
  const int64_t gi = t.row0 + r;                               // stacked row
  const int64_t li = gi - bat * np;                            // row within its matrix
  float inv_s = 1.0f;
  if constexpr (F16) {
    if (p.p_scale) inv_s = 1.0f / p.p_scale[bat];
    if (p.q_scale) inv_s /= p.q_scale[0];
  }
  if constexpr (EPI == EPI_PLAIN) {
    float zm = 0.0f;
#pragma unroll
    for (int c0 = 0; c0 < TCOLS; c0 += 16) {
      float* dst = p.out + gi * np + t.col0 + grp * TCOLS + c0;
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        v[j] = acc[c0 + j] * inv_s;
        zm = fmaxf(zm, fabsf(v[j]));
      }
      st256f(dst, v);
      st256f(dst + 8, v + 8);
    }
    if (p.zmax) {
      for (int o = 16; o > 0; o >>= 1) zm = fmaxf(zm, __shfl_xor_sync(0xffffffffu, zm, o));
      if (lane == 0 && zm > 0.0f) atomicMax(reinterpret_cast<int*>(&p.zmax[bat]), __float_as_int(zm));
    }
  } else {
    // X_{n+1} (EPI_SQUARE: C = X_n^2) or Y_{n+1} (EPI_SYMM: C = Y_n X_n + X_n Y_n) is
    // C for sigma > 0 and 2 M_n - C for sigma < 0 (M_n the previous iterate)
    const float os = (F16 && EPI == EPI_SYMM && p.o_scale) ? p.o_scale[bat] : 1.0f;
    const int64_t mbase = bat * np * np;   // first entry of this batch entry's matrix
    // per-thread partials over at most 64 entries of one row, the squares summed
    // with their rounding errors (FP64-equivalent); lanes, warps and tiles add in
    // FP64: Tr, ||.||_F^2 and (EPI_SQUARE) ||X_n - X_n^2||_F^2, whose residual is
    // X_n - X_{n+1} up to its sign in either branch. Tr takes the one diagonal
    // entry a thread's row segment can hold, as it is.
    float t1 = 0.0f;
    ExactSqSum t2, f;
#pragma unroll
    for (int c0 = 0; c0 < TCOLS; c0 += 16) {
      const int64_t gj0 = t.col0 + grp * TCOLS + c0;
      if (gj0 + 15 < li) continue;  // whole group below the diagonal
      float val[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) val[j] = acc[c0 + j] * inv_s;
      {
        float xin[16];
        if (EPI == EPI_SQUARE || sg < 0) {
          const float* xp = p.prev + gi * np + gj0;
          ld256f(xp, xin);
          ld256f(xp + 8, xin + 8);
          if (sg < 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) val[j] = 2.0f * xin[j] - val[j];
          }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int64_t gj = gj0 + j;
          if (gj < li) continue;
          const float d = val[j], w2 = gj == li ? 1.0f : 2.0f;
          if (gj == li) t1 += d;
          t2.add_sq(w2, d);
          if constexpr (EPI == EPI_SQUARE) f.add_sq(w2, xin[j] - d);
        }
      }
      uint32_t wh[8], wl[8], wm[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint16_t h0, h1, l0, l1, m0 = 0, m1 = 0;
        if constexpr (X3) {
          split_bf16x3(val[2 * j], h0, m0, l0);
          split_bf16x3(val[2 * j + 1], h1, m1, l1);
        } else if constexpr (F16) {
          split_fp16(val[2 * j], os, h0, l0);
          split_fp16(val[2 * j + 1], os, h1, l1);
        } else {
          split_bf16(val[2 * j], h0, l0);
          split_bf16(val[2 * j + 1], h1, l1);
        }
        wh[j] = (uint32_t)h0 | ((uint32_t)h1 << 16);
        wl[j] = (uint32_t)l0 | ((uint32_t)l1 << 16);
        wm[j] = (uint32_t)m0 | ((uint32_t)m1 << 16);
      }
      if (gj0 >= li) {
        const int64_t o = gi * np + gj0;
        st256f(p.out + o, val);
        st256f(p.out + o + 8, val + 8);
        st256(p.out_hi + o, wh);
        st256(p.out_lo + o, wl);
        if constexpr (X3) st256(p.out_mid + o, wm);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (gj0 + j >= li) {
            const int64_t o = gi * np + gj0 + j;
            const int sh = 16 * (j & 1);
            p.out[o] = val[j];
            p.out_hi[o] = (uint16_t)(wh[j >> 1] >> sh);
            p.out_lo[o] = (uint16_t)(wl[j >> 1] >> sh);
            if constexpr (X3) p.out_mid[o] = (uint16_t)(wm[j >> 1] >> sh);
          }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int64_t gj = gj0 + j;
        if (gj <= li) continue;
        const int64_t o = mbase + gj * np + li;
        const int sh = 16 * (j & 1);
        p.out[o] = val[j];
        p.out_hi[o] = (uint16_t)(wh[j >> 1] >> sh);
        p.out_lo[o] = (uint16_t)(wl[j >> 1] >> sh);
        if constexpr (X3) p.out_mid[o] = (uint16_t)(wm[j >> 1] >> sh);
      }
    }
    double d1 = t1, d2 = t2.value(), d3 = f.value();
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
    asm volatile("bar.sync 1, %0;" ::"r"(EPI_THREADS) : "memory");
    if (e == 0 && lane == 0) {
      double s1 = 0.0, s2 = 0.0, s3 = 0.0;
      for (int w = 0; w < EPI_WARPS; ++w) {
        s1 += red[pb][0][w];
        s2 += red[pb][1][w];
        s3 += red[pb][2][w];
      }
      p.part[pidx] = Part3{s1, s2, s3};
    }
  }
}

// Block-sparse squares: the end (exclusive) of the run of listed K blocks that
// starts at list position q0 and stays inside one dense cross-term chunk (gsz
// blocks of 256), so that with every block listed the chunks are the dense ones.
__device__ __forceinline__ int sparse_run_end(const uint16_t* kl, int kc, int gsz, int q0) {
  const int grp = kl[q0] / gsz;
  int q1 = q0 + 1;
  while (q1 < kc && kl[q1] / gsz == grp) ++q1;
  return q1;
}

// SPARSE (square on CTA pairs only): the tile list, its length and every tile's
// K blocks come from the device (the block-sparse plan); a tile's K axis is its
// listed 256-wide blocks in each segment, hi*hi drained per block and a cross
// term per run of listed blocks inside one dense cross-term chunk, so that with
// every block listed the chunks, and the results, are the dense kernel's. The
// sparse loops are separate from the dense ones, which the SPARSE = false
// kernels alone contain.
template <int KIND, int EPI, int CG, bool SPARSE = false>
__global__ void __launch_bounds__(NUM_THREADS, 1)
k_gemm_tc(const __grid_constant__ KMaps maps, const __grid_constant__ KParams p) {
  static_assert(!SPARSE || (EPI == EPI_SQUARE && CG == 2), "block-sparse squares run on pairs");
  using R = Ring<CG>;
  constexpr int STAGES = R::STAGES;
  constexpr int STAGE_BYTES = R::STAGE_BYTES;
  constexpr bool PAIR = CG == 2;
  constexpr bool F16 = KIND == KIND_FP16X2;
  constexpr uint32_t kIdesc = idesc_for(F16, BM * CG);
  DevState* st = p.st;
  {
    // a pair must take this exit together: stop_at is fixed for the launch, while
    // the abort flag may be raised meanwhile (a pair sees it in its waits instead)
    const int m = *((volatile const int*)&st->stop_at);
    if ((m != 0 && p.step > m) || (!PAIR && *((volatile const int*)&st->abort_flag))) return;
  }
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* pfull = empty + STAGES;   // pair, rank 0: the peer's stage s has landed
  uint64_t* tfull = pfull + STAGES;   // [2] chunk accumulated in TMEM buffer b
  uint64_t* tempty = tfull + 2;       // [2] TMEM buffer b drained by the epilogue warps
  uint64_t* mdone = tempty + 2;       // abort path: the MMA issuer's last operations done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  __shared__ double red[2][3][EPI_WARPS];   // per-tile partials, double-buffered by tile parity

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* abortf = &st->abort_flag;
  // a pair: each CTA loads its own halves of both operands (rows rank*128 .. of the
  // A tile and of the B tile) and drains its own TMEM rows; rank 0 issues the MMAs
  // once its own stage and (relayed by rank 1's warp 1) the peer's have landed.
  // Tiles are indexed per pair.
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool issuer = rank == 0;
  const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int nunits = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  // segments of this launch: the split product, or in the split-tail mode's bulk
  // steps the hi planes alone (one segment; two for the symmetric response)
  const int nbase = (p.tail && st->plane1[p.step]) ? 1 : p.nbase;
  const int nseg = EPI == EPI_SYMM ? 2 * nbase : nbase;
  const int total_kb = nseg * p.nkb;
  // TMEM chunks: the hi x hi segment of each split product (the last of its
  // nbase segments; every segment in the split-tail bulk) every ch k-blocks, the
  // smaller cross terms every ch_lo; both divide nkb, so no chunk spans two segments
  const int ch_hi = p.ch, ch_lo = nbase == 1 ? p.ch : p.ch_lo;
  const int nchunks = (nseg / nbase) * (p.nkb / ch_hi + (nbase - 1) * (p.nkb / ch_lo));
  auto chunk_len = [&](int kb0) {
    return ((kb0 / p.nkb) % nbase) == nbase - 1 ? ch_hi : ch_lo;
  };
  // persistent static schedule: this CTA (pair) handles tiles unit, unit + nunits, ...
  // (block-sparse: the tile count comes from the device)
  int ntiles = p.ntiles;
  if constexpr (SPARSE) ntiles = *((volatile const int*)p.dyn_ntiles);
  const int my_tiles = unit < ntiles ? (ntiles - 1 - unit) / nunits + 1 : 0;
  // block-sparse: a cross-term chunk is a run of listed K blocks inside one dense
  // chunk of ch_lo k-blocks (gsz K blocks of 256)
  const int gsz = p.ch_lo >> 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&pfull[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], CG * EPI_WARPS);   // a pair's rank 0 hears both CTAs' warps
    }
    mbar_init(mdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.pa[0])) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.qb[0])) : "memory");
  }
  if (warp == 1) {
    // a pair allocates the same columns in both CTAs, one warp of each taking part
    if constexpr (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if constexpr (SPARSE) {
     if (lane == 0) {
      // block-sparse square: every segment walks the tile's listed K blocks
      int64_t g = 0;
      RingPos<STAGES> rp;
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it) {
        const int tix = unit + it * nunits;
        const Tile t = p.tiles[tix];
        const int kc = p.kcnt[tix];
        const uint16_t* kl = p.klist + (int64_t)tix * p.nbk;
        for (int seg = 0; seg < nseg && ok; ++seg) {
          int pa, pb;
          seg_planes<KIND>(seg, nbase, pa, pb);
          for (int u = 0; u < 4 * kc; ++u, ++g, rp.next()) {
            const int s = rp.s;
            const uint32_t ph = rp.ph;
            if (!mbar_wait<PAIR>(&empty[s], ph ^ 1u, abortf, p.wait_ns)) {
              ok = false;
              break;
            }
            if (p.withhold && blockIdx.x == 0 && g == 0) continue;  // test hook: never completes
            const int kx = (int)kl[u >> 2] * (4 * BK) + (u & 3) * BK;
            uint8_t* sa = smem + s * STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(&maps.pa[pa], &full[s], sa, kx, t.row0 + (int)rank * BM);
            tma_load_2d(&maps.qb[pb], &full[s], sa + A_BYTES, kx, t.col0 + (int)rank * R::B_ROWS);
          }
        }
      }
      if (!ok) {
        const int64_t first = g > STAGES ? g - STAGES : 0;
        for (int64_t q = first; q < g; ++q) {
          if (p.withhold && blockIdx.x == 0 && q == 0) continue;
          mbar_wait_drain(&full[q % STAGES], (uint32_t)(q / STAGES) & 1u, DRAIN_NS);
        }
      }
     }
    } else if (lane == 0) {
      const int64_t np = p.np;
      const int nkb = p.nkb;
      // k-block counter g runs on across tiles: stage g % STAGES, phase (g / STAGES) & 1
      int64_t g = 0;
      RingPos<STAGES> rp;
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it) {
        const Tile t = p.tiles[unit + it * nunits];
        const int bat = (int)(t.row0 / np);
        for (int seg = 0; seg < nseg && ok; ++seg) {
          // the segment's operands and tile rows, fixed over its k-blocks
          const bool swap = EPI == EPI_SYMM && seg >= nbase;   // second half: [Q | .] . [. ; P]
          int pa, pb;
          seg_planes<KIND>(swap ? seg - nbase : seg, nbase, pa, pb);
          const CUtensorMap* ma = swap ? &maps.qa[pa] : &maps.pa[pa];
          const CUtensorMap* mb = swap ? &maps.pb[pb] : &maps.qb[pb];
          // this CTA's halves: rows [rank*128, +128) of the A tile, [rank*B_ROWS, +B_ROWS)
          // of the B tile (one CTA: all of both)
          const int arow = (swap ? t.row0 - bat * (int)np : t.row0) + (int)rank * BM;
          const int brow = (swap ? bat * (int)np + t.col0 : t.col0) + (int)rank * R::B_ROWS;
          for (int kx = 0; kx < nkb * BK; kx += BK, ++g, rp.next()) {
            const int s = rp.s;
            if (!mbar_wait<PAIR>(&empty[s], rp.ph ^ 1u, abortf, p.wait_ns)) {
              ok = false;
              break;
            }
            if (p.withhold && blockIdx.x == 0 && g == 0) continue;  // test hook: never completes
            uint8_t* sa = smem + s * STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(ma, &full[s], sa, kx, arow);
            tma_load_2d(mb, &full[s], sa + A_BYTES, kx, brow);
          }
        }
      }
      if (!ok) {
        // aborted: let the copies already issued land before the CTA exits
        const int64_t first = g > STAGES ? g - STAGES : 0;
        for (int64_t q = first; q < g; ++q) {
          if (p.withhold && blockIdx.x == 0 && q == 0) continue;
          mbar_wait_drain(&full[q % STAGES], (uint32_t)(q / STAGES) & 1u, DRAIN_NS);
        }
      }
    }
  } else if (warp == 1) {
    if (PAIR && !issuer && lane == 0) {
      // rank 1: pass each landed stage of this CTA on to rank 0's MMA issuer
      const uint32_t pfull_peer = cluster_addr(smem_u32(pfull), 0);
      int64_t total = (int64_t)my_tiles * total_kb;
      if constexpr (SPARSE) {
        total = 0;
        for (int it = 0; it < my_tiles; ++it) total += (int64_t)nseg * 4 * p.kcnt[unit + it * nunits];
      }
      RingPos<STAGES> rp;
      for (int64_t g = 0; g < total; ++g, rp.next()) {
        if (!mbar_wait<PAIR>(&full[rp.s], rp.ph, abortf, p.wait_ns)) break;
        mbar_arrive_cluster_release(pfull_peer + (uint32_t)(rp.s * sizeof(uint64_t)));
      }
    } else if constexpr (SPARSE) {
     if (lane == 0 && issuer) {
      bool ok = true;
      int64_t g = 0, gc = 0;
      RingPos<STAGES> rp;
      const uint64_t adesc0 = sdesc_sw128(smem_u32(smem));
      for (int it = 0; it < my_tiles && ok; ++it) {
        const int tix = unit + it * nunits;
        const int kc = p.kcnt[tix];
        const uint16_t* kl = p.klist + (int64_t)tix * p.nbk;
        for (int seg = 0; seg < nseg && ok; ++seg) {
          const bool hh = seg == nbase - 1;
          for (int q0 = 0; q0 < kc && ok; ++gc) {
            const int q1 = hh ? q0 + 1 : sparse_run_end(kl, kc, gsz, q0);
            const int b = (int)(gc & 1);
            if (!mbar_wait<PAIR>(&tempty[b], ((uint32_t)(gc >> 1) & 1u) ^ 1u, abortf, p.wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dtm = tmem + (uint32_t)b * ACC_COLS;
            for (int u = 4 * q0; u < 4 * q1; ++u, ++g, rp.next()) {
              const int s = rp.s;
              const uint32_t ph = rp.ph;
              if (!mbar_wait<false>(&full[s], ph, abortf, p.wait_ns) ||
                  !mbar_wait<PAIR>(&pfull[s], ph, abortf, p.wait_ns)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint64_t adesc = adesc0 + (uint64_t)(s * (STAGE_BYTES >> 4));
              const uint64_t bdesc = adesc + (uint64_t)(A_BYTES >> 4);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k)
                umma_f16<CG>(dtm, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), kIdesc,
                             (u > 4 * q0 || k > 0) ? 1u : 0u);
              umma_commit_both(&empty[s]);
            }
            if (ok) umma_commit_both(&tfull[b]);
            q0 = q1;
          }
        }
      }
      if (!ok) {
        umma_commit<CG>(mdone);
        mbar_wait_drain(mdone, 0, DRAIN_NS);
      }
     }
    } else if (lane == 0 && issuer) {
      bool ok = true;
      int64_t g = 0, gc = 0;   // k-block and chunk counters across tiles
      RingPos<STAGES> rp;
      // descriptors of a stage: the ring's base descriptor plus the stage offset in
      // 16-byte units (the address field holds bits 4-17 of a shared-memory address
      // below 256 KB, so the addition never carries out of it)
      const uint64_t adesc0 = sdesc_sw128(smem_u32(smem));
      for (int it = 0; it < my_tiles && ok; ++it) {
        int kb0 = 0;   // first k-block of chunk c within the tile
        int segb = 0, kin = 0;   // base segment (seg % nbase) and k-block within the segment
        for (int c = 0; c < nchunks && ok; ++c, ++gc) {
          const int len = segb == nbase - 1 ? ch_hi : ch_lo;   // chunk_len(kb0), no division
          kin += len;
          if (kin == p.nkb) {
            kin = 0;
            if (++segb == nbase) segb = 0;
          }
          const int b = (int)(gc & 1);
          // the epilogue (of both CTAs of a pair) has drained buffer b (chunk gc-2)
          if (!mbar_wait<PAIR>(&tempty[b], ((uint32_t)(gc >> 1) & 1u) ^ 1u, abortf, p.wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dtm = tmem + (uint32_t)b * ACC_COLS;
          for (int kb = kb0; kb < kb0 + len; ++kb, ++g, rp.next()) {
            const int s = rp.s;
            const uint32_t ph = rp.ph;
            // this CTA's own stage (its own copies: CTA-scope acquire), then, on a
            // pair, the peer's stage as relayed by its warp 1
            if (!mbar_wait<false>(&full[s], ph, abortf, p.wait_ns) ||
                (PAIR && !mbar_wait<PAIR>(&pfull[s], ph, abortf, p.wait_ns))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t adesc = adesc0 + (uint64_t)(s * (STAGE_BYTES >> 4));
            const uint64_t bdesc = adesc + (uint64_t)(A_BYTES >> 4);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              // advance 16 elements = 32 bytes along K inside the swizzled row: +2 in 16-byte units
              umma_f16<CG>(dtm, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), kIdesc,
                           (kb > kb0 || k > 0) ? 1u : 0u);
            }
            // the stage is free in both CTAs once these MMAs have read it
            if constexpr (PAIR) umma_commit_both(&empty[s]);
            else umma_commit<CG>(&empty[s]);
          }
          if (ok) {
            if constexpr (PAIR) umma_commit_both(&tfull[b]);
            else umma_commit<CG>(&tfull[b]);
          }
          kb0 += len;
        }
      }
      if (!ok) {
        // aborted: the tensor-core operations already issued still read the ring and
        // write TMEM; one more commit tracks all of them (bounded wait) before dealloc
        umma_commit<CG>(mdone);
        mbar_wait_drain(mdone, 0, DRAIN_NS);
      }
    }
  } else {
    // epilogue warps 2 .. 2+EPI_WARPS-1: warp w reads TMEM lanes 32*(w%4) .. +31 and
    // columns [grp*64, grp*64+64). Each K chunk is drained from TMEM into
    // FP32 registers with round-to-nearest adds; the tile's stores follow while
    // the MMA warp already fills the freed TMEM buffers with the next tile's chunks.
    // The drain loop is the tensor pipe's critical path (the MMA warp runs at most
    // one chunk ahead), so it keeps nothing live beyond the accumulator.
    const int e = warp - 2;
    const int q = warp & 3;
    const int grp = e >> 2;
    const int r = (int)rank * BM + q * 32 + lane;   // row within the (pair) tile
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(grp * TCOLS);
    // a pair's rank 1 reports drained buffers to rank 0's barrier
    const uint32_t tempty_peer = PAIR && !issuer ? cluster_addr(smem_u32(tempty), 0) : 0u;
    // the branch of this step (uniform over the launch); the previous iterate is
    // read by the square and, for sigma < 0, by the response update
    const int sg = EPI == EPI_PLAIN ? 1 : p.st->sigma[p.step];
    const bool need_prev = EPI == EPI_SQUARE || (EPI == EPI_SYMM && sg < 0);
    bool ok = true;
    int64_t gc = 0;
    for (int it = 0; it < my_tiles && ok; ++it) {
      const int tix = unit + it * nunits;
      // the previous-iterate entries the tile-end epilogue reads (256 B of this
      // thread's row), pulled into L2 two chunks ahead of the tile's end
      const float* pf = nullptr;
      if (need_prev) {
        const Tile t = p.tiles[tix];
        pf = p.prev + ((int64_t)t.row0 + r) * p.np + t.col0 + grp * TCOLS;
      }
      float acc[TCOLS];
#pragma unroll
      for (int j = 0; j < TCOLS; ++j) acc[j] = 0.0f;
      if constexpr (SPARSE) {
        // the listed K blocks: hi*hi chunks one block each, cross-term chunks by runs
        const int kc = p.kcnt[tix];
        const uint16_t* kl = p.klist + (int64_t)tix * p.nbk;
        int nruns = 0;
        for (int q0 = 0; q0 < kc; q0 = sparse_run_end(kl, kc, gsz, q0)) ++nruns;
        const int nch = (nbase - 1) * nruns + kc;
        int c = 0;
        for (int seg = 0; seg < nseg && ok; ++seg) {
          const bool hh = seg == nbase - 1;
          for (int q0 = 0; q0 < kc; ++c, ++gc) {
            q0 = hh ? q0 + 1 : sparse_run_end(kl, kc, gsz, q0);
            const int b = (int)(gc & 1);
            bool w = mbar_wait<PAIR>(&tfull[b], (uint32_t)(gc >> 1) & 1u, abortf, p.wait_ns);
            w = __all_sync(0xffffffffu, w);
            if (!w) {
              ok = false;
              break;
            }
            tc_fence_after();
            if (pf && c == nch - 2)
              asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pf),
                           "r"((uint32_t)(TCOLS * sizeof(float)))
                           : "memory");
            float wgt = 1.0f;
            if constexpr (F16) wgt = hh ? 1.0f : 1.0f / kLoScale;
#pragma unroll
            for (int c0 = 0; c0 < TCOLS; c0 += 16) {
              uint32_t v[16];
              tmem_ld16(trow + (uint32_t)b * ACC_COLS + (uint32_t)c0, v);
#pragma unroll
              for (int j = 0; j < 16; ++j) acc[c0 + j] = fmaf(wgt, __uint_as_float(v[j]), acc[c0 + j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if (!issuer)
                mbar_arrive_cluster(tempty_peer + (uint32_t)(b * sizeof(uint64_t)));
              else
                mbar_arrive(&tempty[b]);
            }
          }
        }
        if (!ok || *((volatile int*)abortf)) break;
        tile_end<KIND, EPI>(p, acc, tix, tix * CG + (int)rank, it, e, lane, grp, r, sg, red);
        continue;
      }
      int kb0 = 0;
      for (int c = 0; c < nchunks; ++c, ++gc) {
        const int b = (int)(gc & 1);
        const int seg = kb0 / p.nkb;
        kb0 += chunk_len(kb0);
        bool w = mbar_wait<PAIR>(&tfull[b], (uint32_t)(gc >> 1) & 1u, abortf, p.wait_ns);
        w = __all_sync(0xffffffffu, w);
        if (!w) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (pf && c == nchunks - 2)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pf),
                       "r"((uint32_t)(TCOLS * sizeof(float)))
                       : "memory");
        float wgt = 1.0f;
        if constexpr (F16) wgt = (seg % nbase) == nbase - 1 ? 1.0f : 1.0f / kLoScale;
#pragma unroll
        for (int c0 = 0; c0 < TCOLS; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(trow + (uint32_t)b * ACC_COLS + (uint32_t)c0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[c0 + j] = fmaf(wgt, __uint_as_float(v[j]), acc[c0 + j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (PAIR && !issuer)
            mbar_arrive_cluster(tempty_peer + (uint32_t)(b * sizeof(uint64_t)));
          else
            mbar_arrive(&tempty[b]);
        }
      }
      if (!ok || *((volatile int*)abortf)) break;
      tile_end<KIND, EPI>(p, acc, tix, tix * CG + (int)rank, it, e, lane, grp, r, sg, red);
    }
  }

  // a CTA (pair) leaves only when every copy into its shared memory and every
  // tensor-core operation on its TMEM is done or drained above
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(TMEM_COLS)
                   : "memory");
    else
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
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
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

// The tensor maps of a launch are a function of its plane addresses, shapes and
// box sizes alone, and a solve uses a handful of such combinations (the two X
// buffers, the response buffers), so they are encoded once and reused: encoding
// the twelve maps of a launch anew cost tens of microseconds of host time per
// step, which bounds the step rate of small problems. A small table, replaced
// round robin, shared by every thread of the process.
struct MapKey {
  const void* planes[6];
  int64_t prows, qrows, np;
  int cg, f16;
};

bool cached_maps(const MapKey& k, KMaps* out) {
  constexpr int kSlots = 32;
  static std::mutex mu;
  static MapKey keys[kSlots];
  static KMaps maps[kSlots];
  static bool used[kSlots] = {};
  static int next = 0;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < kSlots; ++i)
    if (used[i] && memcmp(&keys[i], &k, sizeof k) == 0) {
      *out = maps[i];
      return true;
    }
  KMaps m;
  bool ok = true;
  for (int i = 0; i < 3; ++i) {
    ok = ok && make_map(&m.pa[i], k.planes[i], k.prows, k.np, BM, k.f16) &&
         make_map(&m.qb[i], k.planes[3 + i], k.qrows, k.np, BN / k.cg, k.f16);
    // EPI_SYMM's second half reads X as the left and Y as the right factor
    ok = ok && make_map(&m.qa[i], k.planes[3 + i], k.qrows, k.np, BM, k.f16) &&
         make_map(&m.pb[i], k.planes[i], k.prows, k.np, BN / k.cg, k.f16);
  }
  if (!ok) return false;
  keys[next] = k;
  maps[next] = m;
  used[next] = true;
  next = (next + 1) % kSlots;
  *out = m;
  return true;
}

// one launch of the (KIND, EPI, CG) kernel over `units` CTAs or CTA pairs (at most
// the resident ones), with its shared-memory attribute and its resident-pair
// count queried once
template <int KIND, int EPI, int CG, bool SPARSE = false>
cudaError_t launch_kind(const KMaps& maps, const KParams& p, int units, cudaStream_t s) {
  static int resident = 0;
  auto kern = k_gemm_tc<KIND, EPI, CG, SPARSE>;
  constexpr int smem = Ring<CG>::SMEM_BYTES;
  if (!resident) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (CG == 1) {
      resident = nsm;   // one CTA per SM: the ring leaves no room for a second
    } else {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = CG;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(CG * (nsm / CG)));
      cfg.blockDim = dim3(NUM_THREADS);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nc = 0;
      e = cudaOccupancyMaxActiveClusters(&nc, kern, &cfg);
      if (e != cudaSuccess) return e;
      if (nc < 1) return cudaErrorNotSupported;
      resident = nc;
    }
  }
  const int n = units < resident ? units : resident;
  if (CG == 1) {
    kern<<<n, NUM_THREADS, smem, s>>>(maps, p);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CG;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(CG * n));
  cfg.blockDim = dim3(NUM_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, maps, p);
}

template <int KIND, int CG>
cudaError_t launch_epi(int epi, const KMaps& maps, const KParams& p, int units, cudaStream_t s) {
  if (epi == EPI_SQUARE) return launch_kind<KIND, EPI_SQUARE, CG>(maps, p, units, s);
  if (epi == EPI_SYMM) return launch_kind<KIND, EPI_SYMM, CG>(maps, p, units, s);
  return launch_kind<KIND, EPI_PLAIN, CG>(maps, p, units, s);
}

// the block-sparse square: one launch over every resident pair, the tile count
// read on the device
cudaError_t launch_sparse(int kind, const KMaps& maps, const KParams& p, int units, cudaStream_t s) {
  if (kind == KIND_FP16X2) return launch_kind<KIND_FP16X2, EPI_SQUARE, 2, true>(maps, p, units, s);
  if (kind == KIND_BF16X3) return launch_kind<KIND_BF16X3, EPI_SQUARE, 2, true>(maps, p, units, s);
  return launch_kind<KIND_BF16X2, EPI_SQUARE, 2, true>(maps, p, units, s);
}

template <int CG>
cudaError_t launch_cg(int kind, int epi, const KMaps& maps, const KParams& p, int units,
                      cudaStream_t s) {
  if (kind == KIND_FP16X2) return launch_epi<KIND_FP16X2, CG>(epi, maps, p, units, s);
  if (kind == KIND_BF16X3) return launch_epi<KIND_BF16X3, CG>(epi, maps, p, units, s);
  return launch_epi<KIND_BF16X2, CG>(epi, maps, p, units, s);
}

}  // namespace

void tc_tile_shape(int pair, int* bm, int* bn) {
  *bm = pair ? 2 * BM : BM;
  *bn = BN;
}

cudaError_t launch_gemm_tc(const TcLaunch& L, cudaStream_t s, char* errbuf, size_t errlen) {
  if (L.ntiles <= 0) return cudaSuccess;
  const int mode = L.mode;
  const int kind = mode == SP2_MODE_FP16X2 ? KIND_FP16X2
                                           : (mode == SP2_MODE_BF16X3 ? KIND_BF16X3 : KIND_BF16X2);
  const bool f16 = kind == KIND_FP16X2, x3 = kind == KIND_BF16X3;
  const int cg = L.tune.pair ? 2 : 1;   // the tile list was built for this tile shape
  const TcOperand& P = L.P;
  const TcOperand& Q = L.Q;
  // the middle planes exist only in BF16X3; elsewhere the hi maps stand in (never read)
  const uint16_t* p_mid = x3 ? P.mid : P.hi;
  const uint16_t* q_mid = x3 ? Q.mid : Q.hi;
  const bool sym_out = L.epi != EPI_PLAIN;
  if (x3 && (!p_mid || !q_mid || (sym_out && !L.out.mid))) {
    snprintf(errbuf, errlen, "tcgen05 product: BF16X3 operand without its middle plane");
    return cudaErrorInvalidValue;
  }
  if (sym_out && !L.prev) {
    snprintf(errbuf, errlen, "tcgen05 product: symmetric epilogue without the previous iterate");
    return cudaErrorInvalidValue;
  }
  // TMA box/stride rules: 16-byte aligned bases, np*2-byte row pitch (np % 256 == 0),
  // every x coordinate a multiple of 64 elements; tiles never leave their operand.
  const int64_t np = L.np;
  if ((reinterpret_cast<uintptr_t>(P.hi) | reinterpret_cast<uintptr_t>(P.lo) |
       reinterpret_cast<uintptr_t>(Q.hi) | reinterpret_cast<uintptr_t>(Q.lo) |
       reinterpret_cast<uintptr_t>(p_mid) | reinterpret_cast<uintptr_t>(q_mid)) & 15u ||
      np % 256 != 0 || P.rows % np != 0 || Q.rows % np != 0 || P.rows % (BM * cg) != 0 ||
      Q.rows % BN != 0 || (L.epi == EPI_SYMM && Q.rows != np) ||
      (L.epi == EPI_SQUARE && P.rows != np) || P.rows > (int64_t)1 << 30) {
    snprintf(errbuf, errlen, "tcgen05 product: operand alignment/shape violates the TMA rules");
    return cudaErrorInvalidValue;
  }
  KMaps maps;
  MapKey key;
  memset(&key, 0, sizeof key);   // padding bytes too: the key is compared bytewise
  key.planes[0] = P.hi;
  key.planes[1] = P.lo;
  key.planes[2] = p_mid;
  key.planes[3] = Q.hi;
  key.planes[4] = Q.lo;
  key.planes[5] = q_mid;
  key.prows = P.rows;
  key.qrows = Q.rows;
  key.np = np;
  key.cg = cg;
  key.f16 = f16 ? 1 : 0;
  if (!cached_maps(key, &maps)) {
    snprintf(errbuf, errlen, "cuTensorMapEncodeTiled failed (driver entry point unavailable?)");
    return cudaErrorInvalidValue;
  }
  KParams p;
  p.nkb = (int)(np / BK);
  // K chunk drained from TMEM into FP32 registers: 4 k-blocks (256 products per
  // accumulator pass). np is a multiple of 256, so 4 divides every segment and
  // the lo-plane weight changes only at a chunk boundary. The tensor core's
  // FP32 accumulation truncates, and its bias grows with the chunk length: at
  // N=4096 (FP16X2) 256-wide chunks give a 1.0e-5 density error against the
  // exact form, 512-wide 2.5e-5 and 2048-wide 7.6e-4, for 3% more time per
  // product than 512-wide chunks.
  p.ch = 4;
  // The cross terms (hi*lo, lo*hi; in BF16X3 everything after hi*hi) are small
  // once weighted, so the truncation bias of a longer TMEM accumulation shrinks
  // with them: a chunk's bias scales with its length times the size of its
  // terms. Every chunk boundary costs the MMA issuer a commit and a wait, so the
  // cross terms take the longest chunk whose bias stays a few percent of the
  // hi*hi chunks' (256 x 1): FP16X2 (weight 2^-11) up to 16384 wide (256
  // k-blocks, 16384 x 2^-11 = 8), the bfloat16 modes (2^-8) up to 2048 (32
  // k-blocks, also 8); the largest power of two up to that which divides np / BK.
  p.ch_lo = f16 ? 256 : 32;
  while ((np / BK) % p.ch_lo != 0) p.ch_lo >>= 1;
  p.nbase = x3 ? 6 : 3;
  p.nseg = L.epi == EPI_SYMM ? 2 * p.nbase : p.nbase;
  p.np = np;
  p.out = static_cast<float*>(L.out.master);
  p.out_hi = L.out.hi;
  p.out_lo = L.out.lo;
  p.out_mid = L.out.mid;
  p.prev = L.prev;
  p.part = L.part;
  p.tiles = L.tiles;
  p.ntiles = L.ntiles;
  p.st = L.st;
  p.step = L.step;
  p.p_scale = f16 ? L.p_scale : nullptr;
  p.q_scale = f16 ? L.q_scale : nullptr;
  p.o_scale = f16 ? L.o_scale : nullptr;
  p.zmax = f16 ? L.zmax : nullptr;
  p.wait_ns = L.tune.wait_ns;
  p.withhold = L.tune.withhold;
  p.tail = L.tail;
  // persistent: one CTA per SM (the shared-memory ring allows no second one)
  p.dyn_ntiles = L.dyn_ntiles;
  p.kcnt = L.kcnt;
  p.klist = L.klist;
  p.nbk = L.nbk;
  if (L.dyn_ntiles) {
    if (cg != 2 || L.epi != EPI_SQUARE || L.tail || !L.kcnt || !L.klist || L.nbk * 256 != np) {
      snprintf(errbuf, errlen, "tcgen05 product: block-sparse launches are squares on CTA pairs");
      return cudaErrorInvalidValue;
    }
    return launch_sparse(kind, maps, p, L.ntiles, s);
  }
  // persistent: one CTA (pair) per SM (pair of SMs), the launch's tiles spread over them
  if (cg == 2) return launch_cg<2>(kind, L.epi, maps, p, L.ntiles, s);
  return launch_cg<1>(kind, L.epi, maps, p, L.ntiles, s);
}

}  // namespace sp2
