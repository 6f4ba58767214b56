// Internal declarations shared by the translation units of libsp2.so.
// Not part of the public ABI (that is include/sp2.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sp2.h"

namespace sp2 {

// Internal matrices are padded to a multiple of the largest tile edge of their
// arithmetic mode, zero outside the caller's N x N block: 256 for the split
// modes (the tensor-core tiles and the TMA row pitch), 128 for FP32 (its
// CUDA-core tiles), 64 for FP64 (its tiles; GB300's FP64 rate makes every padded
// row count). Zero padding is invariant under all recursions (X -> X^2,
// 2X - X^2, Y -> YX + XY), so it never touches results.
constexpr int kPad = 256;

inline int64_t pad_n(int64_t n, int mode) {
  const int64_t q = mode == SP2_MODE_FP64 ? 64 : (mode == SP2_MODE_FP32 ? 128 : kPad);
  return (n + q - 1) / q * q;
}

// Device-resident SP2 control state: traces of every X_n, the branch signs
// and the stop decision. Written only by k_decide; read by the step kernels
// (which become no-ops once the recursion has stopped) and by the host.
struct DevState {
  double t1[SP2_MAX_ITER + 2];   // Tr[X_n], index n = 1..M+1
  double t2[SP2_MAX_ITER + 2];   // ||X_n||_F^2
  double f[SP2_MAX_ITER + 2];    // ||X_n - X_n^2||_F^2, known after step n
  int sigma[SP2_MAX_ITER + 2];   // sigma_n, the branch taken by step n (X_n -> X_{n+1})
  int plane1[SP2_MAX_ITER + 2];  // split-tail mode: 1 if step n uses the hi planes alone
  double fill[SP2_MAX_ITER + 2]; // block-sparse: share of the upper blocks step n formed
  int stop_at;                   // M once a stop rule fired, else 0
  int nonfinite;                 // a trace was NaN/Inf
  int abort_flag;                // a device wait timed out (kernel bailed out)
  int pad_;
  double bounds[2];              // Gershgorin eps_min, eps_max
  double fbest;                  // smallest f among the floor candidates (f <= floor_gate)
  int nbest;                     // its iterate index n (X_n), 0 if none yet
  int keep_step;                 // step whose input X_n (and Y_n) is to be kept now
  int backtracked;               // the floor stop returned X_nbest, not the last iterate
  int stop_step;                 // the step after which the stop test fired
  double alpha, beta;            // X_1 = alpha I + beta H, from the (widened) bounds
  double work_kblocks;           // block-sparse: 256-wide K blocks the squares ran, all tiles
};
// The host reads the trailing part of DevState (from stop_at on) after every step.
inline size_t devstate_tail_offset() { return offsetof(DevState, stop_at); }

// Storage of one padded matrix (or a batch of them) in a given mode.
struct MatBuf {
  void* master = nullptr;        // double (FP64 mode) or float, rows x np, unscaled
  uint16_t* hi = nullptr;        // split modes: hi plane (bf16 or fp16 bits)
  uint16_t* lo = nullptr;        // split modes: lo plane
  uint16_t* mid = nullptr;       // BF16X3: the middle plane
};

inline bool split_mode(int mode) {
  return mode == SP2_MODE_BF16X2 || mode == SP2_MODE_FP16X2 || mode == SP2_MODE_BF16X3;
}
inline int n_planes(int mode) { return mode == SP2_MODE_BF16X3 ? 3 : (split_mode(mode) ? 2 : 0); }

// Eq. doubleHalf with bfloat16: hi = bf16(v), lo = bf16(v - hi).
__device__ __forceinline__ void split_bf16(float v, uint16_t& h, uint16_t& l) {
  const __nv_bfloat16 hb = __float2bfloat16_rn(v);
  const __nv_bfloat16 lb = __float2bfloat16_rn(v - __bfloat162float(hb));
  h = __bfloat16_as_ushort(hb);
  l = __bfloat16_as_ushort(lb);
}

// Three bfloat16 planes of v: hi = bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid).
// Both residuals are exact in FP32, so hi + mid + lo = v for normal v.
__device__ __forceinline__ void split_bf16x3(float v, uint16_t& h, uint16_t& m, uint16_t& l) {
  const __nv_bfloat16 hb = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(hb);
  const __nv_bfloat16 mb = __float2bfloat16_rn(r1);
  const __nv_bfloat16 lb = __float2bfloat16_rn(r1 - __bfloat162float(mb));
  h = __bfloat16_as_ushort(hb);
  m = __bfloat16_as_ushort(mb);
  l = __bfloat16_as_ushort(lb);
}

// The fp16 lo plane holds the residual times 2^11 (one fp16 significand), so
// it stays out of the subnormal range; products with it are scaled back by
// 2^-11 from a separate accumulator.
constexpr float kLoScale = 2048.0f;

// Eq. doubleHalf with fp16 on s * v (s a power of two chosen per matrix so
// that |s v| <= 2^14 < 65504): hi = fp16(s v), lo = fp16((s v - hi) * 2^11).
__device__ __forceinline__ void split_fp16(float v, float s, uint16_t& h, uint16_t& l) {
  const float vs = v * s;
  const __half hh = __float2half_rn(vs);
  const __half ll = __float2half_rn((vs - __half2float(hh)) * kLoScale);
  h = __half_as_ushort(hh);
  l = __half_as_ushort(ll);
}

// Power-of-two plane scale for a matrix whose entries are bounded by `bound`:
// 2^(14 - e) with bound <= 2^e, so every scaled entry is at most 2^14.
__device__ __forceinline__ float pow2_scale(float bound) {
  if (!(bound > 0.0f) || !isfinite(bound)) return 1.0f;
  int e;
  frexpf(bound, &e);
  int k = 14 - e;
  k = k < -120 ? -120 : (k > 120 ? 120 : k);
  return ldexpf(1.0f, k);
}

// Per-matrix scale state of a batch of B response matrices (FP16X2 only).
struct ScaleBuf {
  float* ymax = nullptr;    // [2][B] max |Y| of the matrix in each ping-pong slot
  float* yscale = nullptr;  // [2][B] power-of-two scale of each slot's fp16 planes
  float* zmax = nullptr;    // [B]    max |Z| of the current step's product Z = Y X
  int64_t B = 0;
};

enum Epi : int {
  EPI_SQUARE = 0,   // out = sigma>0 ? C : 2 X - C, symmetric (upper tiles, mirrored), traces
  EPI_PLAIN = 1,    // out = C (fp32/fp64 Z), all tiles
  EPI_SYMM = 2,     // out = sigma>0 ? YX+XY : 2Y - (YX+XY), symmetric batch (upper tiles, mirrored)
};

// Per-block partial sums written by the kernels that produce an X_{n+1}:
// t1 = Tr[X_{n+1}], t2 = ||X_{n+1}||_F^2, f = ||X_n - X_n^2||_F^2.
struct Part3 {
  double t1, t2, f;
};

struct Tile {       // one output tile of a product kernel
  int row0;         // first output row (within the stacked A operand)
  int col0;         // first output column
};

// ---------------------------------------------------------------- launchers
// elementwise / reduction kernels (kernels_elem.cu)
// Gershgorin bounds of H into st->bounds (widened for a point spectrum) and the
// coefficients st->alpha, st->beta of X_1 = alpha I + beta H; NaN/Inf bounds set
// st->nonfinite and stop the recursion before its first step (stop_at = -1).
cudaError_t launch_bounds(const void* H, int64_t n, int dtype, double2* part, int nparts,
                          DevState* st, cudaStream_t s);
int bounds_nparts(int64_t n);
// the same from given bounds
cudaError_t launch_set_bounds(DevState* st, double eps_min, double eps_max, cudaStream_t s);
// preset branch signs sigma_1..sigma_m (m <= SP2_MAX_ITER), passed by value
cudaError_t launch_set_sigma(DevState* st, const int8_t* sigma, int m, cudaStream_t s);

// X_1 = alpha I + beta H (or Y_1 = beta B for a batch), caller layout -> padded mode layout.
// diag_only: B given as diagonals (batch x n). symmetrize: use (B + B^T)/2.
// part (nullable): trace partials, one per block.
// FP16X2: planes are written with scale 1 when ymax is null (X), otherwise only
// the master is written and max|entry| per batch entry is accumulated into
// ymax (planes follow from launch_split_scaled).
// coef: INIT_ARGS uses (alpha, beta); INIT_STATE takes alpha, beta from st;
// INIT_STATE_BETA takes (0, st->beta).
enum InitCoef : int { INIT_ARGS = 0, INIT_STATE = 1, INIT_STATE_BETA = 2 };
cudaError_t launch_init(const void* src, int64_t n, int64_t np, int64_t batch, int dtype,
                        int diag_only, int symmetrize, double alpha, double beta, int mode,
                        MatBuf dst, Part3* part, int nparts, float* ymax, cudaStream_t s,
                        int coef = INIT_ARGS, const DevState* st = nullptr);
int init_nparts(int64_t np);

// reduce trace partials of X_n, decide stop/sigma (see DevState)
struct DecideParams {
  int n;             // index of the X just produced (X_n)
  int nparts;
  double nocc, idem_tol, floor_gate;
  int min_iter, max_iter;
  int fixed_m;       // > 0: sigma preset, stop when n - 1 == fixed_m
  double tail_f;     // > 0: single-plane products while f of the last iterate exceeds it
  int ratio_floor = 0;  // block-sparse recursion: the threshold-floor test as well
};
constexpr double kRatioGate = 1e-4;   // f from which a pair of opposite steps must cut f 600-fold
cudaError_t launch_decide(const Part3* part, DevState* st, DecideParams p, cudaStream_t s);
// copy `count` entries of the master src -> dst when st->keep_step == step (the
// floor candidate with the smallest f so far), else nothing
cudaError_t launch_keep_best(const void* src, void* dst, int64_t count, int mode, const DevState* st,
                             int step, cudaStream_t s);

// Y_{n+1} = sigma>0 ? Z + Z^T : 2 Y - (Z + Z^T) for a batch; step n reads sigma_n.
// FP16X2: the planes of Y_{n+1} use the scale bounded by 2 max|Z| (+ 2 max|Y_n|
// when sigma<0) from sc (slots slot_in -> slot_out); max|Y_{n+1}| is recorded.
cudaError_t launch_symm_update(const void* Z, MatBuf y_in, MatBuf y_out, int64_t np, int64_t batch,
                               int mode, const DevState* st, int step, ScaleBuf sc, int slot_in,
                               int slot_out, cudaStream_t s);

// padded mode layout -> caller layout (N x N per batch entry), times `scale`
// (times st->beta as well when beta_state is given)
cudaError_t launch_copy_out(MatBuf src, int64_t n, int64_t np, int64_t batch, int mode,
                            double scale, void* dst, int dtype, cudaStream_t s,
                            const DevState* beta_state = nullptr);
// reset of the fields an adjoint recursion does not use (stop, keep, abort, nonfinite)
cudaError_t launch_adjoint_state(DevState* st, cudaStream_t s);

// regenerate hi/lo planes from the FP32 master, rows x np (plane scale 1)
cudaError_t launch_split(MatBuf m, int64_t rows, int64_t np, int mode, cudaStream_t s);
// FP16X2 batch of B matrices: scale of slot `slot` from its ymax, then planes
cudaError_t launch_split_scaled(MatBuf m, int64_t np, ScaleBuf sc, int slot, cudaStream_t s);

// response_contract
cudaError_t launch_contract(const void* P, int64_t L, const void* Q, int64_t K, int64_t n,
                            int dtype, int q_diag, double* part, int nparts, double* out,
                            cudaStream_t s);
int contract_nparts(int64_t n, int q_diag);

// product kernels
// The step decision taken by the last block of a CUDA-core square (one launch
// fewer per step): its parameters, the state it writes, and a completion counter
// that is zero between launches (the last block resets it).
struct SimtDecide {
  DecideParams p;
  DevState* st = nullptr;
  unsigned* done = nullptr;
};
// SIMT (FP64 / FP32): C = A * X with A rows x np (stacked), X np x np symmetric.
// dec (squares only, may be null): take the step decision in the last block.
cudaError_t launch_gemm_simt(int mode, int epi, const void* A, int64_t a_rows, const void* X,
                             int64_t np, void* out, const void* x_prev, Part3* part,
                             const Tile* tiles, int ntiles, const DevState* st, int step,
                             cudaStream_t s, const SimtDecide* dec = nullptr);
void simt_tile_shape(int mode, int64_t np, int* bm, int* bn);

// tcgen05 split-precision (BF16X2 / FP16X2 / BF16X3)
struct TcOperand {   // hi/lo (and BF16X3 mid) planes of a stacked operand, rows x np
  const uint16_t* hi = nullptr;
  const uint16_t* lo = nullptr;
  int64_t rows = 0;
  const uint16_t* mid = nullptr;
};
// Launch settings of the product kernel that are not part of the arithmetic.
struct TcTuning {
  unsigned long long wait_ns = 2000000000ull;  // limit of every mbarrier wait
  int withhold = 0;    // test hook: the first TMA load of CTA 0 is never issued
  int fused_response = 0;  // response step as one EPI_SYMM launch (else EPI_PLAIN + transpose-add)
  int pair = 1;        // 256 x 256 tiles on CTA pairs (tcgen05 cta_group::2), else 128 x 256
};
// (TcLaunch.tail: the split-tail mode; the kernel reads st->plane1[step] and uses
// the hi planes alone, one product per segment pair, where it is set.)
// One product launch: C = P Q (EPI_SQUARE: P = Q = X; EPI_PLAIN: P = stacked A,
// Q = symmetric B; EPI_SYMM: P = stacked symmetric Y, Q = X, C = Y X + X Y).
struct TcLaunch {
  int mode = 0;
  int epi = 0;
  TcOperand P, Q;
  int64_t np = 0;
  MatBuf out;                      // master + planes (planes only for the symmetric epilogues)
  const float* prev = nullptr;     // EPI_SQUARE: X_n master; EPI_SYMM: Y_n master
  Part3* part = nullptr;           // per-tile partials (>= ntiles)
  const Tile* tiles = nullptr;
  int ntiles = 0;
  DevState* st = nullptr;
  int step = 0;
  const float* p_scale = nullptr;  // FP16X2: per batch entry of P, the plane scale to divide out
  const float* q_scale = nullptr;  // FP16X2: the plane scale of Q (nullable)
  const float* o_scale = nullptr;  // FP16X2 EPI_SYMM: per batch entry, scale of the output planes
  float* zmax = nullptr;           // FP16X2 EPI_PLAIN: per batch entry, receives max |C|
  int tail = 0;                    // split-tail mode (st->plane1 decides per step)
  TcTuning tune;
  // block-sparse square (CTA pairs): tiles, their count and their K-block lists
  // are written on the device by the plan kernel; ntiles is then the upper bound
  const int* dyn_ntiles = nullptr;
  const int* kcnt = nullptr;
  const uint16_t* klist = nullptr;
  int nbk = 0;                     // K blocks of 256 (np / 256): the stride of klist
};
cudaError_t launch_gemm_tc(const TcLaunch& L, cudaStream_t s, char* errbuf, size_t errlen);

// ---- block-sparse recursion (sparse_kernels.cu): 256 x 256 blocks, N <= 65536
constexpr int kMaxSparseBlocks = 256;
struct SparseBufs {
  int nb = 0;                      // blocks per dimension (np / 256)
  double tau2 = 0.0;               // a block stays when its norm^2 > tau2 (or it is diagonal)
  uint8_t* mask[2] = {};           // content mask of X[0], X[1] (nb x nb, symmetric)
  Tile* tiles[2] = {};             // tile lists, by step parity (step n squares tiles[n % 2])
  int* ntiles[2] = {};
  int* kcnt[2] = {};
  uint16_t* klist[2] = {};         // nb K blocks per tile
  uint32_t* zero = nullptr;        // blocks to zero: (I << 16) | J, I <= J
  int* nzero = nullptr;
  double* nrm2 = nullptr;          // nb x nb scratch: block norms^2
  Part3* psum = nullptr;           // the decision's one partial: traces of X~, and f
};
// ||block||_F^2 of the upper blocks of a master into nrm2
cudaError_t launch_block_norms(const float* master, int64_t np, int nb, double* nrm2,
                               cudaStream_t s);
// threshold the iterate just formed (init: X_1 from nrm2 and the init partials;
// else the square of `step`, from its two partials per tile), list the blocks to
// zero in buffer xo, reduce the decision's partial, and write the next square's
// tiles and K lists into tiles[tl_out]. No-op after the stop (but for init).
cudaError_t launch_sparse_plan(const SparseBufs& B, int init, int xo, int tl_in, int tl_out,
                               const Part3* part, int nparts_init, DevState* st, int step,
                               cudaStream_t s);
// zero the listed blocks (and mirrors) of x's master and planes
cudaError_t launch_zero_blocks(const SparseBufs& B, MatBuf x, int64_t np, int mode,
                               const DevState* st, int step, int init, cudaStream_t s);
void tc_tile_shape(int pair, int* bm, int* bn);   // output tile of one CTA (pair)

// FP16X2 scale of the next symmetric response step: per batch entry, the sum of
// the EPI_SYMM tile partials (||Y_{n+1}||_F^2) and the plane scale of Y_{n+2},
// pow2_scale(2 ||Y_{n+1}||_F) (|Y_{n+2}|_max <= ||Y_{n+2}||_2 <= 2 ||Y_{n+1}||_2).
// No-op when the recursion stopped before `step`.
cudaError_t launch_sym_scale(const Part3* part, int ppt, const Tile* tiles, int ntiles, int64_t np,
                             int64_t batch, const DevState* st, int step, float* scale_out,
                             cudaStream_t s);
// FP16X2: the same bound from a batch's masters (the first response step)
cudaError_t launch_fro_scale(const float* master, int64_t np, int64_t batch, double* part,
                             int nparts, float* scale_out, cudaStream_t s);
int fro_nparts();

// finite temperature (fermi_kernels.cu)
// out = z1 (Z1 + Z1^T) + z2 (Z2 + Z2^T) + a A + id I on the padded np x np
// matrices (null operands skipped, I only on the caller's n x n block);
// amax (nullable) receives max |out| (must start at 0).
cudaError_t launch_combine(int mode, void* out, int64_t np, int64_t n, const void* Z1, double z1,
                           const void* Z2, double z2, const void* A, double a, double id,
                           float* amax, cudaStream_t s);
// out[0] = Tr of the caller's n x n block, FP64
cudaError_t launch_trace(int mode, const void* M, int64_t np, int64_t n, double* out,
                         cudaStream_t s);

// self-consistent response and MLP (scf_kernels.cu)
cudaError_t launch_sgemm(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                         int ta, const float* B, int64_t ldb, int tb, float beta, float* C,
                         int64_t ldc, int relu, int bf16, cudaStream_t s);
cudaError_t launch_site_potential(const double* V, const double* K, const double* q, int64_t F,
                                  int64_t ns, double* u, cudaStream_t s);
cudaError_t launch_expand_sites(const double* u, int64_t F, int64_t ns, int norb, void* out,
                                int dtype, cudaStream_t s);
cudaError_t launch_site_charges(const void* Y, int mode, int64_t F, int64_t ns, int norb,
                                int64_t np, double* q, cudaStream_t s);
cudaError_t launch_residual(const double* qout, const double* q, int64_t total, double* r,
                            double* out2, cudaStream_t s);
cudaError_t launch_axpy_d(double* y, double a, const double* x, int64_t total, cudaStream_t s);
cudaError_t launch_gram(const double* R, int m, int64_t F, int64_t ns, int64_t stride, double* G,
                        cudaStream_t s);
cudaError_t launch_anderson_combine(const double* Qh, const double* Rh, const double* c, int m,
                                    int64_t F, int64_t ns, int64_t stride, double alpha, double* q,
                                    cudaStream_t s);
cudaError_t launch_normalise_rows(const double* r, int64_t F, int64_t ns, float* x, double* nr,
                                  cudaStream_t s);
cudaError_t launch_apply_update(double* q, const float* y, const double* nr, int64_t F, int64_t ns,
                                cudaStream_t s);
cudaError_t launch_mse_grad(const float* Y, const float* T, int64_t total, float scale, float* dY,
                            double* loss, cudaStream_t s);
cudaError_t launch_relu_mask(float* dH, const float* Hr, int64_t total, cudaStream_t s);
cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int64_t total, float lr,
                        float b1, float b2, float eps, int t, cudaStream_t s);

}  // namespace sp2
