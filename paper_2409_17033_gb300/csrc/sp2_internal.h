// Internal declarations shared by the translation units of libsp2.so.
// Not part of the public ABI (that is include/sp2.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/sp2.h"

namespace sp2 {

// Internal matrices are padded to a multiple of this (the largest tile edge),
// zero outside the caller's N x N block. Zero padding is invariant under all
// recursions (X -> X^2, 2X - X^2, Y -> YX + XY), so it never touches results.
constexpr int kPad = 256;

inline int64_t pad_n(int64_t n) { return (n + kPad - 1) / kPad * kPad; }

// Device-resident SP2 control state: traces of every X_n, the branch signs
// and the stop decision. Written only by k_decide; read by the step kernels
// (which become no-ops once the recursion has stopped) and by the host.
struct DevState {
  double t1[SP2_MAX_ITER + 2];   // Tr[X_n], index n = 1..M+1
  double t2[SP2_MAX_ITER + 2];   // ||X_n||_F^2
  int sigma[SP2_MAX_ITER + 2];   // sigma_n, the branch taken by step n (X_n -> X_{n+1})
  int stop_at;                   // M once a stop rule fired, else 0
  int nonfinite;                 // a trace was NaN/Inf
  int abort_flag;                // a device wait timed out (kernel bailed out)
  int pad_;
  double bounds[2];              // Gershgorin eps_min, eps_max
};

// Storage of one padded matrix (or a batch of them) in a given mode.
struct MatBuf {
  void* master = nullptr;        // double (FP64 mode) or float, rows x np
  __nv_bfloat16* hi = nullptr;   // BF16X2 only: hi plane
  __nv_bfloat16* lo = nullptr;   // BF16X2 only: lo plane
};

enum Epi : int {
  EPI_SQUARE = 0,   // out = sigma>0 ? C : 2 X - C, symmetric (upper tiles, mirrored), traces
  EPI_PLAIN = 1,    // out = C (fp32/fp64 Z), all tiles
};

struct Tile {       // one output tile of a product kernel
  int row0;         // first output row (within the stacked A operand)
  int col0;         // first output column
};

// ---------------------------------------------------------------- launchers
// elementwise / reduction kernels (kernels_elem.cu)
cudaError_t launch_bounds(const void* H, int64_t n, int dtype, double2* part, int nparts,
                          DevState* st, cudaStream_t s);
int bounds_nparts(int64_t n);

// X_1 = alpha I + beta H (or Y_1 = beta B for a batch), caller layout -> padded mode layout.
// diag_only: B given as diagonals (batch x n). symmetrize: use (B + B^T)/2.
// part (nullable): trace partials, one per block.
cudaError_t launch_init(const void* src, int64_t n, int64_t np, int64_t batch, int dtype,
                        int diag_only, int symmetrize, double alpha, double beta, int mode,
                        MatBuf dst, double2* part, int nparts, cudaStream_t s);
int init_nparts(int64_t np);

// reduce trace partials of X_n, decide stop/sigma (see DevState)
struct DecideParams {
  int n;             // index of the X just produced (X_n)
  int nparts;
  double nocc, idem_tol, floor_gate;
  int min_iter, max_iter;
  int fixed_m;       // > 0: sigma preset, stop when n - 1 == fixed_m
};
cudaError_t launch_decide(const double2* part, DevState* st, DecideParams p, cudaStream_t s);

// Y_{n+1} = sigma>0 ? Z + Z^T : 2 Y - (Z + Z^T) for a batch; step n reads sigma_n.
cudaError_t launch_symm_update(const void* Z, MatBuf y_in, MatBuf y_out, int64_t np, int64_t batch,
                               int mode, const DevState* st, int step, cudaStream_t s);

// padded mode layout -> caller layout (N x N per batch entry), times `scale`
cudaError_t launch_copy_out(MatBuf src, int64_t n, int64_t np, int64_t batch, int mode,
                            double scale, void* dst, int dtype, cudaStream_t s);

// regenerate hi/lo planes from the FP32 master (BF16X2), rows x np
cudaError_t launch_split(MatBuf m, int64_t rows, int64_t np, cudaStream_t s);

// response_contract
cudaError_t launch_contract(const void* P, int64_t L, const void* Q, int64_t K, int64_t n,
                            int dtype, int q_diag, double* part, int nparts, double* out,
                            cudaStream_t s);
int contract_nparts(int64_t n, int q_diag);

// product kernels
// SIMT (FP64 / FP32): C = A * X with A rows x np (stacked), X np x np symmetric.
cudaError_t launch_gemm_simt(int mode, int epi, const void* A, int64_t a_rows, const void* X,
                             int64_t np, void* out, const void* x_prev, double2* part,
                             const Tile* tiles, int ntiles, const DevState* st, int step,
                             cudaStream_t s);
void simt_tile_shape(int mode, int* bm, int* bn);

// tcgen05 split-precision (BF16X2)
struct TcOperand {   // hi/lo planes of a stacked operand, rows x np
  const __nv_bfloat16* hi;
  const __nv_bfloat16* lo;
  int64_t rows;
};
cudaError_t launch_gemm_tc(int epi, TcOperand A, TcOperand B, int64_t np, MatBuf out,
                           const float* x_prev, double2* part, const Tile* tiles, int ntiles,
                           DevState* st, int step, cudaStream_t s, char* errbuf, size_t errlen);
void tc_tile_shape(int* bm, int* bn);

}  // namespace sp2
