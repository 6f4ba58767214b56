// The SP2 branch and stop decision of one step (Eq. DM0 with the readings of
// the stop rule in sp2.h): one block of threads reduces the step's trace
// partials in a fixed order and one thread updates the device state. Shared by
// the decision kernel and by the CUDA-core square, whose last block takes it.
#pragma once
#include "sp2_internal.h"

namespace sp2 {
namespace {

constexpr int kStall = 4;  // steps without a new minimum of f that mark the precision floor

__device__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;  // valid in thread 0
}

// Reads the partials with cache-global loads: in the CUDA-core square they come
// from the other blocks of the same launch.
__device__ __noinline__ void decide_block(const Part3* part, DevState* st, const DecideParams& p) {
  double t1 = 0.0, t2 = 0.0, f = 0.0;
  for (int i = threadIdx.x; i < p.nparts; i += blockDim.x) {
    t1 += __ldcg(&part[i].t1);
    t2 += __ldcg(&part[i].t2);
    f += __ldcg(&part[i].f);
  }
  t1 = block_sum(t1);
  __syncthreads();
  t2 = block_sum(t2);
  __syncthreads();
  f = block_sum(f);
  if (threadIdx.x != 0) return;
  if (st->stop_at != 0) return;  // already stopped: later steps are no-ops
  const int n = p.n;
  st->t1[n] = t1;
  st->t2[n] = t2;
  if (n >= 2) st->f[n - 1] = f;  // the step that produced X_n measured X_{n-1}
  // split-tail mode: step n (X_n -> X_{n+1}) uses single-plane products while the
  // idempotency error of the last measured iterate exceeds tail_f; once a step
  // has used split products, every later one does
  if (p.tail_f > 0.0)
    st->plane1[n] = n == 1 ? 1 : (st->plane1[n - 1] && st->f[n - 1] > p.tail_f ? 1 : 0);
  if (!isfinite(t1) || !isfinite(t2)) {
    st->nonfinite = 1;
    st->stop_at = (n - 1 >= 1) ? n - 1 : -1;
    return;
  }
  const int s = n - 1;  // the step that produced X_n (0 for X_1)
  // floor candidates: X_s (f known now) with f <= gate and the smallest f so far
  if (p.fixed_m == 0 && p.floor_gate > 0.0 && s >= 2 && st->f[s] <= p.floor_gate &&
      (st->nbest == 0 || st->f[s] < st->fbest)) {
    st->fbest = st->f[s];
    st->nbest = s;
    st->keep_step = s;
  }
  if (p.fixed_m > 0) {
    if (s == p.fixed_m) st->stop_at = s;
    return;  // branches preset by the host
  }
  if (s >= 1 && s >= p.min_iter) {
    const double e = fabs(t1 - t2);
    bool stop = false, floor_stop = false;
    if (p.idem_tol > 0.0 && e <= p.idem_tol) stop = true;
    // precision floor on f (see the stop rule in sp2.h):
    //   opposite branches at steps s-2, s-1, f_{s-2} <= gate and f_s >= f_{s-2}; or
    //   min f_1..f_{s-STALL} <= gate and none of f_{s-STALL+1..s} below it
    if (!stop && p.floor_gate > 0.0) {
      if (s >= 3 && st->sigma[s - 2] != st->sigma[s - 1] && st->f[s - 2] <= p.floor_gate &&
          st->f[s] >= st->f[s - 2])
        floor_stop = true;
      // block-sparse recursion: from f <= 1e-4 a pair of opposite steps cuts f at
      // least 600-fold in exact arithmetic; less than twofold is the threshold's floor
      if (!floor_stop && p.ratio_floor && s >= 3 && st->sigma[s - 2] != st->sigma[s - 1] &&
          st->f[s - 2] <= kRatioGate && st->f[s] >= 0.5 * st->f[s - 2])
        floor_stop = true;
      if (!floor_stop && s > kStall) {
        double best = st->f[1];
        for (int k = 2; k <= s - kStall; ++k) best = fmin(best, st->f[k]);
        double recent = st->f[s - kStall + 1];
        for (int k = s - kStall + 2; k <= s; ++k) recent = fmin(recent, st->f[k]);
        if (best <= p.floor_gate && recent >= best) floor_stop = true;
      }
      if (floor_stop) stop = true;
    }
    if (stop) {
      st->stop_step = s;
      // at the floor the result is the kept candidate X_nbest (M = nbest - 1 steps)
      if (floor_stop && st->nbest >= 2 && st->nbest - 1 < s) {
        st->stop_at = st->nbest - 1;
        st->backtracked = 1;
      } else {
        st->stop_at = s;
      }
      return;
    }
  }
  // Eq. DM0 branch: the trace after X^2 is t2, after 2X - X^2 it is 2 t1 - t2.
  st->sigma[n] = (fabs(t2 - p.nocc) <= fabs(2.0 * t1 - t2 - p.nocc)) ? 1 : -1;
}

}  // namespace
}  // namespace sp2
