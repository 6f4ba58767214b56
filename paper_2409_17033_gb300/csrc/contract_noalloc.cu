// response_contract_noalloc: the response contraction for callers that cannot
// allocate device memory. Its reduction partials live in a fixed file-scope
// device array instead of handle-owned workspace, and nothing is allocated or
// freed on any call.
#include <mutex>

#include "sp2_internal.h"

namespace {

// Capacity of the shared partial-sum array, in doubles (1 MiB). Every GPU that
// loads the library holds this array until the process exits.
constexpr int64_t kScratchDoubles = (int64_t)1 << 17;
// Largest L * K accepted (one grid row per pair; at least two partials each).
constexpr int64_t kMaxPairs = 65535;

static __device__ __align__(256) double g_contract_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_contract_scratch on the current device. The host-side
// name of the array is only a stand-in for it, so the address is looked up
// once per device (with that device current) and cached.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_contract_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Device (or managed) memory of the current device: memory of another GPU may
// not be reachable from this one, and a kernel touching it would fault.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int response_contract_noalloc(const void* P, int64_t L, const void* Q, int64_t K,
                                         int64_t N, int dtype, int q_diag_only, double* out,
                                         void* cuda_stream) {
  if (L < 0 || K < 0 || N < 0) return SP2_EINVAL;
  if (dtype != SP2_F64 && dtype != SP2_F32) return SP2_EINVAL;
  if (L == 0 || K == 0) return SP2_OK;
  if (L * K > kMaxPairs) return SP2_EINVAL;  // more (l, k) pairs than the scratch serves
  if (!out || (N > 0 && (!P || !Q))) return SP2_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SP2_ECUDA;
  }
  if (!on_device(out, dev) || (N > 0 && (!on_device(P, dev) || !on_device(Q, dev))))
    return SP2_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (N == 0)
    return cudaMemsetAsync(out, 0, sizeof(double) * L * K, s) == cudaSuccess ? SP2_OK : SP2_ECUDA;
  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return SP2_ECUDA;
  }
  // partials per (l, k) pair: the usual count, reduced so that all pairs fit
  int64_t nparts = sp2::contract_nparts(N, q_diag_only);
  if (nparts * L * K > kScratchDoubles) nparts = kScratchDoubles / (L * K);
  const cudaError_t e = sp2::launch_contract(P, L, Q, K, N, dtype, q_diag_only,
                                             static_cast<double*>(scratch), (int)nparts, out, s);
  return e == cudaSuccess ? SP2_OK : SP2_ECUDA;
}
