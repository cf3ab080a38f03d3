// Allocation-free contract-all for callers that cannot allocate device
// memory.
//
// lqc_contract_all_fp64 needs caller-provided scratch for its per-block
// partial sums.  Some callers cannot call cudaMalloc at the point they run a
// contraction: code running inside a CUDA stream capture that must not add
// allocation nodes, plugins of a host framework that owns every device
// allocation, or real-time loops where an allocation could block.  This
// variant takes its scratch from a fixed array that lives in this library's
// device image instead, so a call allocates nothing.
//
// Limits and sharing rules:
//  * the array holds kNoAllocPartials complex128 partial sums (64 KiB), so a
//    call is rejected with LQC_ERR_ARG when lt * chunks exceeds that; with
//    the chunking of the contract-all kernel this means lt <= 4096 slices;
//  * every GPU that loads the library keeps the array until the process
//    exits;
//  * all calls on a device share the one array: calls whose kernels overlap
//    on the GPU (different streams, no ordering between them) race on it
//    and produce wrong sums.  Calls on one stream are ordered and safe;
//  * nothing in the array has to start at zero: each call writes every
//    partial it later reads, so the previous call's leftovers are harmless;
//  * the device address of the array is looked up on the first call on each
//    device (cudaGetSymbolAddress, with that device current); make that first
//    call before starting any stream capture.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.hpp"

namespace {

constexpr int kNoAllocPartials = 4096;  // double2 slots = 64 KiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocPartials];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// device address of the array on the current device (looked up once)
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LQC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return LQC_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return LQC_OK;
}

}  // namespace

extern "C" {

int lqc_contract_all_fp64_noalloc(const double* A, int rank_a, const int64_t* ext_a,
                                  const double* B, int rank_b, const int64_t* ext_b, int npairs,
                                  const int* la, const int* ra, int64_t lt, double* C,
                                  void* stream) {
  if (!A || !B || !C || !ext_a || !ext_b || !la || !ra || lt < 1) return LQC_ERR_ARG;
  lqc::ContractAllDesc d;
  std::string err;
  if (!lqc::make_contract_all_desc(rank_a, ext_a, rank_b, ext_b, npairs, la, ra, lt, &d, &err))
    return LQC_ERR_ARG;
  if (lt * (int64_t)d.chunks > kNoAllocPartials) return LQC_ERR_ARG;  // beyond the fixed array
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != LQC_OK) return rc;
  lqc::clear_pending_error();
  int k = lqc::launch_contract_all_fp64(d, A, B, C, static_cast<double*>(scratch),
                                         static_cast<cudaStream_t>(stream));
  return lqc::launch_status(k);
}

}  // extern "C"
