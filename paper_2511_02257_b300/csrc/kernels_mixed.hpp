// Descriptors and launchers of the mixed-precision kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.hpp"

namespace lqc {

// one operand of a contraction for the pack kernel
struct PackArgs {
  int which;        // 0: A operand (rows = M), 1: B operand (rows = N)
  int rows, K;      // complex rows and paired extent
  long long kp;     // padded real row length of the planes
  long long ts;     // complex elements per time slice of the operand
  int k_fast;       // operand's unit-stride axis is a paired axis
  Group rg, kg;     // row group (free axes) and k group (paired axes)
};

struct MixedDesc {
  ContractDesc cd;
  bool bf16;
  int64_t kp;               // real k (2K) padded to 16-byte rows
  int splits, kblocks;      // k splits and k blocks per split
  int64_t plane_a, plane_b; // bytes of one hi or lo plane
  int64_t a_off, b_off, part_off, scratch_bytes;
};

bool make_mixed_desc(const ContractDesc& cd, bool bf16, MixedDesc* d);
// A, B, C: complex64 tensors (interleaved floats); scratch: d.scratch_bytes.
// Returns kernels launched, -1 launch error, -2 tensor-map encode failure.
int launch_contract_mixed(const MixedDesc& d, const float* A, const float* B, float* C,
                          void* scratch, cudaStream_t s);
// Correlator of two complex64 tensors, FP64 accumulation, times `scale`.
int launch_contract_all_c64(const ContractAllDesc& d, const float* A, const float* B, double* C,
                            double* scratch, double scale, cudaStream_t s);
// First error code recorded by a mixed kernel (bounded wait expired), or 0;
// -1 if it cannot be read.  reset = clear it after reading.
int mixed_error_status(bool reset);

}  // namespace lqc
