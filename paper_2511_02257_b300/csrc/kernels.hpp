// Device-kernel descriptors and launchers shared by the executor and the
// single-contraction entry points.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/lqc.h"

namespace lqc {

// One-shot C entry points: an error that earlier, unrelated runtime calls of
// this thread left pending must not fail this call, and this call's own
// launch error must not fail later ones.  Clear before launching, consume
// after a failed launch (a sticky device error still fails both).
inline void clear_pending_error() { (void)cudaGetLastError(); }
inline int launch_status(int kernels) {
  if (kernels >= 0) return LQC_OK;
  (void)cudaGetLastError();
  return LQC_ERR_CUDA;
}

// A set of tensor axes flattened row-major into one index: element offset of
// flattened index i = sum_d digit_d(i) * stride[d], digits taken with the
// last axis innermost.
struct Group {
  int n;
  int ext[LQC_MAX_RANK];
  long long stride[LQC_MAX_RANK];
};

// One binary contraction viewed as a batched complex GEMM after index
// permutation: C[t][m][n] = sum_k A[t][am(m) + ak(k)] * B[t][bk(k) + bn(n)].
// m runs over the left operand's free axes, n over the right operand's free
// axes, k over the paired axes (pair order); strides are in complex elements.
struct ContractDesc {
  long long M, N, K, lt;
  long long a_ts, b_ts;          // complex elements per time slice of A, B
  Group am, ak, bk, bn;
  int a_kfast;                    // 1: A's unit-stride axis is a paired axis
  int b_kfast;                    // 1: B's unit-stride axis is a paired axis
};

// Contract-all: C[t] = sum_i A[t][i] * B[t][bp(i)], i = A's element index.
struct ContractAllDesc {
  long long S, lt;                // elements per slice, slices
  Group bp;                       // A's axes with the strides of B's paired axes
  int chunks;                     // partial sums per slice
};

// Build descriptors from shapes (rank/extents exclude the batch axis).
// Return false with *err set when shapes or pairs are inconsistent.
bool make_contract_desc(int rank_a, const int64_t* ext_a, int rank_b, const int64_t* ext_b,
                        int npairs, const int* la, const int* ra, int64_t lt,
                        ContractDesc* d, std::string* err);
bool make_contract_all_desc(int rank_a, const int64_t* ext_a, int rank_b, const int64_t* ext_b,
                            int npairs, const int* la, const int* ra, int64_t lt,
                            ContractAllDesc* d, std::string* err);
int64_t contract_all_scratch_bytes(const ContractAllDesc& d);
int contract_all_chunks(int64_t lt, int64_t S);

// Launchers (asynchronous on `s`); return the number of kernels launched,
// or -1 on a launch error (cudaGetLastError() holds the cause).
int launch_contract_fp64(const ContractDesc& d, const double* A, const double* B, double* C,
                         cudaStream_t s);
int launch_contract_all_fp64(const ContractAllDesc& d, const double* A, const double* B,
                             double* C, double* scratch, cudaStream_t s);
int launch_fill_nan(void* p, int64_t bytes, cudaStream_t s);

}  // namespace lqc
