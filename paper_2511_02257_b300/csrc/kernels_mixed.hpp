// Descriptors and launchers of the mixed-precision kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

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

// Permuted copy of a complex64 tensor into a contiguous layout:
// dst[t][i] = src[t][offset of dst index i], the dst axes listed row-major with
// their source strides.  Rows that stay contiguous in the source are copied
// as runs; otherwise 32 x 32 tiles are transposed through shared memory, so
// both the reads and the writes are coalesced.
struct PermDesc {
  int lt;
  long long n, src_ts;   // elements per slice of dst, of src
  int mode;              // 0: runs along dst's innermost axis, 1: transposed tiles
  int X, Y;              // extents: dst innermost axis; (mode 1) the src-contiguous axis
  long long sX, dY;      // (mode 1) src stride of the dst innermost axis, dst stride of Y
  int nout;              // outer axes (everything else), row-major
  int oext[LQC_MAX_RANK];
  long long osrc[LQC_MAX_RANK], odst[LQC_MAX_RANK];
  long long outer;       // outer index combinations
  long long blocks;      // blocks per slice
};
struct MixedDesc {
  ContractDesc cd;
  bool bf16;
  int64_t kp;               // real k (2K) padded to 16-byte rows
  int splits, kblocks;      // k splits and k blocks per split
  int64_t plane_a, plane_b; // bytes of one hi or lo plane
  int64_t a_off, b_off, part_off, scratch_bytes;
  // fused form (TF32, even K): raw complex64 operands, read in place when
  // already [rows][K] with K unit-stride, else reordered into scratch
  bool fused;
  bool a_direct, b_direct;
  bool b_mn;                // B read in place as [k][n]; the GEMM's converters transpose it
  bool b_mn2;               // ... as [k][outer n][inner n] blocks (4-d map)
  bool a_mn;                // A read in place as [k][rows] (rows unit-stride), or with a_ni
                            // as [outer rows][k][inner rows]; transposed by the converters
  int64_t a_ni;             // a_mn: 0 = one row group, else the inner row extent
  int64_t a_outer_stride;   // a_ni: complex elements between outer row blocks
  bool swap;                // operands exchanged: the GEMM computes C^T = B^T A^T (its rows
                            // are C's columns) and stores it transposed; cd describes the
                            // exchanged roles
  int64_t a_rowstride, b_rowstride;  // complex elements between operand rows (a_mn: k rows)
  PermDesc a_perm, b_perm;
  bool tmem_a;              // fused form: A split by converter warps into tensor memory
  bool pair;                // fused form: CTA pairs (cta_group::2) on 256-row tiles
};
bool make_fused_desc(const ContractDesc& cd, MixedDesc* d, int split_policy);

// Choices the autotuner makes per DAG: right operands of at most
// fused_max_n complex columns take the fused form (TF32, even K); split
// policy 0 splits k while the output tiles cannot fill the GPU (and for the
// FP32 chunk bound), 1 only for the FP32 chunk bound.
struct MixedTune {
  int64_t fused_max_n = 64;
  int split_policy = 0;
  int fused_kernel = 0;     // fused form: 0 = A staged in shared memory, 1 = A in TMEM,
                            // 2 = as 0 with CTA pairs for products of more than 128 rows
};
bool make_mixed_desc(const ContractDesc& cd, bool bf16, MixedDesc* d,
                     const MixedTune& tune = MixedTune());

// g: dst axes (extent, source stride), row-major order.
void make_perm_desc(const Group& g, int64_t lt, int64_t src_ts, PermDesc* d);
// true when the permute / correlator blocks can index the slices (32-bit)
bool perm_fits(const PermDesc& d);
int launch_permute_c64(const PermDesc& d, const float* src, float* dst, cudaStream_t s);
// bytes of scratch the complex64 contract-all needs (partials + a reordered
// copy of the right operand when its pairing is not contiguous)
int64_t contract_all_c64_scratch_bytes(const ContractAllDesc& d);
// A, B, C: complex64 tensors (interleaved floats); scratch: d.scratch_bytes.
// Returns kernels launched, -1 launch error, -2 tensor-map encode failure.
int launch_contract_mixed(const MixedDesc& d, const float* A, const float* B, float* C,
                          void* scratch, cudaStream_t s);
// Correlator of two complex64 tensors, FP64 accumulation, times `scale`.
int launch_contract_all_c64(const ContractAllDesc& d, const float* A, const float* B, double* C,
                            double* scratch, double scale, cudaStream_t s);
// ---- grouped window levels (mixed precisions)
// one exterior contraction of a level: its descriptor, operands, output and
// its own scratch region (planes, split partials) of d->scratch_bytes
struct GroupExt {
  const MixedDesc* d;
  const float* A;
  const float* B;
  float* C;
  char* scratch;
};
// one correlator of a level: its scratch region `part` of
// contract_all_c64_scratch_bytes (the per-block FP64 partial sums)
struct GroupRoot {
  const ContractAllDesc* d;
  const float* A;
  const float* B;
  double* C;
  double* part;
  double scale;
};
// task tables of one level (device pointers after rebase_level)
// (each *_starts array: the tasks' first block indices, ascending, for the
// block -> task search of the grouped kernels)
struct LevelDev {
  const void* pack;
  const long long* pack_starts;
  int npack;
  long long pack_blocks;
  const void* gemm;
  int ngemm;
  long long gemm_tiles;
  const void* gemm_fused;
  int ngemm_fused;
  long long gemm_fused_tiles;
  bool fused_tmem_a;        // the fused tasks run the A-in-tensor-memory kernel
  bool fused_amn;           // ... and some reads A as [k][rows] tiles
  const void* gemm_pair;    // fused tasks run by CTA pairs (one more launch)
  int ngemm_pair;
  long long gemm_pair_tiles;
  bool pair_amn;
  const void* red;
  const long long* red_starts;
  int nred;
  long long red_blocks;
  const void* perm;
  const long long* perm_starts;
  int nperm;
  long long perm_blocks;
  const void* ca;
  const long long* ca_starts;   // first block of each (task, slice) segment
  const void* ca_segs;          // the segments, slice-major
  int nca, nca_seg;
  long long ca_blocks, ca_threads;
  bool bf16;
};
// Append a level's task tables to `buf` (offsets stored in *lvl, relative to
// the start of buf); false if a tensor map cannot be encoded.  Pointers in
// the members must already be final device addresses.
bool append_level_tasks(const std::vector<GroupExt>& ext, const std::vector<GroupRoot>& roots,
                        bool bf16, std::vector<char>* buf, LevelDev* lvl);
// turn the offsets into device addresses once buf has been copied to `base`
void rebase_level(LevelDev* lvl, const char* base);
// kinds (lqc_launch_kind) of the launches of one level, in launch order;
// returns their number
int level_launch_kinds(const LevelDev& lvl, int kinds[LQC_NUM_KINDS]);
// launch one level on `s`; returns kernels launched or -1.  marks (nullable):
// level_launch_kinds() + 1 events, marks[i] recorded before the i-th launch
// and the last after the final one, with cudaEventRecordWithFlags(mark_flags)
int launch_level(const LevelDev& lvl, cudaStream_t s, cudaEvent_t* marks = nullptr,
                 unsigned mark_flags = 0);

// First error code recorded by a mixed kernel (bounded wait expired), or 0;
// -1 if it cannot be read.  reset = clear it after reading.
int mixed_error_status(bool reset);

}  // namespace lqc
