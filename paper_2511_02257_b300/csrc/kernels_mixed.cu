// Mixed-precision kernels: complex64 storage, split (hi + lo) tensor-core
// products with FP32 accumulation in TMEM, FP64 where sums form results.
//
// Real embedding of a complex contraction C = A B (per time slice):
//   A' [m][2k]   = Re A(m,k),  A' [m][2k+1]  = Im A(m,k)   (the complex64 row)
//   B'T[2n][2k]  = Re B(k,n),  B'T[2n][2k+1] = -Im B(k,n)
//   B'T[2n+1][2k]= Im B(k,n),  B'T[2n+1][2k+1]= Re B(k,n)
// so that the real product A' B' is the complex product already interleaved
// as (re, im): D'[m][2n] = Re C(m,n), D'[m][2n+1] = Im C(m,n).  Each operand
// value x is split into hi = x rounded to the tensor-core type and lo =
// (x - hi) rounded.
//
// K3  pack (plane form): gathers one operand (any axis permutation, folded
//     into the loads) and writes its hi/lo planes in that layout.
// K4  gemm, persistent over a tile sequence (one contraction or a grouped
//     level's task table): TMA (128-byte swizzle) feeds a shared-memory ring;
//     one thread issues tcgen05.mma (kind::tf32, or kind::f16 with bf16):
//     hi*hi into one FP32 accumulator in TMEM and lo*hi + hi*lo into a
//     second, so the small terms never round against the large running sum.
//     The tensor core's own FP32 accumulation is kept short: every
//     kChunkBlocks k-blocks the MMA thread switches to the other of two TMEM
//     buffers and eight drain warps add the finished one into FP32 registers
//     (one output row per thread), then stage 32x16 output blocks through
//     shared memory for coalesced stores.  Fused form (TF32): TMA brings raw
//     complex64 tiles (K-major, [k][rows] for left operands contracted over
//     their leading axis, or [k][n] for right operands read in place through
//     maps of up to 5 dimensions) and converter warps build the hi/lo operand
//     tiles.  Products with fewer rows than a tile run exchanged (C^T = B^T
//     A^T) and the epilogue stores them transposed.  Products of more than
//     128 rows can run on CTA pairs (cta_group::2, 256-row tiles, each CTA
//     converting half of the B' tile).  Contractions longer than kMaxChunk
//     real k are split over k into FP32 partial tiles summed in double-float.
// Reorder / K2m: a PermDesc maps destination elements to source offsets;
//     blocks of runs or of transposed tiles copy operands into [rows][K]
//     order, and the correlators (contract-all, double-float sums per thread
//     and per block, FP64 across blocks) visit their partner in place.
// Grouped launches run each kind over every member of a window level.
//
// Every wait on an mbarrier is bounded (2 s of %globaltimer); on expiry the
// kernel records an error code, drains what it started and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "kernels.hpp"
#include "kernels_mixed.hpp"

namespace lqc {

namespace {

constexpr int kBM = 128;        // UMMA M (rows of A' per CTA)
constexpr int kBN = 128;        // UMMA N (real columns of D' per CTA)
constexpr int kStages = 3;
constexpr int kTmemCols = 4 * kBN;  // 2 main accumulators (per chunk) + 2 correction (per tile)
constexpr int64_t kMaxChunk = 1024;  // real k summed in FP32 registers before an FP64 sum
constexpr int kDrainWarps = 8;  // two per TMEM lane quarter, one per column half
constexpr int kConvWarps = 6;   // fused form: raw complex64 tiles -> hi/lo operand tiles
constexpr int kGemmThreads = 64 + 32 * kDrainWarps;
constexpr int kChunkBlocks = 2;     // k-blocks per TMEM accumulation before a drain
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ int g_mixed_error = 0;  // first error code seen by a mixed kernel

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Rounding to TF32 (10 stored mantissa bits) to nearest, ties away from
// zero: add half a unit of the last kept bit to the magnitude bits and clear
// the 13 dropped bits (a carry into the exponent is the correct round-up).
// Two full-rate integer operations instead of a conversion instruction; the
// converter warps issue two per split value.  Equal to cvt.rna.tf32.f32 for
// finite inputs (checked on the device by lqc_test_tf32_rounding).
__device__ __forceinline__ float round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait: false after limit_ns (kWaitNs in every kernel but the
// wait probe below)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// Test of the TF32 rounding: n values x_i spread over every binade and
// mantissa pattern (x_i = bit pattern hash(seed, i), finite values only),
// each rounded by round_tf32 and by the hardware conversion cvt.rna; counts
// the values where the two differ.
__global__ void k_tf32_rounding_check(long long n, unsigned seed, unsigned long long* bad) {
  unsigned long long local = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 0x9E3779B1u ^ seed;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    if ((h & 0x7F800000u) == 0x7F800000u) h &= 0xBF7FFFFFu;  // Inf / NaN patterns -> finite
    if (i < 4096) h = (h & 0xFFFFE000u) | 0x1000u;           // exact ties first
    const float x = __uint_as_float(h);
    uint32_t hw;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hw) : "f"(x));
    if (__float_as_uint(round_tf32(x)) != hw) ++local;
  }
  if (local) atomicAdd(bad, local);
}

// Test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives on, for limit_ns; the expiry takes the GEMM's path (the device
// error word) and the kernel returns.
__global__ void k_wait_probe(unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0, limit_ns)) atomicCAS(&g_mixed_error, 0, 1);
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(c4)
      : "memory");
}
// K-major operand tile with 128-byte swizzle: rows of 128 B, 8-row atoms of
// 1024 B (stride-dimension offset), descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
template <bool BF16>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accum) {
  if (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  }
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// ---- CTA pairs (cluster of 2, cta_group::2)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// arrive on the mbarrier at the same shared-memory offset in CTA 0 of the
// pair.  The default (CTA-scope release) form: the converters' stores are
// ordered for the tensor core by their fence.proxy.async before it; the
// cluster-scope release form measured 26 % slower on 256^3 products.
__device__ __forceinline__ void mbar_arrive_leader(uint64_t* bar) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(remote) : "r"(smem_u32(bar)));
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}
// 2-SM MMA issued by CTA 0: A rows 0..127 from CTA 0's shared memory and
// 128..255 from CTA 1's (same offsets), B' rows (output columns) split the
// same way; D rows land in each CTA's own tensor memory
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
// arrive on the mbarrier at this offset in both CTAs once the pair's MMAs
// issued so far have completed
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)), "h"((unsigned short)3)
      : "memory");
}

// two 16-column TMEM loads in flight before one wait
__device__ __forceinline__ void tmem_ld16_pair(uint32_t ta, uint32_t tb, uint32_t* r,
                                               uint32_t* s) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]),
        "=r"(s[7]), "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]),
        "=r"(s[14]), "=r"(s[15])
      : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <bool BF16>
struct Split;
template <>
struct Split<false> {
  typedef float T;
  __device__ static void split(float x, float& hi, float& lo) {
    hi = round_tf32(x);
    lo = round_tf32(x - hi);  // x - hi is exact
  }
  __device__ static void store2(float* p, float a, float b) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
  }
};
template <>
struct Split<true> {
  typedef __nv_bfloat16 T;
  __device__ static void split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
  }
  __device__ static void store2(__nv_bfloat16* p, __nv_bfloat16 a, __nv_bfloat16 b) {
    __nv_bfloat162 v;
    v.x = a;
    v.y = b;
    *reinterpret_cast<__nv_bfloat162*>(p) = v;
  }
};

// instruction descriptor: D f32, A/B tf32 (kind::tf32) or bf16 (kind::f16),
// both K-major, M = 128, N = kBN
template <bool BF16>
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) |
         ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

// ------------------------------------------------------------ K4 GEMM
// One GEMM of the split form: tensor maps of the four planes, output and
// tiling.  A launch covers one task (single contraction, passed as a kernel
// parameter) or a table of tasks in global memory (a grouped window level);
// tiles of all tasks form one sequence, task k owning
// [tile_start, tile_start + tiles).
struct GemmTask {  // 64-byte aligned through its tensor maps
  CUtensorMap map[4];   // Ahi, Alo, Bhi, Blo
  float* out;           // splits == 1: D' [lt][M][Nr]; else partials [splits][lt][M][Nr]
  int M, Nr, kblocks, splits, lt, ntn, ntm, tiles;
  int b_mn;             // fused form: B read in place with n unit-stride ([k][n] tiles that the
                        // converters transpose): 1 = one k and one n axis (3-d map); 2 = general
  int b_ni;             // 2: columns of the inner n axis (b_no: an outer n axis follows the k axes)
  int b_nk, b_no;       // 2: k axes in the map (innermost first), outer n axis present
  int b_kext[3];        // 2: extents of the k axes, innermost first
  long long tile_start;
  // fused form, A read by the converters themselves (A in tensor memory):
  // complex64 rows [lt][M][kc] with row stride a_rs and slice stride a_ts
  // (complex elements, both even), 16-byte aligned
  const float2* a_raw;
  long long a_ts, a_rs;
  int kc;
  int a_mn;             // fused form: A read in place with its rows unit-stride, transposed
                        // by the converters: 1 = [k][rows] (3-d map, raw tile [16 k][128
                        // rows]); 2 = [outer rows][k][inner rows] (4-d map, raw tile
                        // [128 / a_ni outer][16 k][a_ni inner])
  int a_ni;             // a_mn: inner rows per raw-tile block (128 for a_mn 1; 16, 32, 64 or
                        // 128 for a_mn 2)
  int a_nio;            // a_mn 2: the inner row extent (a multiple of 128 when a_ni = 128)
  int out_t;            // D' row r, real column c -> out[((c / 2) * M + r) * 2 + (c & 1)]
                        // of each slice: the transposed product of exchanged operands
};

struct GemmParams {
  GemmTask single;        // used when tasks == nullptr
  const GemmTask* tasks;  // grouped launch: task table in global memory
  int ntasks;
  long long total_tiles;
};

// task owning global tile g; k is a cursor that only moves forward (a CTA's
// tiles increase)
__device__ __forceinline__ const GemmTask* tile_task(const GemmParams& gp, long long g, int& k,
                                                     int& local) {
  if (!gp.tasks) {
    local = (int)g;
    return &gp.single;
  }
  while (g >= gp.tasks[k].tile_start + gp.tasks[k].tiles) ++k;
  local = (int)(g - gp.tasks[k].tile_start);
  return &gp.tasks[k];
}


// FUSED (TF32 only): the producer loads raw complex64 K-major tiles (A: 128
// rows, B: 64 complex rows, 128 bytes of k each) into a raw ring and
// converter warps write the hi/lo operand tiles (B' rows 2n / 2n+1 built from
// complex row n) into the operand ring; otherwise the producer loads the
// four precomputed planes directly into the operand ring.
// PAIR (fused form only): a CTA pair (cluster of 2) computes 256-row tiles
// with cta_group::2 MMAs (M = 256, N = kBN): each CTA stages its own 128 A'
// rows and half of the tile's B' rows (kBN / 2), so each B' tile is
// converted once per pair instead of once per CTA, and the smaller stage
// leaves room for a third operand stage.
template <bool BF16, bool FUSED = false, bool PAIR = false>
struct GemmCfg {
  static constexpr int kElem = BF16 ? 2 : 4;
  static constexpr int kBK = 128 / kElem;           // elements per 128-byte row
  static constexpr int kATile = kBM * 128;          // bytes of one A plane tile
  static constexpr int kBRows = PAIR ? kBN / 2 : kBN;  // B' rows staged by one CTA
  static constexpr int kBTile = kBRows * 128;
  static constexpr int kBCols = kBRows / 2;         // complex columns of B per CTA
  static constexpr int kStageBytes = 2 * kATile + 2 * kBTile;
  static constexpr int kOpStages = FUSED ? (PAIR ? 3 : 2) : kStages;
  static constexpr int kRawStages = FUSED ? 3 : 0;
  static constexpr int kRawA = kBM * 128, kRawB = kBCols * 128;
  static constexpr int kRawBytes = kRawA + kRawB;
  static constexpr int kThreads = kGemmThreads + (FUSED ? 32 * kConvWarps : 0);
  // epilogue staging: per drain warp 32 rows x 16 columns, pitch 20 floats
  static constexpr int kStgPitch = 20;
  static constexpr int kStgBytes = kDrainWarps * 32 * kStgPitch * 4;
  static constexpr int kSmem = kOpStages * kStageBytes + kRawStages * kRawBytes +
                               1024 /* align */ + 256 /* barriers */ + kStgBytes;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent: CTA c handles tiles c, c + gridDim.x, ... of the launch's tile
// sequence; inside a task, tiles are ordered n-tile fastest, then m-tile,
// then (slice, k split), so neighbouring CTAs share operand tiles in L2.
// Warp roles: warp 0 lane 0 = TMA producer, warp 1 lane 0 = MMA issuer,
// warps 2..9 = drain/epilogue (warp w reads TMEM lanes 32*(w%4) .. +31, i.e.
// one output row per thread, and one half of the kBN columns).  All roles walk
// the same flattened (tile, k-block) sequence: the shared-memory ring and the
// two TMEM accumulator buffers (each 2*kBN columns: main + correction) keep
// cycling across tiles and tasks, so a tile's store overlaps the next tile's
// MMAs.  The drain warps empty a buffer every kChunkBlocks k-blocks into FP32
// registers.  AMN: the launch may hold [k][rows] A tiles (a second copy of the
// converters' A loops, taken per task; without it the default loops alone).
// PAIR: launched in clusters of 2; the pair walks 256-row tiles (pair p takes
// tiles p, p + gridDim.x / 2, ...), CTA 0's thread issues the cta_group::2
// MMAs, and the converter and drain warps of CTA 1 arrive on CTA 0's
// barriers; the commits arrive in both CTAs.
template <bool BF16, bool FUSED, bool AMN = false, bool PAIR = false>
__global__ void __launch_bounds__(GemmCfg<BF16, FUSED>::kThreads, 1)
k_gemm_split3(const __grid_constant__ GemmParams gp) {
  using C = GemmCfg<BF16, FUSED, PAIR>;
  static_assert(!PAIR || (FUSED && !BF16), "CTA pairs: fused TF32 form only");
  constexpr int S = C::kOpStages, R = C::kRawStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* raw = smem + S * C::kStageBytes;  // FUSED: raw complex64 ring
  uint64_t* full = reinterpret_cast<uint64_t*>(raw + R * C::kRawBytes);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;         // [2] accumulator buffer ready to drain
  uint64_t* tempty = tfull + 2;        // [2] accumulator buffer drained
  uint64_t* done = tempty + 2;         // every MMA issued has completed
  uint64_t* rfull = done + 1;          // FUSED [R] raw stage landed
  uint64_t* rempty = rfull + R;        // FUSED [R] raw stage converted
  uint64_t* cempty = rempty + R;       // [2] correction accumulator of a tile drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(cempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* stage_out = reinterpret_cast<float*>(raw + R * C::kRawBytes + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tile walk: this CTA's (or pair's) first tile and stride; rank in the pair
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const long long tile0 = PAIR ? (long long)(blockIdx.x >> 1) : (long long)blockIdx.x;
  const long long tstep = PAIR ? (long long)(gridDim.x >> 1) : (long long)gridDim.x;
  constexpr int kTileRows = PAIR ? 2 * kBM : kBM;  // rows of a (pair) tile
  constexpr int kPeers = PAIR ? 2 : 1;             // CTAs arriving on CTA 0's barriers

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], FUSED ? kConvWarps * kPeers : 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < R; ++i) {
      mbar_init(&rfull[i], 1);
      mbar_init(&rempty[i], kConvWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kDrainWarps * kPeers);
      mbar_init(&cempty[b], kDrainWarps * kPeers);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    if constexpr (PAIR) {  // one warp of each CTA of the pair, collectively
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(kTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(kTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if constexpr (PAIR) cluster_sync_all();  // both CTAs' barriers initialised
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      constexpr int RS = FUSED ? R : S;  // ring the producer fills
      uint64_t* rf = FUSED ? rfull : full;
      uint64_t* re = FUSED ? rempty : empty;
      int g = 0, issued = 0, k = 0, local = 0;
      bool stop = false;
      for (long long tile = tile0; tile < gp.total_tiles && !stop; tile += tstep) {
        const GemmTask* tk = tile_task(gp, tile, k, local);
        const int tn = local % tk->ntn, tm = (local / tk->ntn) % tk->ntm;
        const int z = local / (tk->ntn * tk->ntm);
        const int t = z % tk->lt, split = z / tk->lt;
        // this CTA's rows and B' columns (a pair: CTA r takes rows 128 r.. of
        // the 256-row tile and B' columns kBN / 2 * r .. of its kBN)
        const int n0 = tn * kBN + (int)rank * (kBN / 2), m0 = tm * kTileRows + (int)rank * kBM;
        const int kb0 = split * tk->kblocks;
        for (int i = 0; i < tk->kblocks; ++i, ++g) {
          const int st = g % RS;
          const uint32_t ph = (uint32_t)(g / RS) & 1u;
          if (!mbar_wait(&re[st], ph ^ 1u) || *abort_flag) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          const int k0 = (kb0 + i) * C::kBK;
          if (FUSED) {
            uint8_t* rp = raw + st * C::kRawBytes;
            mbar_expect_tx(&rf[st], C::kRawBytes);
            if (tk->a_mn == 1)  // [16 complex k rows][128 complex rows], unswizzled
              tma_load_3d(rp, &tk->map[0], &rf[st], 2 * m0, k0 / 2, t);
            else if (tk->a_mn == 2)  // [outer][16 k][inner] blocks holding rows m0 .. m0 + 127
              tma_load_4d(rp, &tk->map[0], &rf[st], 2 * (m0 % tk->a_nio), k0 / 2,
                          m0 / tk->a_nio, t);
            else
              tma_load_3d(rp, &tk->map[0], &rf[st], k0, m0, t);
            if (tk->b_mn == 2) {  // the same tile inside one block of every outer axis
              int c[5], nd = 0, kk = k0 / 2;
              c[nd++] = n0 % (2 * tk->b_ni);
              for (int a = 0; a < tk->b_nk; ++a) {
                c[nd++] = kk % tk->b_kext[a];
                kk /= tk->b_kext[a];
              }
              if (tk->b_no) c[nd++] = n0 / (2 * tk->b_ni);
              c[nd++] = t;
              if (nd == 3) tma_load_3d(rp + C::kRawA, &tk->map[2], &rf[st], c[0], c[1], c[2]);
              else if (nd == 4)
                tma_load_4d(rp + C::kRawA, &tk->map[2], &rf[st], c[0], c[1], c[2], c[3]);
              else
                tma_load_5d(rp + C::kRawA, &tk->map[2], &rf[st], c[0], c[1], c[2], c[3], c[4]);
            } else if (tk->b_mn)  // [16 complex k rows][kBN/2 complex n], unswizzled
              tma_load_3d(rp + C::kRawA, &tk->map[2], &rf[st], n0, k0 / 2, t);
            else
              tma_load_3d(rp + C::kRawA, &tk->map[2], &rf[st], k0, n0 / 2, t);
          } else {
            uint8_t* sp = smem + st * C::kStageBytes;
            mbar_expect_tx(&rf[st], C::kStageBytes);
            tma_load_3d(sp, &tk->map[0], &rf[st], k0, m0, t);
            tma_load_3d(sp + C::kATile, &tk->map[1], &rf[st], k0, m0, t);
            tma_load_3d(sp + 2 * C::kATile, &tk->map[2], &rf[st], k0, n0, t);
            tma_load_3d(sp + 2 * C::kATile + C::kBTile, &tk->map[3], &rf[st], k0, n0, t);
          }
          issued = g + 1;
        }
      }
      // every issued load must have landed before the CTA exits
      for (int i = (issued > RS ? issued - RS : 0); i < issued; ++i)
        if (!mbar_wait(&rf[i % RS], (uint32_t)(i / RS) & 1u)) break;
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ---- MMA issuer (a pair: CTA 0's)
      constexpr uint32_t idesc =
          make_idesc<BF16>() + (PAIR ? ((uint32_t)(kBM >> 4) << 24) : 0u);  // M = 256
      int g = 0, cc = 0, tt = 0, k = 0, local = 0;  // k-blocks, chunks, tiles walked
      bool stop = false;
      for (long long tile = tile0; tile < gp.total_tiles && !stop; tile += tstep, ++tt) {
        const GemmTask* tk = tile_task(gp, tile, k, local);
        const int kblocks = tk->kblocks;
        // the tile's correction accumulator: free once the drain warps have
        // read the one of tile tt - 2
        if (!mbar_wait(&cempty[tt & 1], ((uint32_t)(tt >> 1) & 1u) ^ 1u) || *abort_flag) {
          *abort_flag = 1;
          break;
        }
        const uint32_t dcorr = tmem + (uint32_t)((2 + (tt & 1)) * kBN);
        for (int i = 0; i < kblocks; ++i, ++g) {
          const int b = cc & 1;
          const bool first = (i % kChunkBlocks) == 0;
          const bool last = (i % kChunkBlocks) == kChunkBlocks - 1 || i == kblocks - 1;
          if (first) {  // wait until the drain warps have emptied this buffer
            if (!mbar_wait(&tempty[b], ((uint32_t)(cc >> 1) & 1u) ^ 1u) || *abort_flag) {
              *abort_flag = 1;
              stop = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          }
          const int st = g % S;
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(&full[st], ph) || *abort_flag) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t base = smem_u32(smem + st * C::kStageBytes);
          const uint32_t ahi = base, alo = base + C::kATile;
          const uint32_t bhi = base + 2 * C::kATile, blo = bhi + C::kBTile;
          const uint32_t dmain = tmem + (uint32_t)(b * kBN);
#pragma unroll
          for (int kk = 0; kk < 128 / 32; ++kk) {  // 32-byte k-steps inside the 128-byte row
            const uint32_t off = kk * 32;
            const uint32_t acc0 = (!first || kk > 0) ? 1u : 0u;     // main: fresh per chunk
            const uint32_t accc = (i > 0 || kk > 0) ? 1u : 0u;      // correction: per tile
            if constexpr (PAIR) {
              umma_pair(dcorr, sdesc_sw128(alo + off), sdesc_sw128(bhi + off), idesc, accc);
              umma_pair(dcorr, sdesc_sw128(ahi + off), sdesc_sw128(blo + off), idesc, 1u);
              umma_pair(dmain, sdesc_sw128(ahi + off), sdesc_sw128(bhi + off), idesc, acc0);
            } else {
              umma<BF16>(dcorr, sdesc_sw128(alo + off), sdesc_sw128(bhi + off), idesc, accc);
              umma<BF16>(dcorr, sdesc_sw128(ahi + off), sdesc_sw128(blo + off), idesc, 1u);
              umma<BF16>(dmain, sdesc_sw128(ahi + off), sdesc_sw128(bhi + off), idesc, acc0);
            }
          }
          // stage reusable once these MMAs have read it (a pair: in both CTAs)
          if constexpr (PAIR) umma_commit_pair(&empty[st]);
          else umma_commit(&empty[st]);
          if (last) {
            if constexpr (PAIR) umma_commit_pair(&tfull[b]);
            else umma_commit(&tfull[b]);
            ++cc;
          }
        }
      }
      // all issued MMAs complete (or abandoned)
      if constexpr (PAIR) umma_commit_pair(done);
      else umma_commit(done);
    }
  } else if (warp < 2 + kDrainWarps) {
    // ---- drain / epilogue warps
    constexpr int kHalf = kBN / 2;
    const int q = warp & 3;          // TMEM lane quarter of this warp
    const int c0 = ((warp - 2) >> 2) * kHalf;  // first column of this warp's half
    const uint32_t tlane = ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
    int cc = 0, tt = 0, ok = 1, k = 0, local = 0;
    for (long long tile = tile0; tile < gp.total_tiles && ok; tile += tstep, ++tt) {
      const GemmTask* tk = tile_task(gp, tile, k, local);
      const int tn = local % tk->ntn, tm = (local / tk->ntn) % tk->ntm;
      const int z = local / (tk->ntn * tk->ntm);
      const int t = z % tk->lt, split = z / tk->lt;
      const int M = tk->M, Nr = tk->Nr;
      const int chunks = (tk->kblocks + kChunkBlocks - 1) / kChunkBlocks;
      const int mrow0 = tm * kTileRows + (int)rank * kBM;  // this CTA's first row
      const int row = mrow0 + q * 32 + lane;
      float acc[kHalf];
#pragma unroll
      for (int j = 0; j < kHalf; ++j) acc[j] = 0.f;
      for (int c = 0; c < chunks; ++c, ++cc) {
        const int b = cc & 1;
        if (lane == 0) {
          if (!mbar_wait(&tfull[b], (uint32_t)(cc >> 1) & 1u) || *abort_flag) {
            *abort_flag = 1;
            ok = 0;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the chunk's main accumulator; after the tile's last chunk (whose
        // commit covers every MMA of the tile) also its correction accumulator,
        // which stays in TMEM for the whole tile: its values are about 2^-11
        // of the main ones, so its in-TMEM rounding is negligible
        const bool last = c == chunks - 1;
        const uint32_t tb = tmem + tlane + (uint32_t)(b * kBN);
        const uint32_t tc = tmem + tlane + (uint32_t)((2 + (tt & 1)) * kBN);
#pragma unroll
        for (int j = 0; j < kHalf; j += 32) {
          uint32_t r[16], r2[16];
          tmem_ld16_pair(tb + j, tb + j + 16, r, r2);  // collective: every lane loads
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            acc[j + u] += __uint_as_float(r[u]);
            acc[j + 16 + u] += __uint_as_float(r2[u]);
          }
          if (last) {
            tmem_ld16_pair(tc + j, tc + j + 16, r, r2);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              acc[j + u] += __uint_as_float(r[u]);
              acc[j + 16 + u] += __uint_as_float(r2[u]);
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (PAIR && rank != 0) {  // the MMA thread of CTA 0 waits on its own barriers
            mbar_arrive_leader(&tempty[b]);
            if (last) mbar_arrive_leader(&cempty[tt & 1]);
          } else {
            mbar_arrive(&tempty[b]);
            if (last) mbar_arrive(&cempty[tt & 1]);
          }
        }
      }
      if (ok && tk->out_t) {
        // transposed store: this thread's row r is an output column, its
        // column pairs (re, im) are output rows: for each pair the warp
        // writes 32 consecutive complex values
        if (row < M) {
          float* base = tk->out + ((size_t)split * tk->lt + t) * (size_t)M * Nr;
          const int col0 = tn * kBN + c0;
#pragma unroll
          for (int j = 0; j < kHalf; j += 2) {
            const int col = col0 + j;
            if (col < Nr)
              *reinterpret_cast<float2*>(base + ((size_t)(col >> 1) * M + row) * 2) =
                  make_float2(acc[j], acc[j + 1]);
          }
        }
      } else if (ok) {  // warp-uniform: the staging below is collective
        // each thread holds one row of the tile; 16 columns at a time go
        // through this warp's shared-memory pitch so that a store covers 8 rows
        // x 64 contiguous bytes instead of 32 rows x 16 bytes
        float* stg = stage_out + (warp - 2) * (32 * C::kStgPitch);
        float* base = tk->out + ((size_t)split * tk->lt + t) * (size_t)M * Nr;
        const int row0 = mrow0 + q * 32, col0 = tn * kBN + c0;
        const bool vec = (Nr & 3) == 0;
        (void)row;
#pragma unroll
        for (int j = 0; j < kHalf; j += 16) {
          float4* w = reinterpret_cast<float4*>(stg + lane * C::kStgPitch);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            w[u] = make_float4(acc[j + 4 * u], acc[j + 4 * u + 1], acc[j + 4 * u + 2],
                               acc[j + 4 * u + 3]);
          __syncwarp();
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int rr = (lane >> 2) + 8 * p, cc = (lane & 3) * 4;
            const float4 v = *reinterpret_cast<const float4*>(stg + rr * C::kStgPitch + cc);
            const int orow = row0 + rr, col = col0 + j + cc;
            if (orow < M) {
              float* d = base + (size_t)orow * Nr + col;
              if (vec && col + 4 <= Nr) {
                *reinterpret_cast<float4*>(d) = v;
              } else {
                if (col < Nr) d[0] = v.x;
                if (col + 1 < Nr) d[1] = v.y;
                if (col + 2 < Nr) d[2] = v.z;
                if (col + 3 < Nr) d[3] = v.w;
              }
            }
          }
          __syncwarp();
        }
      }
    }
  } else if constexpr (FUSED) {
    // ---- converter warps: raw complex64 tiles -> hi/lo operand tiles
    const int ct = threadIdx.x - 32 * (2 + kDrainWarps);  // 0 .. 32*kConvWarps-1
    constexpr int kCT = 32 * kConvWarps;
    int g = 0, k = 0, local = 0, ok = 1;
    for (long long tile = tile0; tile < gp.total_tiles && ok; tile += tstep) {
      const GemmTask* tk = tile_task(gp, tile, k, local);
      for (int i = 0; i < tk->kblocks; ++i, ++g) {
        const int r = g % R, st = g % S;
        // the raw tile first: its loads overlap the wait for a free operand stage
        if (lane == 0) {
          if (!mbar_wait(&rfull[r], (uint32_t)(g / R) & 1u) || *abort_flag) {
            *abort_flag = 1;
            ok = 0;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        const uint8_t* rp = raw + r * C::kRawBytes;
        uint8_t* sp = smem + st * C::kStageBytes;
        // Every raw load of this thread's units is issued first (A: 16-byte
        // chunks, B: one complex k pair of one column each), then the splits
        // and stores: the loads overlap instead of one unit's round trip after
        // another.
        constexpr int NB = C::kBCols;                         // complex B columns staged
        constexpr int kUA = (C::kRawA / 16 + kCT - 1) / kCT;  // A units per thread
        constexpr int kUB = (NB * 8 + kCT - 1) / kCT;         // B units per thread
        static_assert(NB == 64 || NB == 32, "unit decode: 32 or 64 complex columns");
        constexpr int kNBlk = NB / 16, kCShift = NB == 64 ? 7 : 6;
        float4 va[kUA], vb[kUB];
        // A unit c: K-major tiles: the 16-byte chunk c, written to the same
        // place; in-place [k][rows] / [outer][k][inner] tiles: row n = c % 128
        // (outer block n / a_ni, inner row n % a_ni), complex k pair c / 128
        // (lanes on consecutive rows: contiguous loads, and the swizzled stores
        // of a quarter warp fall on 8 distinct chunk positions)
        const bool amn = AMN && tk->a_mn != 0;
        const float2* ra = reinterpret_cast<const float2*>(rp);
        if (amn) {  // warp-uniform (one task per tile): two copies of the loop
          const int ni = tk->a_ni, nsh = __ffs(ni) - 1;
#pragma unroll
          for (int j = 0; j < kUA; ++j) {
            const int c = ct + j * kCT;
            if (c < C::kRawA / 16) {
              const int n = c & (kBM - 1), kc2 = c / kBM;
              const int blk = ((n >> nsh) * 16 + 2 * kc2) * ni + (n & (ni - 1));
              const float2 v0 = ra[blk], v1 = ra[blk + ni];
              va[j] = make_float4(v0.x, v0.y, v1.x, v1.y);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < kUA; ++j) {
            const int c = ct + j * kCT;
            if (c < C::kRawA / 16) va[j] = *reinterpret_cast<const float4*>(rp + 16 * c);
          }
        }
        // B unit it -> (column n, chunk c).  [k][n] tiles: a warp takes 16
        // consecutive n at two chunks c, c ^ 1, a quarter warp four n at one
        // chunk and the next four at the other, so that a half warp's loads
        // fall on 16 distinct bank pairs and a quarter warp's swizzled B'
        // stores on 8 distinct chunk positions (no bank conflicts):
        // n = [3:0] + 16*[6:5], c = 2*[8:7] + ([2] ^ [4]) (32 columns, CTA
        // pairs: n = [3:0] + 16*[5], c = 2*[7:6] + ([2] ^ [4])).  K-major tiles:
        // n = it / 8, c = it % 8.
        const bool bmn = tk->b_mn != 0;  // [k][n] raw tile (3-d or 4-d map alike)
        const float2* rb = reinterpret_cast<const float2*>(rp + C::kRawA);
        auto unit = [&](int it, int& n, int& c) {
          if (bmn) {
            n = (it & 15) + 16 * ((it >> 5) & (kNBlk - 1));
            c = 2 * (it >> kCShift) + (((it >> 2) ^ (it >> 4)) & 1);
          } else {
            n = it >> 3;
            c = it & 7;
          }
        };
#pragma unroll
        for (int j = 0; j < kUB; ++j) {
          const int it = ct + j * kCT;
          if (it < NB * 8) {
            int n, c;
            unit(it, n, c);
            if (bmn) {  // complex (k, n) at k = 2c and 2c + 1
              const float2 v0 = rb[(2 * c) * NB + n], v1 = rb[(2 * c + 1) * NB + n];
              vb[j] = make_float4(v0.x, v0.y, v1.x, v1.y);
            } else {
              vb[j] = *reinterpret_cast<const float4*>(rp + C::kRawA + n * 128 + 16 * (c ^ (n & 7)));
            }
          }
        }
        // the raw tile is in registers now: its slot goes back to the TMA
        // producer before this warp's splits and stores, so that the next
        // loads start a conversion earlier (the arrive orders the warp's
        // loads before it)
        __syncwarp();
        if (lane == 0) mbar_arrive(&rempty[r]);
        if (lane == 0) {
          if (!mbar_wait(&empty[st], ((uint32_t)(g / S) & 1u) ^ 1u) || *abort_flag) {
            *abort_flag = 1;
            ok = 0;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        // A: K-major tiles keep their 128-byte-swizzled layout, element by
        // element; [k][rows] tiles go to row n, chunk kc2 ^ (n & 7)
        auto split_a = [&](int j, int o) {
          const float4 v = va[j];
          float h0, l0, h1, l1, h2, l2, h3, l3;
          Split<false>::split(v.x, h0, l0);
          Split<false>::split(v.y, h1, l1);
          Split<false>::split(v.z, h2, l2);
          Split<false>::split(v.w, h3, l3);
          *reinterpret_cast<float4*>(sp + o) = make_float4(h0, h1, h2, h3);
          *reinterpret_cast<float4*>(sp + C::kATile + o) = make_float4(l0, l1, l2, l3);
        };
        if (amn) {
#pragma unroll
          for (int j = 0; j < kUA; ++j) {
            const int c = ct + j * kCT;
            if (c >= C::kRawA / 16) continue;
            const int n = c & (kBM - 1), kc2 = c / kBM;
            split_a(j, n * 128 + 16 * (kc2 ^ (n & 7)));
          }
        } else {
#pragma unroll
          for (int j = 0; j < kUA; ++j) {
            const int c = ct + j * kCT;
            if (c >= C::kRawA / 16) continue;
            split_a(j, 16 * c);
          }
        }
        // B: complex column n -> B' rows 2n (re, -im) and 2n+1 (im, re); the
        // 16-byte chunk c (complex k 2c, 2c+1) of row r sits at chunk
        // c ^ (r & 7) (128-byte swizzle)
#pragma unroll
        for (int j = 0; j < kUB; ++j) {
          const int it = ct + j * kCT;
          if (it >= NB * 8) continue;
          int n, c;
          unit(it, n, c);
          const float4 v = vb[j];
          const int r0 = 2 * n, r1 = 2 * n + 1;
          const int o0 = r0 * 128 + 16 * (c ^ (r0 & 7)), o1 = r1 * 128 + 16 * (c ^ (r1 & 7));
          float h[4], l[4];
          Split<false>::split(v.x, h[0], l[0]);
          Split<false>::split(-v.y, h[1], l[1]);
          Split<false>::split(v.z, h[2], l[2]);
          Split<false>::split(-v.w, h[3], l[3]);
          uint8_t* bh = sp + 2 * C::kATile;
          uint8_t* bl = bh + C::kBTile;
          *reinterpret_cast<float4*>(bh + o0) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(bl + o0) = make_float4(l[0], l[1], l[2], l[3]);
          // row 2n+1 = (im, re): the same split parts, re-paired
          *reinterpret_cast<float4*>(bh + o1) = make_float4(-h[1], h[0], -h[3], h[2]);
          *reinterpret_cast<float4*>(bl + o1) = make_float4(-l[1], l[0], -l[3], l[2]);
        }
        // generic-proxy writes -> visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (PAIR && rank != 0) mbar_arrive_leader(&full[st]);  // CTA 0 issues the MMAs
          else mbar_arrive(&full[st]);
        }
      }
    }
  }
  // teardown: no MMA may still write TMEM when it is released (a pair: the
  // commit of CTA 0's last MMA arrives in both CTAs; neither CTA leaves while
  // the other may still arrive on its barriers or its MMAs read the peer)
  if (warp == 1 && lane == 0) {
    if (!mbar_wait(done, 0)) *abort_flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if constexpr (PAIR) cluster_sync_all();
  if (*abort_flag && threadIdx.x == 0) atomicCAS(&g_mixed_error, 0, 1);
  if (warp == 0) {
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(kTmemCols));
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(kTmemCols));
  }
}

// ------------------------------------------------------------ K4t: A in TMEM
// Fused TF32 split-3 GEMM whose A' hi/lo operands live in tensor memory.
// TMA brings raw complex64 tiles of A (128 rows) and B (64 complex columns)
// into a shared-memory ring (the maps of the fused form).  Four A-converter
// warps (one per TMEM lane quarter, one A' row per thread) read their row
// of the raw A tile, split it into hi/lo and write both into tensor memory
// with tcgen05.st; tcgen05.mma reads A from there and only B' from shared
// memory, where two B-converter warps build the hi/lo B' tiles.  Per k-block
// the MMA thread issues the two correction products (lo*hi, hi*lo) first,
// into a fresh accumulator, then hi*hi, and the drain warps add the
// finished accumulator into FP32 registers: four accumulations at full
// magnitude per drain.  Shared-memory traffic per k-block: raw A and B
// written and read (48 KB), B' hi/lo written (32 KB), B' read by the MMAs
// (48 KB) -- 128 KB against 208 KB when the A' planes are staged in shared
// memory as well (three MMAs read each of them).
struct TaCfg {
  static constexpr int kRawStages = 4;              // raw A + B ring
  static constexpr int kStages = 3;                 // B' operand ring
  static constexpr int kBTile = kBN * 128;          // one B' plane tile: kBN rows x 128 B
  static constexpr int kBStage = 2 * kBTile;        // hi + lo
  static constexpr int kRawA = kBM * 128;           // raw complex64 A tile (128-byte swizzle)
  static constexpr int kRawB = (kBN / 2) * 128;     // raw complex64 B tile
  static constexpr int kRaw = kRawA + kRawB;
  static constexpr int kAConv = 4, kBConv = 2;      // converter warps
  static constexpr int kThreads = 64 + 32 * (kDrainWarps + kAConv + kBConv);
  static constexpr int kStgPitch = 20;
  static constexpr int kStgBytes = kDrainWarps * 32 * kStgPitch * 4;
  static constexpr int kSmem = kStages * kBStage + kRawStages * kRaw + 1024 + 256 + kStgBytes;
  static constexpr int kACol = 2 * kBN;             // TMEM: [0, 2 kBN) accumulators, then A
  static constexpr int kTmemCols = 512;
};
static_assert(TaCfg::kACol + 2 * 64 <= TaCfg::kTmemCols, "A stages must fit in TMEM");
static_assert(TaCfg::kThreads == 512, "warp roles: 2 + 8 drain + 4 A + 2 B converters");

__device__ __forceinline__ void umma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                        uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

__global__ void __launch_bounds__(TaCfg::kThreads, 1)
k_gemm_tf32_tmem_a(const __grid_constant__ GemmParams gp) {
  using C = TaCfg;
  constexpr int S = C::kStages, R = C::kRawStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* raw = smem + S * C::kBStage;  // raw complex64 ring: A tile, then B tile
  uint64_t* bfull = reinterpret_cast<uint64_t*>(raw + R * C::kRaw);  // [S] B' stage built
  uint64_t* bempty = bfull + S;        // [S] B' stage read by its MMAs
  uint64_t* rfull = bempty + S;        // [R] raw A + B landed
  uint64_t* rempty = rfull + R;        // [R] raw A and B read by the converters
  uint64_t* afull = rempty + R;        // [2] A stage written to TMEM
  uint64_t* aempty = afull + 2;        // [2] A stage read by its MMAs
  uint64_t* tfull = aempty + 2;        // [2] accumulator ready to drain
  uint64_t* tempty = tfull + 2;        // [2] accumulator drained
  uint64_t* done = tempty + 2;         // every MMA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* stage_out = reinterpret_cast<float*>(raw + R * C::kRaw + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kAWarp0 = 2 + kDrainWarps, kBWarp0 = kAWarp0 + C::kAConv;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&bfull[i], C::kBConv);
      mbar_init(&bempty[i], 1);
    }
    for (int i = 0; i < R; ++i) {
      mbar_init(&rfull[i], 1);
      mbar_init(&rempty[i], C::kAConv + C::kBConv);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], C::kAConv);
      mbar_init(&aempty[b], 1);
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kDrainWarps);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer: raw A and B tiles
      int g = 0, issued = 0, k = 0, local = 0;
      bool stop = false;
      for (long long tile = blockIdx.x; tile < gp.total_tiles && !stop; tile += gridDim.x) {
        const GemmTask* tk = tile_task(gp, tile, k, local);
        const int tn = local % tk->ntn, tm = (local / tk->ntn) % tk->ntm;
        const int z = local / (tk->ntn * tk->ntm);
        const int t = z % tk->lt, split = z / tk->lt;
        const int n0 = tn * kBN, m0 = tm * kBM, kb0 = split * tk->kblocks;
        for (int i = 0; i < tk->kblocks; ++i, ++g) {
          const int st = g % R;
          if (!mbar_wait(&rempty[st], ((uint32_t)(g / R) & 1u) ^ 1u) || *abort_flag) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          const int k0 = (kb0 + i) * 32;  // floats
          uint8_t* ra = raw + st * C::kRaw;
          uint8_t* rp = ra + C::kRawA;
          mbar_expect_tx(&rfull[st], C::kRaw);
          tma_load_3d(ra, &tk->map[0], &rfull[st], k0, m0, t);
          if (tk->b_mn == 2) {  // the same tile inside one block of every outer axis
            int c[5], nd = 0, kk = k0 / 2;
            c[nd++] = n0 % (2 * tk->b_ni);
            for (int a = 0; a < tk->b_nk; ++a) {
              c[nd++] = kk % tk->b_kext[a];
              kk /= tk->b_kext[a];
            }
            if (tk->b_no) c[nd++] = n0 / (2 * tk->b_ni);
            c[nd++] = t;
            if (nd == 3) tma_load_3d(rp, &tk->map[2], &rfull[st], c[0], c[1], c[2]);
            else if (nd == 4)
              tma_load_4d(rp, &tk->map[2], &rfull[st], c[0], c[1], c[2], c[3]);
            else
              tma_load_5d(rp, &tk->map[2], &rfull[st], c[0], c[1], c[2], c[3], c[4]);
          } else if (tk->b_mn) {  // [16 complex k rows][kBN/2 complex n], unswizzled
            tma_load_3d(rp, &tk->map[2], &rfull[st], n0, k0 / 2, t);
          } else {
            tma_load_3d(rp, &tk->map[2], &rfull[st], k0, n0 / 2, t);
          }
          issued = g + 1;
        }
      }
      // every issued load must have landed before the CTA exits
      for (int i = (issued > R ? issued - R : 0); i < issued; ++i)
        if (!mbar_wait(&rfull[i % R], (uint32_t)(i / R) & 1u)) break;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: A from TMEM, B' from shared memory
      constexpr uint32_t idesc = make_idesc<false>();
      int g = 0, k = 0, local = 0;
      bool stop = false;
      for (long long tile = blockIdx.x; tile < gp.total_tiles && !stop; tile += gridDim.x) {
        const GemmTask* tk = tile_task(gp, tile, k, local);
        for (int i = 0; i < tk->kblocks; ++i, ++g) {
          const int b = g & 1, st = g % S;
          const uint32_t ph2 = (uint32_t)(g >> 1) & 1u;
          if (!mbar_wait(&tempty[b], ph2 ^ 1u) || !mbar_wait(&afull[b], ph2) ||
              !mbar_wait(&bfull[st], (uint32_t)(g / S) & 1u) || *abort_flag) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t bhi = smem_u32(smem + st * C::kBStage), blo = bhi + C::kBTile;
          const uint32_t d = tmem + (uint32_t)(b * kBN);
          const uint32_t ahi = tmem + (uint32_t)(C::kACol + b * 64), alo = ahi + 32;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)  // corrections first, into a fresh accumulator
            umma_ta(d, alo + kk * 8, sdesc_sw128(bhi + kk * 32), idesc, kk > 0 ? 1u : 0u);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            umma_ta(d, ahi + kk * 8, sdesc_sw128(blo + kk * 32), idesc, 1u);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            umma_ta(d, ahi + kk * 8, sdesc_sw128(bhi + kk * 32), idesc, 1u);
          umma_commit(&bempty[st]);
          umma_commit(&aempty[b]);
          umma_commit(&tfull[b]);
        }
      }
      umma_commit(done);
    }
  } else if (warp < 2 + kDrainWarps) {
    // ---- drain / epilogue warps: one accumulator per k-block
    constexpr int kHalf = kBN / 2;
    const int q = warp & 3;
    const int c0 = ((warp - 2) >> 2) * kHalf;
    const uint32_t tlane = ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
    int g = 0, ok = 1, k = 0, local = 0;
    for (long long tile = blockIdx.x; tile < gp.total_tiles && ok; tile += gridDim.x) {
      const GemmTask* tk = tile_task(gp, tile, k, local);
      const int tn = local % tk->ntn, tm = (local / tk->ntn) % tk->ntm;
      const int z = local / (tk->ntn * tk->ntm);
      const int t = z % tk->lt, split = z / tk->lt;
      const int M = tk->M, Nr = tk->Nr;
      float acc[kHalf];
#pragma unroll
      for (int j = 0; j < kHalf; ++j) acc[j] = 0.f;
      for (int i = 0; i < tk->kblocks; ++i, ++g) {
        const int b = g & 1;
        if (lane == 0) {
          if (!mbar_wait(&tfull[b], (uint32_t)(g >> 1) & 1u) || *abort_flag) {
            *abort_flag = 1;
            ok = 0;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tb = tmem + tlane + (uint32_t)(b * kBN);
#pragma unroll
        for (int j = 0; j < kHalf; j += 32) {
          uint32_t r[16], r2[16];
          tmem_ld16_pair(tb + j, tb + j + 16, r, r2);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            acc[j + u] += __uint_as_float(r[u]);
            acc[j + 16 + u] += __uint_as_float(r2[u]);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
      if (ok) {  // warp-uniform: the staging below is collective
        float* stg = stage_out + (warp - 2) * (32 * C::kStgPitch);
        float* base = tk->out + ((size_t)split * tk->lt + t) * (size_t)M * Nr;
        const int row0 = tm * kBM + q * 32, col0 = tn * kBN + c0;
        const bool vec = (Nr & 3) == 0;
#pragma unroll
        for (int j = 0; j < kHalf; j += 16) {
          float4* w = reinterpret_cast<float4*>(stg + lane * C::kStgPitch);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            w[u] = make_float4(acc[j + 4 * u], acc[j + 4 * u + 1], acc[j + 4 * u + 2],
                               acc[j + 4 * u + 3]);
          __syncwarp();
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int rr = (lane >> 2) + 8 * p, cc = (lane & 3) * 4;
            const float4 v = *reinterpret_cast<const float4*>(stg + rr * C::kStgPitch + cc);
            const int orow = row0 + rr, col = col0 + j + cc;
            if (orow < M) {
              float* dst = base + (size_t)orow * Nr + col;
              if (vec && col + 4 <= Nr) {
                *reinterpret_cast<float4*>(dst) = v;
              } else {
                if (col < Nr) dst[0] = v.x;
                if (col + 1 < Nr) dst[1] = v.y;
                if (col + 2 < Nr) dst[2] = v.z;
                if (col + 3 < Nr) dst[3] = v.w;
              }
            }
          }
          __syncwarp();
        }
      }
    }
  } else if (warp < kBWarp0) {
    // ---- A converters: this thread's row of the raw A tile -> hi/lo A' row in TMEM
    const int q = warp & 3, r = q * 32 + lane;  // the row = the TMEM lane it writes
    const uint32_t ta0 = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)C::kACol;
    int g = 0, k = 0, local = 0, ok = 1;
    for (long long tile = blockIdx.x; tile < gp.total_tiles && ok; tile += gridDim.x) {
      const GemmTask* tk = tile_task(gp, tile, k, local);
      for (int i = 0; i < tk->kblocks; ++i, ++g) {
        const int st = g % R, s = g & 1;
        if (lane == 0) {
          if (!mbar_wait(&rfull[st], (uint32_t)(g / R) & 1u) || *abort_flag) {
            *abort_flag = 1;
            ok = 0;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        // chunk c of row r sits at chunk c ^ (r & 7): a quarter-warp's 16-byte
        // reads (8 rows) cover all 32 banks
        const uint8_t* ra = raw + st * C::kRaw + r * 128;
        float4 v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = *reinterpret_cast<const float4*>(ra + 16 * (c ^ (r & 7)));
        __syncwarp();
        if (lane == 0) mbar_arrive(&rempty[st]);
        if (lane == 0) {
          if (!mbar_wait(&aempty[s], ((uint32_t)(g >> 1) & 1u) ^ 1u) || *abort_flag) {
            *abort_flag = 1;
            ok = 0;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        const uint32_t ta = ta0 + (uint32_t)(s * 64);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float h[16], l[16];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 x = v[half * 4 + u];
            Split<false>::split(x.x, h[4 * u], l[4 * u]);
            Split<false>::split(x.y, h[4 * u + 1], l[4 * u + 1]);
            Split<false>::split(x.z, h[4 * u + 2], l[4 * u + 2]);
            Split<false>::split(x.w, h[4 * u + 3], l[4 * u + 3]);
          }
          tmem_st16(ta + (uint32_t)(half * 16), h);
          tmem_st16(ta + 32u + (uint32_t)(half * 16), l);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&afull[s]);
      }
    }
  } else {
    // ---- B converters: raw complex64 B tiles -> hi/lo B' tiles in shared memory
    const int ct = threadIdx.x - 32 * kBWarp0;  // 0 .. 32*kBConv-1
    constexpr int kCT = 32 * C::kBConv;
    constexpr int kUB = ((kBN / 2) * 8 + kCT - 1) / kCT;  // B units per thread
    static_assert(kBN / 2 == 64, "unit decode assumes 64 complex columns per tile");
    int g = 0, k = 0, local = 0, ok = 1;
    for (long long tile = blockIdx.x; tile < gp.total_tiles && ok; tile += gridDim.x) {
      const GemmTask* tk = tile_task(gp, tile, k, local);
      const bool bmn = tk->b_mn != 0;  // [k][n] raw tile (3-d, 4-d or 5-d map alike)
      for (int i = 0; i < tk->kblocks; ++i, ++g) {
        const int st = g % S, rs = g % R;
        const uint32_t ph = (uint32_t)(g / S) & 1u;
        if (lane == 0) {
          if (!mbar_wait(&rfull[rs], (uint32_t)(g / R) & 1u) || *abort_flag) {
            *abort_flag = 1;
            ok = 0;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        const uint8_t* rp = raw + rs * C::kRaw + C::kRawA;
        const float2* rb = reinterpret_cast<const float2*>(rp);
        float4 vb[kUB];
        // unit it -> (column n, chunk c): [k][n] tiles: a warp takes 16
        // consecutive n at two chunks c, c ^ 1, alternating every four lanes
        // (conflict-free loads and stores); K-major tiles: n = it / 8
#pragma unroll
        for (int j = 0; j < kUB; ++j) {
          const int it = ct + j * kCT;
          if (it < (kBN / 2) * 8) {
            int n, c;
            if (bmn) {
              n = (it & 15) + 16 * ((it >> 5) & 3);
              c = 2 * (it >> 7) + (((it >> 2) ^ (it >> 4)) & 1);
              const float2 v0 = rb[(2 * c) * (kBN / 2) + n], v1 = rb[(2 * c + 1) * (kBN / 2) + n];
              vb[j] = make_float4(v0.x, v0.y, v1.x, v1.y);
            } else {
              n = it >> 3;
              c = it & 7;
              vb[j] = *reinterpret_cast<const float4*>(rp + n * 128 + 16 * (c ^ (n & 7)));
            }
          }
        }
        if (lane == 0) {
          if (!mbar_wait(&bempty[st], ph ^ 1u) || *abort_flag) {
            *abort_flag = 1;
            ok = 0;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        uint8_t* bh = smem + st * C::kBStage;
        uint8_t* bl = bh + C::kBTile;
#pragma unroll
        for (int j = 0; j < kUB; ++j) {
          const int it = ct + j * kCT;
          if (it >= (kBN / 2) * 8) continue;
          int n, c;
          if (bmn) {
            n = (it & 15) + 16 * ((it >> 5) & 3);
            c = 2 * (it >> 7) + (((it >> 2) ^ (it >> 4)) & 1);
          } else {
            n = it >> 3;
            c = it & 7;
          }
          // complex column n -> B' rows 2n (re, -im) and 2n+1 (im, re); the
          // 16-byte chunk c of row r sits at chunk c ^ (r & 7) (128-byte swizzle)
          const float4 v = vb[j];
          const int r0 = 2 * n, r1 = 2 * n + 1;
          const int o0 = r0 * 128 + 16 * (c ^ (r0 & 7)), o1 = r1 * 128 + 16 * (c ^ (r1 & 7));
          float h[4], l[4];
          Split<false>::split(v.x, h[0], l[0]);
          Split<false>::split(-v.y, h[1], l[1]);
          Split<false>::split(v.z, h[2], l[2]);
          Split<false>::split(-v.w, h[3], l[3]);
          *reinterpret_cast<float4*>(bh + o0) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(bl + o0) = make_float4(l[0], l[1], l[2], l[3]);
          *reinterpret_cast<float4*>(bh + o1) = make_float4(-h[1], h[0], -h[3], h[2]);
          *reinterpret_cast<float4*>(bl + o1) = make_float4(-l[1], l[0], -l[3], l[2]);
        }
        // generic-proxy writes -> visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&bfull[st]);
          mbar_arrive(&rempty[rs]);
        }
      }
    }
  }
  // teardown: no MMA may still write TMEM when it is released
  if (warp == 1 && lane == 0) {
    if (!mbar_wait(done, 0)) *abort_flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicCAS(&g_mixed_error, 0, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::kTmemCols));
}

// K4r: out c64 [lt][M][N] = sum over splits of the FP32 partials
// The k-split partials of one output element summed in double-float (Knuth's
// TwoSum per partial, the rounding errors gathered apart) and rounded once to
// FP32: the correctly rounded sum but for rare ties, with FP32 arithmetic
// (B300 issues FP64 at a small fraction of its FP32 rate).
__device__ __forceinline__ float sum_splits(const float* __restrict__ p, long long stride, int n) {
  float h = 0.f, l = 0.f;
  for (int k = 0; k < n; ++k) {
    const float x = p[(long long)k * stride];
    const float t = __fadd_rn(h, x);
    const float bp = __fsub_rn(t, h);
    l = __fadd_rn(l, __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
    h = t;
  }
  return __fadd_rn(h, l);
}

__global__ void k_reduce_splits(const float* __restrict__ part, float* __restrict__ out,
                                long long per_split, int splits) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < per_split;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = sum_splits(part + i, per_split, splits);
}

// ------------------------------------------------------------ K3 pack
__device__ __forceinline__ long long goff(const Group& g, unsigned idx) {
  long long off = 0;
#pragma unroll
  for (int d = LQC_MAX_RANK - 1; d >= 0; --d) {
    if (d < g.n) {
      unsigned e = (unsigned)g.ext[d];
      unsigned q = idx / e;
      off += (long long)(idx - q * e) * g.stride[d];
      idx = q;
    }
  }
  return off;
}

template <bool BF16>
struct PackPair {
  PackArgs op[2];                          // [0] A operand, [1] B operand
  const float2* X[2];
  typename Split<BF16>::T* hi[2];
  typename Split<BF16>::T* lo[2];
  int lt;
};

// Both operands of one contraction in one launch (grid.z = 2 * lt).  One 32
// (rows) x 32 (complex k) block per CTA through shared memory, so that both
// the gather (along the operand's unit-stride axis) and the plane writes
// (along k) are coalesced.
template <bool BF16>
__device__ __forceinline__ void pack_block(const PackArgs& p, const float2* __restrict__ X,
                                           typename Split<BF16>::T* __restrict__ hi,
                                           typename Split<BF16>::T* __restrict__ lo, int t,
                                           unsigned r0, unsigned k0);

template <bool BF16>
__global__ void __launch_bounds__(256)
k_pack(const __grid_constant__ PackPair<BF16> pp) {
  const int which = blockIdx.z >= (unsigned)pp.lt ? 1 : 0;
  const int t = blockIdx.z - which * pp.lt;
  const PackArgs& p = pp.op[which];
  const unsigned r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  if (r0 >= (unsigned)p.rows) return;  // the grid spans the larger operand
  pack_block<BF16>(p, pp.X[which], pp.hi[which], pp.lo[which], t, r0, k0);
}

// one 32 x 32 block of one operand (see k_pack)
template <bool BF16>
__device__ __forceinline__ void pack_block(const PackArgs& p, const float2* __restrict__ X,
                                           typename Split<BF16>::T* __restrict__ hi,
                                           typename Split<BF16>::T* __restrict__ lo, int t,
                                           unsigned r0, unsigned k0) {
  typedef typename Split<BF16>::T T;
  __shared__ float2 tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  X += (long long)t * p.ts;
  // the index decompositions of this block's 32 rows and 32 k once, not per element
  __shared__ long long roff[32], koff[32];
  if (threadIdx.x < 32) {
    const unsigned r = r0 + threadIdx.x;
    roff[threadIdx.x] = r < (unsigned)p.rows ? goff(p.rg, r) : 0;
  } else if (threadIdx.x < 64) {
    const unsigned k = k0 + threadIdx.x - 32;
    koff[threadIdx.x - 32] = k < (unsigned)p.K ? goff(p.kg, k) : 0;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    unsigned r, k;
    if (p.k_fast) { k = k0 + tx; r = r0 + ty + 8 * j; }
    else { r = r0 + tx; k = k0 + ty + 8 * j; }
    float2 v = make_float2(0.f, 0.f);
    if (r < (unsigned)p.rows && k < (unsigned)p.K) v = X[roff[r - r0] + koff[k - k0]];
    tile[r - r0][k - k0] = v;
  }
  __syncthreads();
  const size_t plane_rows = p.which == 0 ? (size_t)p.rows : 2 * (size_t)p.rows;
  T* Hb = hi + (size_t)t * plane_rows * p.kp;
  T* Lb = lo + (size_t)t * plane_rows * p.kp;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const unsigned r = r0 + ty + 8 * j, k = k0 + tx;
    if (r >= (unsigned)p.rows || 2 * k >= (unsigned)p.kp) continue;
    const float2 v = tile[r - r0][k - k0];  // zero beyond K: fills the padding
    T hr, lr, hi_, li;
    Split<BF16>::split(v.x, hr, lr);
    Split<BF16>::split(v.y, hi_, li);
    if (p.which == 0) {
      Split<BF16>::store2(Hb + (size_t)r * p.kp + 2 * k, hr, hi_);
      Split<BF16>::store2(Lb + (size_t)r * p.kp + 2 * k, lr, li);
    } else {
      T hni, lni;  // -Im
      Split<BF16>::split(-v.y, hni, lni);
      Split<BF16>::store2(Hb + (size_t)(2 * r) * p.kp + 2 * k, hr, hni);
      Split<BF16>::store2(Lb + (size_t)(2 * r) * p.kp + 2 * k, lr, lni);
      Split<BF16>::store2(Hb + (size_t)(2 * r + 1) * p.kp + 2 * k, hi_, hr);
      Split<BF16>::store2(Lb + (size_t)(2 * r + 1) * p.kp + 2 * k, li, lr);
    }
  }
}

// ------------------------------------------------------------ K2m
// (sh, sl) += a * b without rounding loss: the product's exact error from an
// FMA and Knuth's TwoSum for the addition; the _rn intrinsics keep the
// compiler from contracting these steps into other FMAs.
__device__ __forceinline__ void df_acc_prod(float& sh, float& sl, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(sh, p);
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}
// (h, l) += (h2, l2) for double-float values: Knuth's TwoSum of the high
// parts, the low parts and the rounding error added to the low part
__device__ __forceinline__ void df_add(float& h, float& l, float h2, float l2) {
  const float t = __fadd_rn(h, h2);
  const float bp = __fsub_rn(t, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(h2, bp));
  h = t;
  l = __fadd_rn(l, __fadd_rn(err, l2));
}
// ------------------------------------------------------------ permute
// A PermDesc maps every element e of a destination order (row-major over its
// axes) to a source offset.  Two block shapes move it with coalesced reads
// and writes, and serve both the reorder copies and the correlator sums
// (which multiply instead of storing, so a partner is never copied):
//  * runs (mode 0): the destination's innermost axis X is unit-stride in the
//    source too.  A block takes kPermElems consecutive destination elements;
//    the source offsets of the runs it touches are computed once into
//    shared memory (32-bit index arithmetic: slices below 2^31 elements).
//  * tiles (mode 1): the source's unit-stride axis Y is another axis.  A
//    block takes kPermTiles 32x32 tiles (X by Y) of one outer index, all
//    loaded along Y before one barrier, then used along X.
constexpr int kPermElems = 2048;
constexpr int kPermTiles = 4;
constexpr int kPermSmem = kPermTiles * 32 * 33 * 8;  // >= (kPermElems + 1) * 4

// source and destination offsets of outer index o (row-major digits)
__device__ __forceinline__ unsigned perm_outer(const PermDesc& d, unsigned o, unsigned* dso) {
  unsigned so = 0, ds = 0;
#pragma unroll
  for (int a = LQC_MAX_RANK - 1; a >= 0; --a) {
    if (a < d.nout) {
      const unsigned e = (unsigned)d.oext[a];
      const unsigned q = o / e;
      const unsigned r = o - q * e;
      so += r * (unsigned)d.osrc[a];
      ds += r * (unsigned)d.odst[a];
      o = q;
    }
  }
  *dso = ds;
  return so;
}

// calls op(e, src value, pre(e)) for the elements of block b (one slice);
// pre(e) is issued for every element before the block's barrier, so its
// loads overlap the source loads (a correlator's left operand)
template <typename Pre, typename Op>
__device__ __forceinline__ void perm_visit(const PermDesc& d, const float2* __restrict__ src,
                                           unsigned b, unsigned char* smem, Pre pre, Op op) {
  if (d.mode == 0) {
    constexpr int J = kPermElems / 256;
    unsigned* so_tab = reinterpret_cast<unsigned*>(smem);
    const unsigned X = (unsigned)d.X;
    const unsigned e0 = b * kPermElems;
    const unsigned e1 = min(e0 + (unsigned)kPermElems, (unsigned)d.n);
    const unsigned r0 = e0 / X, r1 = (e1 - 1) / X;
    float2 pv[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const unsigned e = e0 + j * 256 + threadIdx.x;
      pv[j] = e < e1 ? pre(e) : make_float2(0.f, 0.f);
    }
    unsigned dummy;
    for (unsigned r = r0 + threadIdx.x; r <= r1; r += blockDim.x)
      so_tab[r - r0] = perm_outer(d, r, &dummy);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const unsigned e = e0 + j * 256 + threadIdx.x;
      if (e < e1) {
        const unsigned r = e / X;
        op(e, src[so_tab[r - r0] + (e - r * X)], pv[j]);
      }
    }
    return;
  }
  float2 (*tile)[32][33] = reinterpret_cast<float2 (*)[32][33]>(smem);
  const unsigned xb = ((unsigned)d.X + 31) / 32;
  const unsigned ygb = (((unsigned)d.Y + 31) / 32 + kPermTiles - 1) / kPermTiles;
  const unsigned o = b / (xb * ygb), rem = b - o * (xb * ygb);
  const unsigned x0 = (rem % xb) * 32, yg = rem / xb;
  unsigned dso;
  const unsigned so = perm_outer(d, o, &dso);
  const unsigned tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const unsigned sX = (unsigned)d.sX, dY = (unsigned)d.dY;
  const unsigned X = (unsigned)d.X, Y = (unsigned)d.Y;
  float2 pv[kPermTiles][4];
#pragma unroll
  for (int q = 0; q < kPermTiles; ++q) {  // destination-order operand, along X
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned x = x0 + tx, y = (yg * kPermTiles + q) * 32 + ty + 8 * j;
      pv[q][j] = (y < Y && x < X) ? pre(dso + y * dY + x) : make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int q = 0; q < kPermTiles; ++q) {  // source, along its unit-stride axis Y
    const unsigned y = (yg * kPermTiles + q) * 32 + tx;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned x = x0 + ty + 8 * j;
      if (y < Y && x < X) tile[q][ty + 8 * j][tx] = src[so + y + x * sX];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kPermTiles; ++q) {  // along the destination's unit-stride axis X
    const unsigned x = x0 + tx;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned y = (yg * kPermTiles + q) * 32 + ty + 8 * j;
      if (y < Y && x < X) op(dso + y * dY + x, tile[q][tx][ty + 8 * j], pv[q][j]);
    }
  }
}

__device__ __forceinline__ void permute_block(const PermDesc& d, const float2* __restrict__ src,
                                              float2* __restrict__ dst, int t, long long b) {
  __shared__ __align__(16) unsigned char smem[kPermSmem];
  src += (long long)t * d.src_ts;
  dst += (long long)t * d.n;
  perm_visit(
      d, src, (unsigned)b, smem, [](unsigned) { return make_float2(0.f, 0.f); },
      [&](unsigned e, float2 v, float2) { dst[e] = v; });
}

__global__ void __launch_bounds__(256)
k_permute_c64(const float2* __restrict__ src, float2* __restrict__ dst, const PermDesc d) {
  permute_block(d, src, dst, blockIdx.y, blockIdx.x);
}

// partial sum of block b of slice t of one correlator, r(t) = sum_e A[e] *
// B[src(e)] with the destination order of `d` = the left operand's order;
// fixed reduction order, so every launch form gives the same bits.  Runs
// (mode 0) go through perm_visit; transposed pairs (mode 1) without shared
// memory: each warp sums one 32x32 tile, A read along X (coalesced), B
// along its unit-stride axis Y per lane (each lane's lines stay in L1
// across the tile's 32 rows), kCaWarpTiles tiles per block.
constexpr int kCaWarpTiles = 8;

__device__ __forceinline__ void ca_acc(float& rh, float& rl, float& ih, float& il, float2 a,
                                       float2 bv) {
  df_acc_prod(rh, rl, a.x, bv.x);
  df_acc_prod(rh, rl, -a.y, bv.y);
  df_acc_prod(ih, il, a.x, bv.y);
  df_acc_prod(ih, il, a.y, bv.x);
}

__device__ __forceinline__ void ca_partial_block(const float2* __restrict__ A,
                                                 const float2* __restrict__ B,
                                                 double2* __restrict__ part, const PermDesc& d,
                                                 long long t, unsigned b) {
  __shared__ __align__(16) unsigned char smem[(kPermElems + 1) * 4];
  A += t * d.n;
  B += t * d.src_ts;
  // per thread and across the block: double-float sums (exact FP32 products,
  // TwoSum accumulation, ~44 significant bits) at FP32 throughput; across
  // blocks: FP64
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  if (d.mode == 0) {
    perm_visit(d, B, b, smem, [&](unsigned e) { return A[e]; },
               [&](unsigned, float2 bv, float2 a) { ca_acc(rh, rl, ih, il, a, bv); });
  } else {
    const unsigned X = (unsigned)d.X, Y = (unsigned)d.Y;
    const unsigned xb = (X + 31) / 32, yb = (Y + 31) / 32;
    const unsigned tile = b * kCaWarpTiles + (threadIdx.x >> 5);
    const unsigned lane = threadIdx.x & 31;
    if (tile < (unsigned)d.outer * xb * yb) {
      const unsigned o = tile / (xb * yb), rem = tile - o * (xb * yb);
      const unsigned x = (rem % xb) * 32 + lane, y0 = (rem / xb) * 32;
      unsigned dso;
      const unsigned so = perm_outer(d, o, &dso);
      if (x < X) {
        const float2* a = A + dso + x;
        const float2* bp = B + so + x * (unsigned)d.sX;
        const unsigned dY = (unsigned)d.dY;
        const unsigned ny = min(32u, Y - y0);
        if (((so | (unsigned)d.sX) & 1u) == 0 && (ny & 1u) == 0) {
          // B 16-byte aligned along y (y0 is a multiple of 32): two complex
          // values per load, the same summation order
#pragma unroll 4
          for (unsigned yy = 0; yy < ny; yy += 2) {
            const unsigned y = y0 + yy;
            const float4 b2 = *reinterpret_cast<const float4*>(bp + y);
            ca_acc(rh, rl, ih, il, a[y * dY], make_float2(b2.x, b2.y));
            ca_acc(rh, rl, ih, il, a[(y + 1) * dY], make_float2(b2.z, b2.w));
          }
        } else {
#pragma unroll 8
          for (unsigned yy = 0; yy < ny; ++yy) {
            const unsigned y = y0 + yy;
            ca_acc(rh, rl, ih, il, a[y * dY], bp[y]);
          }
        }
      }
    }
  }
  // block sum in double-float as well (FP32 shuffles and TwoSum adds; B300
  // issues FP64 at a small fraction of the FP32 rate), FP64 once per block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h1 = __shfl_down_sync(0xffffffffu, rh, o), l1 = __shfl_down_sync(0xffffffffu, rl, o);
    const float h2 = __shfl_down_sync(0xffffffffu, ih, o), l2 = __shfl_down_sync(0xffffffffu, il, o);
    df_add(rh, rl, h1, l1);
    df_add(ih, il, h2, l2);
  }
  __shared__ float4 w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = make_float4(rh, rl, ih, il);
  __syncthreads();
  if (threadIdx.x < 32) {
    const float4 v = threadIdx.x < 8 ? w[threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
    rh = v.x;
    rl = v.y;
    ih = v.z;
    il = v.w;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      const float h1 = __shfl_down_sync(0xffffffffu, rh, o), l1 = __shfl_down_sync(0xffffffffu, rl, o);
      const float h2 = __shfl_down_sync(0xffffffffu, ih, o), l2 = __shfl_down_sync(0xffffffffu, il, o);
      df_add(rh, rl, h1, l1);
      df_add(ih, il, h2, l2);
    }
    if (threadIdx.x == 0)
      part[t * d.blocks + b] = make_double2((double)rh + (double)rl, (double)ih + (double)il);
  }
}

__global__ void __launch_bounds__(256)
k_contract_all_c64(const float2* __restrict__ A, const float2* __restrict__ B,
                   double2* __restrict__ part, const PermDesc d) {
  ca_partial_block(A, B, part, d, blockIdx.y, blockIdx.x);
}

__global__ void k_contract_all_final_scaled(const double2* __restrict__ part,
                                            double2* __restrict__ C, long long lt, int chunks,
                                            double scale) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= lt) return;
  double2 s = make_double2(0.0, 0.0);
  for (int c = 0; c < chunks; ++c) {
    double2 v = part[t * chunks + c];
    s.x += v.x;
    s.y += v.y;
  }
  C[t] = make_double2(s.x * scale, s.y * scale);
}

// ------------------------------------------------------------ grouped
// One level of a grouped window: independent contractions run together, a
// handful of launches per level instead of a few per contraction.  Every
// launch walks a task table in global memory; a block finds its task by
// binary search over the tasks' first block index.
struct PackTask {  // one operand; identical operands of a level are packed once
  PackArgs op;
  const float2* X;
  void* hi;
  void* lo;
  int kblk, rblk;
  long long block_start;
};

struct CATask {
  const float2* A;
  const float2* B;
  double2* out;
  double2* part;
  PermDesc d;            // B in A's order; d.blocks partial sums per slice
  double scale;
  long long t_start;
};

// The blocks of a grouped correlator launch walk segments of consecutive
// slices (about kCaChunkElems elements of the left operand each) in
// chunk-major order, the tasks that share an operand adjacent: the
// correlators of a level often share a tensor (a leaf), whose chunk is then
// read from DRAM once and from L2 by the others, while each segment still
// streams megabytes of contiguous data.  A block's partial sum does not
// depend on the order.
constexpr long long kCaChunkElems = 1ll << 19;
struct CASeg {
  int task, t0;  // slices t0, t0 + 1, ... (d.blocks blocks each)
};

struct PermTask {
  PermDesc d;
  const float2* src;
  float2* dst;
  long long block_start;
};

struct ReduceTask {
  const float* part;
  float* out;
  long long per;
  int splits;
  long long block_start;
};

constexpr int kReduceElems = 2048;  // elements per block of the grouped reduction

// task owning block b: binary search over the contiguous first-block array
// (a few cache lines, shared by every block of the launch)
__device__ __forceinline__ int find_task(const long long* __restrict__ starts, int n,
                                         long long b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(starts + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <bool BF16>
__global__ void __launch_bounds__(256)
k_pack_grouped(const PackTask* __restrict__ tasks, const long long* __restrict__ starts,
               int n) {
  typedef typename Split<BF16>::T T;
  const PackTask& tk = tasks[find_task(starts, n, blockIdx.x)];
  const long long local = blockIdx.x - tk.block_start;
  const int bx = (int)(local % tk.kblk), by = (int)((local / tk.kblk) % tk.rblk);
  const int t = (int)(local / ((long long)tk.kblk * tk.rblk));
  pack_block<BF16>(tk.op, tk.X, static_cast<T*>(tk.hi), static_cast<T*>(tk.lo), t, by * 32,
                   bx * 32);
}

__global__ void __launch_bounds__(256)
k_permute_grouped(const PermTask* __restrict__ tasks, const long long* __restrict__ starts,
                  int n) {
  const PermTask& tk = tasks[find_task(starts, n, blockIdx.x)];
  const long long local = blockIdx.x - tk.block_start;
  permute_block(tk.d, tk.src, tk.dst, (int)(local / tk.d.blocks), local % tk.d.blocks);
}

__global__ void __launch_bounds__(256)
k_contract_all_grouped(const CATask* __restrict__ tasks, const long long* __restrict__ starts,
                       const CASeg* __restrict__ segs, int n) {
  const int s = find_task(starts, n, blockIdx.x);
  const CASeg sg = segs[s];
  const CATask& tk = tasks[sg.task];
  const unsigned local = (unsigned)(blockIdx.x - __ldg(starts + s)), nb = (unsigned)tk.d.blocks;
  ca_partial_block(tk.A, tk.B, tk.part, tk.d, sg.t0 + local / nb, local % nb);
}

__global__ void k_contract_all_final_grouped(const CATask* __restrict__ tasks, int n,
                                             long long total) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = n - 1;  // task owning slice g (by t_start)
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].t_start <= g) lo = mid;
    else hi = mid - 1;
  }
  const CATask& tk = tasks[lo];
  const long long t = g - tk.t_start;
  double2 s = make_double2(0.0, 0.0);
  for (long long c = 0; c < tk.d.blocks; ++c) {
    const double2 v = tk.part[t * tk.d.blocks + c];
    s.x += v.x;
    s.y += v.y;
  }
  tk.out[t] = make_double2(s.x * tk.scale, s.y * tk.scale);
}

__global__ void __launch_bounds__(256)
k_reduce_grouped(const ReduceTask* __restrict__ tasks, const long long* __restrict__ starts,
                 int n) {
  const ReduceTask& tk = tasks[find_task(starts, n, blockIdx.x)];
  const long long base = (blockIdx.x - tk.block_start) * (long long)kReduceElems;
  for (int e = threadIdx.x; e < kReduceElems; e += 256) {
    const long long i = base + e;
    if (i >= tk.per) break;
    tk.out[i] = sum_splits(tk.part + i, tk.per, tk.splits);
  }
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D map over planes [lt][rows][kp], box (128-byte row, 128 rows, 1)
bool make_map(CUtensorMap* m, const void* base, bool bf16, int64_t kp, int64_t rows, int64_t lt) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)lt};
  cuuint64_t strides[2] = {(cuuint64_t)(kp * es), (cuuint64_t)(kp * rows * es)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), 128u, 1u};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// 3-D fp32 map over raw complex64 rows: dims (2K floats, rows, lt), strides
// in complex elements, box (32 floats = 128 bytes, box_rows, 1)
// [lt][K rows][n2 floats] (n unit-stride), boxes of kBN floats (kBN/2
// complex n) x 16 rows (complex k), unswizzled: the raw tile of a right
// operand stored [k][n]
// operand stored [k][n] (box_w = kBN), or of a left operand stored [k][rows]
// (box_w = 2 * kBM floats: 128 complex rows)
bool make_raw_map_mn(CUtensorMap* m, const void* base, int64_t n2, int64_t krows, int64_t lt,
                     int64_t row_stride, int64_t slice_stride, int box_w = kBN) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)n2, (cuuint64_t)krows, (cuuint64_t)lt};
  cuuint64_t strides[2] = {(cuuint64_t)(row_stride * 8), (cuuint64_t)(slice_stride * 8)};
  cuuint32_t box[3] = {(cuuint32_t)box_w, 16u, 1u};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// A right operand read in place as [k][n] tiles: dimensions (inner n as
// floats, the k axes innermost first, the outer n axis if any, batch), boxes
// of kBN floats x 16 k rows x 1 ...; fills the task's coordinate fields
bool make_raw_map_mnx(CUtensorMap* m, const void* base, const Group& bn, const Group& bk,
                      int64_t lt, int64_t slice_stride, GemmTask* t, int box_w = kBN) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5];
  int nd = 0;
  dims[nd] = (cuuint64_t)(2 * bn.ext[bn.n - 1]);
  box[nd++] = (cuuint32_t)box_w;
  t->b_nk = bk.n;
  for (int a = bk.n - 1; a >= 0; --a) {
    t->b_kext[bk.n - 1 - a] = bk.ext[a];
    dims[nd] = (cuuint64_t)bk.ext[a];
    strides[nd - 1] = (cuuint64_t)(bk.stride[a] * 8);
    box[nd++] = a == bk.n - 1 ? 16u : 1u;
  }
  t->b_no = bn.n == 2 ? 1 : 0;
  if (bn.n == 2) {
    dims[nd] = (cuuint64_t)bn.ext[0];
    strides[nd - 1] = (cuuint64_t)(bn.stride[0] * 8);
    box[nd++] = 1u;
  }
  dims[nd] = (cuuint64_t)lt;
  strides[nd - 1] = (cuuint64_t)(slice_stride * 8);
  box[nd++] = 1u;
  for (int a = 0; a < nd; ++a) estr[a] = 1;
  t->b_ni = bn.ext[bn.n - 1];
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, nd, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// left operand stored [outer rows][k][inner rows] (inner unit-stride): dims
// (2 ni floats, k, outer, lt), boxes of 128 rows = 128 / ni outer blocks of
// ni inner rows (ni <= 128), or 128 inner rows of one outer block
bool make_raw_map_a3(CUtensorMap* m, const void* base, int64_t ni, int64_t krows, int64_t no,
                     int64_t lt, int64_t k_stride, int64_t outer_stride, int64_t slice_stride) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int64_t bi = std::min<int64_t>(ni, kBM);
  cuuint64_t dims[4] = {(cuuint64_t)(2 * ni), (cuuint64_t)krows, (cuuint64_t)no, (cuuint64_t)lt};
  cuuint64_t strides[3] = {(cuuint64_t)(k_stride * 8), (cuuint64_t)(outer_stride * 8),
                           (cuuint64_t)(slice_stride * 8)};
  cuuint32_t box[4] = {(cuuint32_t)(2 * bi), 16u, (cuuint32_t)(kBM / bi), 1u};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_raw_map(CUtensorMap* m, const void* base, int64_t k2, int64_t rows, int64_t lt,
                  int64_t row_stride, int64_t slice_stride, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)k2, (cuuint64_t)std::max<int64_t>(rows, 1), (cuuint64_t)lt};
  cuuint64_t strides[2] = {(cuuint64_t)(row_stride * 8), (cuuint64_t)(slice_stride * 8)};
  cuuint32_t box[3] = {32u, (cuuint32_t)box_rows, 1u};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int num_sms() {  // SMs of the current device (one persistent CTA each)
  static int cached[64] = {0};  // read and written atomically: host threads may race here
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  int c = __atomic_load_n(&cached[dev], __ATOMIC_RELAXED);
  if (!c) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    c = n > 0 ? n : 148;
    __atomic_store_n(&cached[dev], c, __ATOMIC_RELAXED);
  }
  return c;
}

}  // namespace

namespace {
// split count: (policy 0) k splits while the output tiles alone cannot fill
// the GPU, keeping >= 4 k blocks per split; always FP32 chunks of <=
// kMaxChunk real k (error control)
int64_t choose_splits(const ContractDesc& cd, int64_t kblocks, int64_t bk, int policy) {
  const int64_t tiles = ((2 * cd.N + kBN - 1) / kBN) * ((cd.M + kBM - 1) / kBM) * cd.lt;
  int64_t splits = 1;
  if (policy == 0)
    while (tiles * splits * 2 <= 2 * 148 && kblocks / (splits * 2) >= 4) splits *= 2;
  while ((kblocks + splits - 1) / splits * bk > kMaxChunk && splits < 64) splits *= 2;
  return splits;
}
}  // namespace

namespace {
// the same contraction with the operands exchanged: C^T[n][m] = sum_k
// B[k][n] A[m][k] (pairs keep their order, so k runs alike)
ContractDesc exchanged(const ContractDesc& cd) {
  ContractDesc x = cd;
  x.M = cd.N;
  x.N = cd.M;
  x.a_ts = cd.b_ts;
  x.b_ts = cd.a_ts;
  x.am = cd.bn;
  x.ak = cd.bk;
  x.bk = cd.ak;
  x.bn = cd.am;
  x.a_kfast = cd.b_kfast;
  x.b_kfast = cd.a_kfast;
  return x;
}
int64_t gemm_tiles(const ContractDesc& cd) {
  return ((cd.M + kBM - 1) / kBM) * ((2 * cd.N + kBN - 1) / kBN) * cd.lt;
}
// fused form of cd with both operands read in place (no reorder)?
bool fused_in_place(const ContractDesc& cd, int split_policy, MixedDesc* x) {
  std::memset(x, 0, sizeof(*x));
  x->cd = cd;
  x->fused = true;
  return make_fused_desc(cd, x, split_policy) && x->a_direct && x->b_direct;
}
}  // namespace

bool make_mixed_desc(const ContractDesc& cd, bool bf16, MixedDesc* d, const MixedTune& tune) {
  std::memset(d, 0, sizeof(*d));
  // Orientation: a product with fewer rows than a tile (M < 128, e.g. a meson
  // times a baryon over one leg: 64 x 4096) fills half of every 128-row MMA;
  // its transpose (4096 x 64) does not.  The exchanged product is taken when
  // it needs at least a quarter fewer 128 x 64-complex tiles, or no more
  // tiles and no operand reorder where the given orientation needs one; it
  // is stored transposed by the GEMM's epilogue (shared-memory-A kernel).
  if (!bf16 && cd.K % 2 == 0 && tune.fused_kernel != 1 && cd.M <= tune.fused_max_n) {
    MixedDesc x, y;
    const ContractDesc sw = exchanged(cd);
    if (fused_in_place(sw, tune.split_policy, &x)) {
      const int64_t t0 = gemm_tiles(cd), t1 = gemm_tiles(sw);
      const bool normal_in_place =
          cd.N <= tune.fused_max_n && fused_in_place(cd, tune.split_policy, &y);
      if (4 * t1 <= 3 * t0 || (t1 <= t0 && !normal_in_place)) {
        *d = x;
        d->swap = true;
        d->pair = tune.fused_kernel == 2 && sw.M > kBM;
        return true;
      }
    }
    std::memset(d, 0, sizeof(*d));
  }
  d->bf16 = bf16;
  d->cd = cd;
  // fused form: TF32 with an even paired extent (16-byte complex64 rows) and
  // a narrow right operand (by default <= 64 complex columns).  There the hi/lo planes
  // of the plane form cost more HBM traffic than the contraction itself; for
  // wide operands the plane form is faster (its operand tiles reach shared
  // memory by TMA alone, while the converter warps add shared-memory traffic
  // next to the three MMAs per k-step).
  d->fused = !bf16 && (cd.K % 2 == 0) && cd.N <= tune.fused_max_n;
  d->tmem_a = tune.fused_kernel == 1;
  if (d->fused && make_fused_desc(cd, d, tune.split_policy)) {
    d->pair = tune.fused_kernel == 2 && cd.M > kBM;
    return true;
  }
  d->fused = false;
  const int es = bf16 ? 2 : 4;
  d->kp = round_up(2 * cd.K, 16 / es);          // 16-byte rows for TMA
  const int64_t bk = 128 / es;                  // elements per k block
  const int64_t kblocks = (d->kp + bk - 1) / bk;
  const int64_t splits = choose_splits(cd, kblocks, bk, tune.split_policy);
  d->splits = (int)splits;
  d->kblocks = (int)((kblocks + splits - 1) / splits);
  const int64_t plane_a = cd.lt * cd.M * d->kp * es;
  const int64_t plane_b = cd.lt * 2 * cd.N * d->kp * es;
  d->a_off = 0;
  d->b_off = round_up(2 * plane_a, 256);
  d->part_off = round_up(d->b_off + 2 * plane_b, 256);
  d->scratch_bytes = d->part_off + (splits > 1 ? splits * cd.lt * cd.M * 2 * cd.N * 4 : 0);
  d->plane_a = plane_a;
  d->plane_b = plane_b;
  return cd.M < (1 << 30) && 2 * cd.N < (1 << 30) && d->kp < (1 << 30);
}

namespace {
// dst axes (rows group, then k group) with the operand's strides
Group concat_groups(const Group& rows, const Group& ks) {
  Group g;
  g.n = 0;
  for (int a = 0; a < rows.n; ++a) {
    g.ext[g.n] = rows.ext[a];
    g.stride[g.n++] = rows.stride[a];
  }
  for (int a = 0; a < ks.n; ++a) {
    g.ext[g.n] = ks.ext[a];
    g.stride[g.n++] = ks.stride[a];
  }
  return g;
}
}  // namespace

bool make_fused_desc(const ContractDesc& cd, MixedDesc* d, int split_policy) {
  d->kp = 2 * cd.K;                              // real k of a complex64 row
  const int64_t bk = 32;                         // fp32 elements per 128-byte k block
  const int64_t kblocks = (d->kp + bk - 1) / bk;
  const int64_t splits = choose_splits(cd, kblocks, bk, split_policy);
  d->splits = (int)splits;
  d->kblocks = (int)((kblocks + splits - 1) / splits);
  // an operand whose paired axes form its unit-stride axis and whose free
  // axes collapse to one row stride is read in place; otherwise it is
  // reordered into [t][rows][K]
  auto direct = [](const Group& rows, const Group& ks, int kfast) {
    return kfast && ks.n == 1 && ks.stride[0] == 1 &&
           (rows.n == 0 || (rows.n == 1 && rows.stride[0] % 2 == 0));
  };
  d->a_direct = direct(cd.am, cd.ak, cd.a_kfast) && cd.a_ts % 2 == 0;
  d->b_direct = direct(cd.bn, cd.bk, cd.b_kfast) && cd.b_ts % 2 == 0;
  d->a_rowstride = d->a_direct ? (cd.am.n ? cd.am.stride[0] : cd.K) : cd.K;
  d->b_rowstride = d->b_direct ? (cd.bn.n ? cd.bn.stride[0] : cd.K) : cd.K;
  // B stored [k][n] with n unit-stride (a matrix product's right operand):
  // read in place, k rows of 16-byte multiples, transposed by the converters
  d->b_mn = !d->b_direct && !cd.b_kfast && cd.bn.n == 1 && cd.bn.stride[0] == 1 &&
            cd.bk.n == 1 && cd.bk.stride[0] % 2 == 0 && cd.b_ts % 2 == 0;
  // or [k][outer n][inner n] blocks (a propagator contracted over one
  // distillation axis): one TMA box per tile when the inner n extent is a
  // multiple of the tile's 64 complex columns
  // general in-place [k][n] tiles: the inner n axis unit-stride (a multiple
  // of 64 columns if an outer n axis follows), up to 3 k axes whose innermost
  // extent is a multiple of 16 (a k block never straddles), at most 5 map
  // dimensions with the batch axis, all strides 16-byte multiples
  d->b_mn2 = false;
  if (!d->b_direct && !d->b_mn && !cd.b_kfast && (cd.bn.n == 1 || cd.bn.n == 2) &&
      cd.bn.stride[cd.bn.n - 1] == 1 && cd.bk.n >= 1 && cd.bk.n <= 3 &&
      1 + cd.bk.n + (cd.bn.n - 1) + 1 <= 5 && cd.bk.ext[cd.bk.n - 1] % 16 == 0 &&
      (cd.bn.n == 1 || cd.bn.ext[1] % (kBN / 2) == 0) && cd.b_ts % 2 == 0) {
    bool even = cd.bn.stride[0] % 2 == 0 || cd.bn.n == 1;
    for (int a = 0; a < cd.bk.n; ++a) even = even && cd.bk.stride[a] % 2 == 0;
    d->b_mn2 = even;
  }
  if (d->b_mn || d->b_mn2) {
    d->b_direct = true;
    d->b_rowstride = cd.bk.stride[0];
  }
  // A stored [k][rows] with the rows unit-stride (a tensor contracted over
  // its leading axis): read in place, k rows of 16-byte multiples, transposed
  // by the converters (the shared-memory-A kernel only)
  d->a_mn = !d->tmem_a && !d->a_direct && !cd.a_kfast && cd.am.n == 1 &&
            cd.am.stride[0] == 1 && cd.ak.n == 1 && cd.ak.stride[0] % 2 == 0 &&
            cd.a_ts % 2 == 0;
  d->a_ni = 0;
  // ... or [outer rows][k][inner rows] (a baryon contracted over its middle
  // leg): inner extent 16, 32, 64 or a multiple of 128, so that a 128-row
  // tile is whole outer blocks or one piece of one
  if (!d->a_mn && !d->tmem_a && !d->a_direct && !cd.a_kfast && cd.am.n == 2 &&
      cd.am.stride[1] == 1 && cd.ak.n == 1 && cd.ak.stride[0] % 2 == 0 &&
      cd.am.stride[0] % 2 == 0 && cd.a_ts % 2 == 0) {
    const int64_t ni = cd.am.ext[1];
    if (ni == 16 || ni == 32 || ni == 64 || ni % 128 == 0) {
      d->a_mn = true;
      d->a_ni = ni;
      d->a_outer_stride = cd.am.stride[0];
    }
  }
  if (d->a_mn) {
    d->a_direct = true;
    d->a_rowstride = cd.ak.stride[0];
  }
  int64_t off = 0;
  d->a_off = off;
  if (!d->a_direct) {
    make_perm_desc(concat_groups(cd.am, cd.ak), cd.lt, cd.a_ts, &d->a_perm);
    if (!perm_fits(d->a_perm)) return false;
    off = round_up(off + cd.lt * cd.M * cd.K * 8, 256);
  }
  d->b_off = off;
  if (!d->b_direct) {
    make_perm_desc(concat_groups(cd.bn, cd.bk), cd.lt, cd.b_ts, &d->b_perm);
    if (!perm_fits(d->b_perm)) return false;
    off = round_up(off + cd.lt * cd.N * cd.K * 8, 256);
  }
  d->part_off = off;
  d->scratch_bytes = off + (splits > 1 ? splits * cd.lt * cd.M * 2 * cd.N * 4 : 0);
  return cd.M < (1 << 30) && 2 * cd.N < (1 << 30) && d->kp < (1 << 30);
}

static PackArgs pack_args(const ContractDesc& cd, int which, int64_t kp) {
  PackArgs a;
  std::memset(&a, 0, sizeof(a));
  a.which = which;
  a.K = (int)cd.K;
  a.kp = kp;
  if (which == 0) {
    a.rows = (int)cd.M;
    a.rg = cd.am;
    a.kg = cd.ak;
    a.ts = cd.a_ts;
    a.k_fast = cd.a_kfast;
  } else {
    a.rows = (int)cd.N;
    a.rg = cd.bn;
    a.kg = cd.bk;
    a.ts = cd.b_ts;
    a.k_fast = cd.b_kfast;
  }
  return a;
}

// task of one contraction whose planes / partials live in `scratch`
// a_stage / b_stage: where the operand's planes (plane form) or reordered
// copy (fused form) are, when another contraction of the level produced them;
// nullptr = in this contraction's own scratch
bool fill_gemm_task(const MixedDesc& d, const float* A, const float* B, void* scratch, float* C,
                    GemmTask* t, const char* a_stage, const char* b_stage) {
  const ContractDesc& cd = d.cd;
  char* sc = static_cast<char*>(scratch);
  const char* as = a_stage ? a_stage : sc + d.a_off;
  const char* bs = b_stage ? b_stage : sc + d.b_off;
  std::memset(t, 0, sizeof(*t));
  if (d.fused) {
    const void* a = d.a_direct ? (const void*)A : (const void*)as;
    const void* b = d.b_direct ? (const void*)B : (const void*)bs;
    const int64_t ats = d.a_direct ? cd.a_ts : cd.M * cd.K;
    const int64_t bts = d.b_direct ? cd.b_ts : cd.N * cd.K;
    if (d.a_mn && d.a_ni) {  // [outer][k][inner]
      if (!make_raw_map_a3(&t->map[0], a, d.a_ni, cd.K, cd.M / d.a_ni, cd.lt, d.a_rowstride,
                           d.a_outer_stride, ats))
        return false;
      t->a_mn = 2;
      t->a_ni = (int)std::min<int64_t>(d.a_ni, kBM);
      t->a_nio = (int)d.a_ni;
    } else if (d.a_mn) {
      if (!make_raw_map_mn(&t->map[0], a, 2 * cd.M, cd.K, cd.lt, d.a_rowstride, ats, 2 * kBM))
        return false;
      t->a_mn = 1;
      t->a_ni = kBM;
    } else if (!make_raw_map(&t->map[0], a, d.kp, cd.M, cd.lt, d.a_rowstride, ats, kBM)) {
      return false;
    }
    // raw B boxes: kBN / 2 complex columns, or half that for a CTA of a pair
    const int bcols = d.pair ? kBN / 4 : kBN / 2;
    if (d.b_mn2) {
      if (!make_raw_map_mnx(&t->map[2], b, cd.bn, cd.bk, cd.lt, bts, t, 2 * bcols)) return false;
    } else if (d.b_mn ? !make_raw_map_mn(&t->map[2], b, 2 * cd.N, cd.K, cd.lt, d.b_rowstride, bts,
                                         2 * bcols)
                      : !make_raw_map(&t->map[2], b, d.kp, cd.N, cd.lt, d.b_rowstride, bts,
                                      bcols)) {
      return false;
    }
    t->b_mn = d.b_mn2 ? 2 : (d.b_mn ? 1 : 0);
    t->a_raw = static_cast<const float2*>(a);
    t->a_ts = ats;
    t->a_rs = d.a_rowstride;
    t->kc = (int)cd.K;
  } else if (!make_map(&t->map[0], as, d.bf16, d.kp, cd.M, cd.lt) ||
             !make_map(&t->map[1], as + d.plane_a, d.bf16, d.kp, cd.M, cd.lt) ||
             !make_map(&t->map[2], bs, d.bf16, d.kp, 2 * cd.N, cd.lt) ||
             !make_map(&t->map[3], bs + d.plane_b, d.bf16, d.kp, 2 * cd.N, cd.lt))
    return false;
  t->M = (int)cd.M;
  t->Nr = (int)(2 * cd.N);
  t->kblocks = d.kblocks;
  t->splits = d.splits;
  t->lt = (int)cd.lt;
  t->ntn = (t->Nr + kBN - 1) / kBN;
  const int rows = d.pair ? 2 * kBM : kBM;  // a pair's tile: 256 rows
  t->ntm = (t->M + rows - 1) / rows;
  t->tiles = t->ntn * t->ntm * t->lt * t->splits;
  t->out = d.splits > 1 ? reinterpret_cast<float*>(sc + d.part_off) : C;
  t->out_t = d.swap ? 1 : 0;
  return true;
}

// operand reorders of a fused contraction (0, 1 or 2 launches)
int launch_fused_copies(const MixedDesc& d, const float* A, const float* B, void* scratch,
                        cudaStream_t s) {
  int nk = 0;
  char* sc = static_cast<char*>(scratch);
  if (!d.a_direct) {
    if (launch_permute_c64(d.a_perm, A, reinterpret_cast<float*>(sc + d.a_off), s) < 0) return -1;
    ++nk;
  }
  if (!d.b_direct) {
    if (launch_permute_c64(d.b_perm, B, reinterpret_cast<float*>(sc + d.b_off), s) < 0) return -1;
    ++nk;
  }
  return nk;
}

template <bool BF16, bool FUSED, bool AMN = false>
void launch_gemm_t(const GemmParams& gp, dim3 grid, cudaStream_t s) {
  using C = GemmCfg<BF16, FUSED>;
  cudaFuncSetAttribute(k_gemm_split3<BF16, FUSED, AMN>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  k_gemm_split3<BF16, FUSED, AMN><<<grid, C::kThreads, C::kSmem, s>>>(gp);
}

// CTA-pair form: clusters of 2, as many pairs as can be resident at once
// (one CTA per SM), at most one per pair tile
template <bool AMN>
int launch_gemm_pair_t(const GemmParams& gp, cudaStream_t s) {
  using C = GemmCfg<false, true, true>;
  auto kern = k_gemm_split3<false, true, AMN, true>;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(C::kThreads);
  cfg.dynamicSmemBytes = C::kSmem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // resident pairs of this kernel form, found once (a function-local static:
  // initialised by one thread; sized on the first device that launches it)
  static const int np = [&]() {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
    cudaLaunchConfig_t probe = cfg;
    probe.gridDim = dim3(2 * (num_sms() / 2));
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &probe) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = num_sms() / 2;
    }
    return n;
  }();
  cfg.gridDim = dim3((unsigned)(2 * std::min<long long>(gp.total_tiles, np)));
  return cudaLaunchKernelEx(&cfg, kern, gp) == cudaSuccess ? 1 : -1;
}

// amn: some fused task of the launch reads A as [k][rows] tiles; pair: the
// launch's tasks are tiled for CTA pairs
int launch_gemm(const GemmParams& gp, bool bf16, bool fused, cudaStream_t s,
                bool tmem_a = false, bool amn = false, bool pair = false) {
  if (gp.total_tiles <= 0) return 0;
  if (fused && pair) return amn ? launch_gemm_pair_t<true>(gp, s) : launch_gemm_pair_t<false>(gp, s);
  dim3 grid((unsigned)std::min<long long>(gp.total_tiles, num_sms()));
  if (fused && tmem_a) {
    cudaFuncSetAttribute(k_gemm_tf32_tmem_a, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         TaCfg::kSmem);
    k_gemm_tf32_tmem_a<<<grid, TaCfg::kThreads, TaCfg::kSmem, s>>>(gp);
  } else if (fused && amn) launch_gemm_t<false, true, true>(gp, grid, s);
  else if (fused) launch_gemm_t<false, true>(gp, grid, s);
  else if (bf16) launch_gemm_t<true, false>(gp, grid, s);
  else launch_gemm_t<false, false>(gp, grid, s);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_contract_mixed(const MixedDesc& d, const float* A, const float* B, float* C,
                          void* scratch, cudaStream_t s) {
  const ContractDesc& cd = d.cd;
  if (d.fused) {
    if (d.swap) std::swap(A, B);  // the GEMM's left operand is the contraction's right one
    int nk = launch_fused_copies(d, A, B, scratch, s);
    if (nk < 0) return -1;
    GemmParams gp;
    std::memset(&gp, 0, sizeof(gp));
    if (!fill_gemm_task(d, A, B, scratch, C, &gp.single, nullptr, nullptr)) return -2;
    gp.total_tiles = gp.single.tiles;
    if (launch_gemm(gp, false, true, s, d.tmem_a, d.a_mn, d.pair) < 0) return -1;
    ++nk;
    if (d.splits > 1) {
      const long long per = cd.lt * cd.M * 2 * cd.N;
      unsigned blocks = (unsigned)std::min<long long>((per + 255) / 256, 8 * 148);
      k_reduce_splits<<<blocks, 256, 0, s>>>(gp.single.out, C, per, d.splits);
      ++nk;
    }
    return cudaPeekAtLastError() == cudaSuccess ? nk : -1;
  }
  char* sc = static_cast<char*>(scratch);
  void* ahi = sc + d.a_off;
  void* alo = sc + d.a_off + d.plane_a;
  void* bhi = sc + d.b_off;
  void* blo = sc + d.b_off + d.plane_b;
  int nk = 0;
  {
    const int64_t kc = std::max<int64_t>(cd.K, d.kp / 2);  // complex columns incl. padding
    const int64_t rows = std::max<int64_t>(cd.M, cd.N);
    dim3 grid((unsigned)((kc + 31) / 32), (unsigned)((rows + 31) / 32), (unsigned)(2 * cd.lt));
    if (d.bf16) {
      PackPair<true> pp;
      pp.op[0] = pack_args(cd, 0, d.kp);
      pp.op[1] = pack_args(cd, 1, d.kp);
      pp.X[0] = reinterpret_cast<const float2*>(A);
      pp.X[1] = reinterpret_cast<const float2*>(B);
      pp.hi[0] = (__nv_bfloat16*)ahi;
      pp.lo[0] = (__nv_bfloat16*)alo;
      pp.hi[1] = (__nv_bfloat16*)bhi;
      pp.lo[1] = (__nv_bfloat16*)blo;
      pp.lt = (int)cd.lt;
      k_pack<true><<<grid, 256, 0, s>>>(pp);
    } else {
      PackPair<false> pp;
      pp.op[0] = pack_args(cd, 0, d.kp);
      pp.op[1] = pack_args(cd, 1, d.kp);
      pp.X[0] = reinterpret_cast<const float2*>(A);
      pp.X[1] = reinterpret_cast<const float2*>(B);
      pp.hi[0] = (float*)ahi;
      pp.lo[0] = (float*)alo;
      pp.hi[1] = (float*)bhi;
      pp.lo[1] = (float*)blo;
      pp.lt = (int)cd.lt;
      k_pack<false><<<grid, 256, 0, s>>>(pp);
    }
    ++nk;
  }
  GemmParams gp;
  std::memset(&gp, 0, sizeof(gp));
  if (!fill_gemm_task(d, A, B, scratch, C, &gp.single, nullptr, nullptr)) return -2;
  gp.total_tiles = gp.single.tiles;
  if (launch_gemm(gp, d.bf16, false, s) < 0) return -1;
  ++nk;
  if (d.splits > 1) {
    const long long per = cd.lt * cd.M * 2 * cd.N;
    unsigned blocks = (unsigned)std::min<long long>((per + 255) / 256, 8 * 148);
    k_reduce_splits<<<blocks, 256, 0, s>>>(gp.single.out, C, per, d.splits);
    ++nk;
  }
  return cudaPeekAtLastError() == cudaSuccess ? nk : -1;
}

void make_perm_desc(const Group& g0, int64_t lt, int64_t src_ts, PermDesc* d) {
  std::memset(d, 0, sizeof(*d));
  Group g;  // drop axes of extent 1: they move nothing
  g.n = 0;
  for (int a = 0; a < g0.n; ++a)
    if (g0.ext[a] > 1) {
      g.ext[g.n] = g0.ext[a];
      g.stride[g.n++] = g0.stride[a];
    }
  if (g.n == 0) {
    g.n = 1;
    g.ext[0] = 1;
    g.stride[0] = 1;
  }
  d->lt = (int)lt;
  d->src_ts = src_ts;
  long long dst_stride[LQC_MAX_RANK];
  long long n = 1;
  for (int a = g.n - 1; a >= 0; --a) {
    dst_stride[a] = n;
    n *= g.ext[a];
  }
  d->n = n;
  const int last = g.n - 1;
  int y = -1;
  for (int a = 0; a < g.n; ++a)
    if (g.stride[a] == 1) y = a;
  d->X = g.ext[last];
  d->mode = (g.stride[last] == 1 || y < 0) ? 0 : 1;
  if (d->mode == 1) {
    d->Y = g.ext[y];
    d->sX = g.stride[last];
    d->dY = dst_stride[y];
  }
  d->outer = 1;
  for (int a = 0; a < last; ++a) {
    if (d->mode == 1 && a == y) continue;
    d->oext[d->nout] = g.ext[a];
    d->osrc[d->nout] = g.stride[a];
    d->odst[d->nout++] = dst_stride[a];
    d->outer *= g.ext[a];
  }
  if (d->mode == 0 && g.stride[last] != 1) {
    // no unit-stride axis at all (cannot happen for a permutation of a
    // contiguous tensor with an innermost extent > 1): copy element-wise runs
    // of length 1
    d->oext[d->nout] = g.ext[last];
    d->osrc[d->nout] = g.stride[last];
    d->odst[d->nout++] = 1;
    d->outer *= g.ext[last];
    d->X = 1;
  }
  d->blocks = d->mode == 0
                  ? (d->n + kPermElems - 1) / kPermElems
                  : d->outer * ((d->X + 31) / 32) *
                        (((d->Y + 31) / 32 + kPermTiles - 1) / kPermTiles);
}

bool perm_fits(const PermDesc& d) {  // the block functions use 32-bit offsets
  return d.n < (1ll << 31) && d.src_ts < (1ll << 31) && d.blocks > 0 && d.blocks < (1ll << 31);
}

int launch_permute_c64(const PermDesc& d, const float* src, float* dst, cudaStream_t s) {
  if (d.lt > 65535 || !perm_fits(d)) return -1;
  dim3 grid((unsigned)d.blocks, (unsigned)d.lt);
  k_permute_c64<<<grid, 256, 0, s>>>(reinterpret_cast<const float2*>(src),
                                     reinterpret_cast<float2*>(dst), d);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

namespace {
// correlator plan: B visited in the left operand's order (no copy)
PermDesc ca_perm(const ContractAllDesc& d) {
  PermDesc pd;
  make_perm_desc(d.bp, d.lt, d.S, &pd);
  if (pd.mode == 1)  // warp tiles of 32x32, kCaWarpTiles per block
    pd.blocks = (pd.outer * ((pd.X + 31) / 32) * ((pd.Y + 31) / 32) + kCaWarpTiles - 1) /
                kCaWarpTiles;
  return pd;
}
int64_t ca_part_bytes(const PermDesc& pd) {
  return (pd.lt * (int64_t)pd.blocks * 16 + 255) & ~int64_t(255);
}
}  // namespace

int64_t contract_all_c64_scratch_bytes(const ContractAllDesc& d) {
  return ca_part_bytes(ca_perm(d));
}

int launch_contract_all_c64(const ContractAllDesc& d0, const float* A, const float* B, double* C,
                            double* scratch, double scale, cudaStream_t s) {
  const PermDesc pd = ca_perm(d0);
  if (pd.lt > 65535 || !perm_fits(pd) || pd.blocks > (1 << 20)) return -1;
  dim3 grid((unsigned)pd.blocks, (unsigned)pd.lt);
  double2* part = reinterpret_cast<double2*>(scratch);
  k_contract_all_c64<<<grid, 256, 0, s>>>(reinterpret_cast<const float2*>(A),
                                          reinterpret_cast<const float2*>(B), part, pd);
  k_contract_all_final_scaled<<<(unsigned)((pd.lt + 127) / 128), 128, 0, s>>>(
      part, reinterpret_cast<double2*>(C), pd.lt, (int)pd.blocks, scale);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

int mixed_error_status(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_mixed_error, sizeof(int)) != cudaSuccess) return -1;
  if (reset && v) {
    int z = 0;
    cudaMemcpyToSymbol(g_mixed_error, &z, sizeof(int));
  }
  return v;
}

}  // namespace lqc

// ---------------------------------------------------------------- grouped host side
namespace lqc {
namespace {
size_t align_to(size_t x, size_t a) { return (x + a - 1) / a * a; }
template <typename T>
size_t append(std::vector<char>* buf, const std::vector<T>& v, size_t align) {
  const size_t off = align_to(buf->size(), align);
  buf->resize(off + sizeof(T) * v.size());
  if (!v.empty()) std::memcpy(buf->data() + off, v.data(), sizeof(T) * v.size());
  return off;
}
}  // namespace

bool append_level_tasks(const std::vector<GroupExt>& ext, const std::vector<GroupRoot>& roots,
                        bool bf16, std::vector<char>* buf, LevelDev* lvl) {
  std::memset(lvl, 0, sizeof(*lvl));
  std::vector<PackTask> pk;
  std::vector<GemmTask> gm;
  std::vector<ReduceTask> rd;
  std::vector<CATask> ca;
  std::vector<PermTask> pm;
  std::vector<GemmTask> gf;  // fused-form GEMM tasks
  std::vector<GemmTask> gq;  // ... run by CTA pairs
  long long pb = 0, tiles = 0, rb = 0, cb = 0, ct = 0, mb = 0, ftiles = 0, qtiles = 0;
  bool lvl_pair_amn = false;
  bool lvl_tmem_a = false, lvl_amn = false;
  auto add_perm = [&](const PermDesc& pd, const void* src, void* dst) {
    PermTask t;
    std::memset(&t, 0, sizeof(t));
    t.d = pd;
    t.src = static_cast<const float2*>(src);
    t.dst = static_cast<float2*>(dst);
    t.block_start = mb;
    mb += t.d.blocks * t.d.lt;
    pm.push_back(t);
  };
  auto add_reduce = [&](const MixedDesc& d, const GemmTask& g, float* C) {
    const ContractDesc& cd = d.cd;
    ReduceTask r;
    r.part = g.out;
    r.out = C;
    r.per = cd.lt * cd.M * 2 * cd.N;
    r.splits = d.splits;
    r.block_start = rb;
    rb += (r.per + kReduceElems - 1) / kReduceElems;
    rd.push_back(r);
  };
  // an operand staged (reordered, or split into planes) for one contraction
  // of the level serves every contraction of the level that stages the same
  // tensor the same way: key = source address + the staging descriptor
  std::unordered_map<std::string, const char*> staged;
  auto key_of = [](const void* src, const void* desc, size_t n, int64_t lt) {
    std::string k(reinterpret_cast<const char*>(&src), sizeof(src));
    k.append(reinterpret_cast<const char*>(desc), n);
    k.append(reinterpret_cast<const char*>(&lt), sizeof(lt));
    return k;
  };
  // returns the staged data of (src, desc): existing, or `dst` after
  // registering it (then *fresh = true and the caller adds the task)
  auto stage = [&](const std::string& key, const char* dst, bool* fresh) {
    auto it = staged.find(key);
    *fresh = it == staged.end();
    if (*fresh) staged.emplace(key, dst);
    return *fresh ? dst : it->second;
  };
  for (const GroupExt& e : ext) {
    const MixedDesc& d = *e.d;
    const ContractDesc& cd = d.cd;
    char* sc = e.scratch;
    const char* as = nullptr;
    const char* bs = nullptr;
    bool fresh = false;
    if (d.fused) {
      // operands in the GEMM's roles (exchanged for a transposed product)
      const float* EA = d.swap ? e.B : e.A;
      const float* EB = d.swap ? e.A : e.B;
      if (!d.a_direct) {
        as = stage(key_of(EA, &d.a_perm, sizeof(PermDesc), 0), sc + d.a_off, &fresh);
        if (fresh) add_perm(d.a_perm, EA, sc + d.a_off);
      }
      if (!d.b_direct) {
        bs = stage(key_of(EB, &d.b_perm, sizeof(PermDesc), 0), sc + d.b_off, &fresh);
        if (fresh) add_perm(d.b_perm, EB, sc + d.b_off);
      }
      GemmTask g;
      if (!fill_gemm_task(d, EA, EB, e.scratch, e.C, &g, as, bs)) return false;
      lvl_tmem_a = d.tmem_a;  // one DAG option: every fused task of a level alike
      if (d.pair) {
        lvl_pair_amn = lvl_pair_amn || d.a_mn;
        g.tile_start = qtiles;
        qtiles += g.tiles;
        gq.push_back(g);
      } else {
        lvl_amn = lvl_amn || d.a_mn;
        g.tile_start = ftiles;
        ftiles += g.tiles;
        gf.push_back(g);
      }
      if (d.splits > 1) add_reduce(d, g, e.C);
      continue;
    }
    const int64_t kc = std::max<int64_t>(cd.K, d.kp / 2);
    for (int which = 0; which < 2; ++which) {
      PackTask p;
      std::memset(&p, 0, sizeof(p));
      p.op = pack_args(cd, which, d.kp);
      p.X = reinterpret_cast<const float2*>(which ? e.B : e.A);
      char* dst = sc + (which ? d.b_off : d.a_off);
      const char* got = stage(key_of(p.X, &p.op, sizeof(PackArgs), cd.lt),
                              dst, &fresh);
      (which ? bs : as) = got;
      if (!fresh) continue;
      p.hi = dst;
      p.lo = dst + (which ? d.plane_b : d.plane_a);
      p.kblk = (int)((kc + 31) / 32);
      p.rblk = (int)((p.op.rows + 31) / 32);
      p.block_start = pb;
      pb += (long long)p.kblk * p.rblk * cd.lt;
      pk.push_back(p);
    }
    GemmTask g;
    if (!fill_gemm_task(d, e.A, e.B, e.scratch, e.C, &g, as, bs)) return false;
    g.tile_start = tiles;
    tiles += g.tiles;
    gm.push_back(g);
    if (d.splits > 1) add_reduce(d, g, e.C);
  }
  for (const GroupRoot& r : roots) {
    CATask c;
    std::memset(&c, 0, sizeof(c));
    c.A = reinterpret_cast<const float2*>(r.A);
    c.B = reinterpret_cast<const float2*>(r.B);
    c.out = reinterpret_cast<double2*>(r.C);
    c.part = reinterpret_cast<double2*>(r.part);
    c.d = ca_perm(*r.d);
    if (!perm_fits(c.d)) return false;
    c.scale = r.scale;
    c.t_start = ct;
    ct += c.d.lt;
    ca.push_back(c);
  }
  // correlator segments, chunk-major; within a chunk the tasks ordered by the
  // operand they share most in this level (then the other operand)
  std::vector<long long> seg_start;
  std::vector<CASeg> segs;
  {
    std::unordered_map<const void*, int> uses;
    for (const CATask& c : ca) {
      ++uses[c.A];
      ++uses[c.B];
    }
    struct Key {
      uintptr_t primary, secondary;
      int task;
    };
    std::vector<Key> keys;
    std::vector<int> per(ca.size());  // slices per chunk
    int max_chunks = 0;
    for (size_t i = 0; i < ca.size(); ++i) {
      uintptr_t a = reinterpret_cast<uintptr_t>(ca[i].A), b = reinterpret_cast<uintptr_t>(ca[i].B);
      const int ua = uses[ca[i].A], ub = uses[ca[i].B];
      if (ub > ua || (ub == ua && b < a)) std::swap(a, b);
      keys.push_back({a, b, (int)i});
      per[i] = (int)std::min<long long>(ca[i].d.lt, std::max<long long>(
                                                        1, kCaChunkElems / std::max(1ll, ca[i].d.n)));
      max_chunks = std::max(max_chunks, (ca[i].d.lt + per[i] - 1) / per[i]);
    }
    std::sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
      if (x.primary != y.primary) return x.primary < y.primary;
      if (x.secondary != y.secondary) return x.secondary < y.secondary;
      return x.task < y.task;
    });
    for (int q = 0; q < max_chunks; ++q)
      for (const Key& k : keys) {
        const CATask& c = ca[k.task];
        const int t0 = q * per[k.task];
        if (t0 >= c.d.lt) continue;
        seg_start.push_back(cb);
        segs.push_back({k.task, t0});
        cb += c.d.blocks * std::min(per[k.task], c.d.lt - t0);
      }
  }
  auto starts = [&](const auto& v) {
    std::vector<long long> st;
    for (const auto& t : v) st.push_back(t.block_start);
    return reinterpret_cast<const long long*>(append(buf, st, 64));
  };
  lvl->pack_starts = starts(pk);
  lvl->red_starts = starts(rd);
  lvl->perm_starts = starts(pm);
  lvl->ca_starts = reinterpret_cast<const long long*>(append(buf, seg_start, 64));
  lvl->ca_segs = reinterpret_cast<const void*>(append(buf, segs, 64));
  lvl->nca_seg = (int)segs.size();
  lvl->pack = reinterpret_cast<const void*>(append(buf, pk, 64));
  lvl->npack = (int)pk.size();
  lvl->pack_blocks = pb;
  lvl->gemm = reinterpret_cast<const void*>(append(buf, gm, 64));
  lvl->ngemm = (int)gm.size();
  lvl->gemm_tiles = tiles;
  lvl->gemm_fused = reinterpret_cast<const void*>(append(buf, gf, 64));
  lvl->ngemm_fused = (int)gf.size();
  lvl->gemm_fused_tiles = ftiles;
  lvl->fused_tmem_a = lvl_tmem_a;
  lvl->fused_amn = lvl_amn;
  lvl->gemm_pair = reinterpret_cast<const void*>(append(buf, gq, 64));
  lvl->ngemm_pair = (int)gq.size();
  lvl->gemm_pair_tiles = qtiles;
  lvl->pair_amn = lvl_pair_amn;
  lvl->red = reinterpret_cast<const void*>(append(buf, rd, 64));
  lvl->nred = (int)rd.size();
  lvl->red_blocks = rb;
  lvl->perm = reinterpret_cast<const void*>(append(buf, pm, 64));
  lvl->nperm = (int)pm.size();
  lvl->perm_blocks = mb;
  lvl->ca = reinterpret_cast<const void*>(append(buf, ca, 64));
  lvl->nca = (int)ca.size();
  lvl->ca_blocks = cb;
  lvl->ca_threads = ct;
  lvl->bf16 = bf16;
  return true;
}

void rebase_level(LevelDev* lvl, const char* base) {
  lvl->pack = base + reinterpret_cast<uintptr_t>(lvl->pack);
  lvl->gemm = base + reinterpret_cast<uintptr_t>(lvl->gemm);
  lvl->red = base + reinterpret_cast<uintptr_t>(lvl->red);
  lvl->perm = base + reinterpret_cast<uintptr_t>(lvl->perm);
  lvl->gemm_fused = base + reinterpret_cast<uintptr_t>(lvl->gemm_fused);
  lvl->gemm_pair = base + reinterpret_cast<uintptr_t>(lvl->gemm_pair);
  lvl->ca = base + reinterpret_cast<uintptr_t>(lvl->ca);
  lvl->ca_segs = base + reinterpret_cast<uintptr_t>(lvl->ca_segs);
  auto rb = [&](const long long*& p) {
    p = reinterpret_cast<const long long*>(base + reinterpret_cast<uintptr_t>(p));
  };
  rb(lvl->pack_starts);
  rb(lvl->red_starts);
  rb(lvl->perm_starts);
  rb(lvl->ca_starts);
}

int level_launch_kinds(const LevelDev& L, int kinds[LQC_NUM_KINDS]) {
  int n = 0;
  if (L.nperm > 0) kinds[n++] = LQC_KIND_REORDER;
  if (L.npack > 0) {
    kinds[n++] = LQC_KIND_PACK;
    kinds[n++] = LQC_KIND_GEMM_PLANES;
  }
  if (L.ngemm_pair > 0) kinds[n++] = LQC_KIND_GEMM_FUSED;
  if (L.ngemm_fused > 0) kinds[n++] = LQC_KIND_GEMM_FUSED;
  if (L.nred > 0) kinds[n++] = LQC_KIND_REDUCE;
  if (L.nca > 0) {
    kinds[n++] = LQC_KIND_CORRELATOR;
    kinds[n++] = LQC_KIND_CORRELATOR_SUM;
  }
  return n;
}

int launch_level(const LevelDev& L, cudaStream_t s, cudaEvent_t* marks, unsigned mark_flags) {
  int nk = 0;
  // marks[i] before the i-th launch, marks[n] after the last
  auto mark = [&]() {
    if (marks) cudaEventRecordWithFlags(marks[nk], s, mark_flags);
  };
  if (L.nperm > 0) {  // operand reorders of fused GEMMs and correlator partners
    mark();
    k_permute_grouped<<<(unsigned)L.perm_blocks, 256, 0, s>>>(
        static_cast<const PermTask*>(L.perm), L.perm_starts, L.nperm);
    ++nk;
  }
  if (L.npack > 0) {
    mark();
    if (L.bf16)
      k_pack_grouped<true><<<(unsigned)L.pack_blocks, 256, 0, s>>>(
          static_cast<const PackTask*>(L.pack), L.pack_starts, L.npack);
    else
      k_pack_grouped<false><<<(unsigned)L.pack_blocks, 256, 0, s>>>(
          static_cast<const PackTask*>(L.pack), L.pack_starts, L.npack);
    ++nk;
    GemmParams gp;
    std::memset(&gp, 0, sizeof(gp));
    gp.tasks = static_cast<const GemmTask*>(L.gemm);
    gp.ntasks = L.ngemm;
    gp.total_tiles = L.gemm_tiles;
    mark();
    if (launch_gemm(gp, L.bf16, false, s) < 0) return -1;
    ++nk;
  }
  if (L.ngemm_pair > 0) {  // the wide products first, by CTA pairs
    GemmParams gp;
    std::memset(&gp, 0, sizeof(gp));
    gp.tasks = static_cast<const GemmTask*>(L.gemm_pair);
    gp.ntasks = L.ngemm_pair;
    gp.total_tiles = L.gemm_pair_tiles;
    mark();
    if (launch_gemm(gp, false, true, s, false, L.pair_amn, true) < 0) return -1;
    ++nk;
  }
  if (L.ngemm_fused > 0) {
    GemmParams gp;
    std::memset(&gp, 0, sizeof(gp));
    gp.tasks = static_cast<const GemmTask*>(L.gemm_fused);
    gp.ntasks = L.ngemm_fused;
    gp.total_tiles = L.gemm_fused_tiles;
    mark();
    if (launch_gemm(gp, false, true, s, L.fused_tmem_a, L.fused_amn) < 0) return -1;
    ++nk;
  }
  if (L.nred > 0) {
    mark();
    k_reduce_grouped<<<(unsigned)L.red_blocks, 256, 0, s>>>(
        static_cast<const ReduceTask*>(L.red), L.red_starts, L.nred);
    ++nk;
  }
  if (L.nca > 0) {
    mark();
    k_contract_all_grouped<<<(unsigned)L.ca_blocks, 256, 0, s>>>(
        static_cast<const CATask*>(L.ca), L.ca_starts, static_cast<const CASeg*>(L.ca_segs),
        L.nca_seg);
    ++nk;
    mark();
    k_contract_all_final_grouped<<<(unsigned)((L.ca_threads + 127) / 128), 128, 0, s>>>(
        static_cast<const CATask*>(L.ca), L.nca, L.ca_threads);
    ++nk;
  }
  mark();
  return cudaPeekAtLastError() == cudaSuccess ? nk : -1;
}

}  // namespace lqc

// ---------------------------------------------------------------- C ABI
extern "C" {

int64_t lqc_contract_mixed_scratch_bytes(int rank_a, const int64_t* ext_a, int rank_b,
                                         const int64_t* ext_b, int npairs, const int* la,
                                         const int* ra, int64_t lt, lqc_precision prec) {
  if (!ext_a || !ext_b || !la || !ra || lt < 1) return 0;
  if (prec != LQC_PREC_TF32X3 && prec != LQC_PREC_BF16X3) return 0;
  lqc::ContractDesc cd;
  lqc::MixedDesc md;
  std::string err;
  if (!lqc::make_contract_desc(rank_a, ext_a, rank_b, ext_b, npairs, la, ra, lt, &cd, &err))
    return 0;
  if (!lqc::make_mixed_desc(cd, prec == LQC_PREC_BF16X3, &md)) return 0;
  return std::max<int64_t>(md.scratch_bytes, 256);  // 0 is reserved for errors
}

int lqc_contract_mixed(const float* A, int rank_a, const int64_t* ext_a, const float* B,
                       int rank_b, const int64_t* ext_b, int npairs, const int* la,
                       const int* ra, int64_t lt, lqc_precision prec, float* C, void* scratch,
                       void* stream) {
  if (!A || !B || !C || !scratch || !ext_a || !ext_b || !la || !ra || lt < 1) return LQC_ERR_ARG;
  if (prec != LQC_PREC_TF32X3 && prec != LQC_PREC_BF16X3) return LQC_ERR_ARG;
  lqc::ContractDesc cd;
  lqc::MixedDesc md;
  std::string err;
  if (!lqc::make_contract_desc(rank_a, ext_a, rank_b, ext_b, npairs, la, ra, lt, &cd, &err))
    return LQC_ERR_ARG;
  if (!lqc::make_mixed_desc(cd, prec == LQC_PREC_BF16X3, &md)) return LQC_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(scratch) & 255) != 0) return LQC_ERR_ARG;
  lqc::clear_pending_error();
  int k = lqc::launch_contract_mixed(md, A, B, C, scratch, static_cast<cudaStream_t>(stream));
  return lqc::launch_status(k);
}

int lqc_contract_all_c64(const float* A, int rank_a, const int64_t* ext_a, const float* B,
                         int rank_b, const int64_t* ext_b, int npairs, const int* la,
                         const int* ra, int64_t lt, double scale, double* C, void* scratch,
                         void* stream) {
  if (!A || !B || !C || !scratch || !ext_a || !ext_b || !la || !ra || lt < 1) return LQC_ERR_ARG;
  lqc::ContractAllDesc d;
  std::string err;
  if (!lqc::make_contract_all_desc(rank_a, ext_a, rank_b, ext_b, npairs, la, ra, lt, &d, &err))
    return LQC_ERR_ARG;
  lqc::clear_pending_error();
  int k = lqc::launch_contract_all_c64(d, A, B, C, static_cast<double*>(scratch), scale,
                                       static_cast<cudaStream_t>(stream));
  return lqc::launch_status(k);
}

int64_t lqc_contract_all_c64_scratch_bytes(int rank_a, const int64_t* ext_a, int rank_b,
                                           const int64_t* ext_b, int npairs, const int* la,
                                           const int* ra, int64_t lt) {
  if (!ext_a || !ext_b || !la || !ra || lt < 1) return 0;
  lqc::ContractAllDesc d;
  std::string err;
  if (!lqc::make_contract_all_desc(rank_a, ext_a, rank_b, ext_b, npairs, la, ra, lt, &d, &err))
    return 0;
  return lqc::contract_all_c64_scratch_bytes(d);
}

int lqc_mixed_error(int reset) { return lqc::mixed_error_status(reset != 0); }

int lqc_test_tf32_rounding(int64_t n, uint32_t seed, int64_t* mismatches) {
  if (n < 1 || !mismatches) return LQC_ERR_ARG;
  lqc::clear_pending_error();
  unsigned long long* bad = nullptr;
  if (cudaMalloc(&bad, sizeof(unsigned long long)) != cudaSuccess) return LQC_ERR_CUDA;
  unsigned long long h = 0;
  int rc = LQC_OK;
  if (cudaMemset(bad, 0, sizeof(h)) != cudaSuccess) rc = LQC_ERR_CUDA;
  if (rc == LQC_OK) {
    lqc::k_tf32_rounding_check<<<4 * 148, 256>>>((long long)n, seed, bad);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = LQC_ERR_CUDA;
  }
  cudaFree(bad);
  if (rc == LQC_OK) *mismatches = (int64_t)h;
  return rc;
}

int lqc_test_expire_wait(int64_t limit_ns, void* stream) {
  if (limit_ns < 1 || limit_ns > 1000000000) return LQC_ERR_ARG;
  lqc::clear_pending_error();
  if (lqc::mixed_error_status(true) < 0) return LQC_ERR_CUDA;  // start from a clear word
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lqc::k_wait_probe<<<1, 32, 0, s>>>((unsigned long long)limit_ns);
  if (cudaGetLastError() != cudaSuccess) return LQC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LQC_ERR_CUDA;
  const int st = lqc::mixed_error_status(true);
  return st < 0 ? LQC_ERR_CUDA : (st ? LQC_ERR_TIMEOUT : LQC_OK);
}

}  // extern "C"
