// FP64 kernels of the plain path.
//
// K1  exterior contraction: one binary contraction of the DAG (Sec. II-B) as
//     a batched complex GEMM whose operand gathers follow the tensors' own
//     strides, so index permutations are folded into the tile loads (no
//     transposed copies).  B300 executes FP64 FMAs at about 1/60 of its FP32
//     rate, so this kernel is bound by the FP64 pipe; the tile loop keeps that
//     pipe fed (register-blocked complex MACs, smem-staged operand tiles,
//     register prefetch of the next k-slab).
// K2  contract-all (a root's "contract all" (HCA), Sec. II-A): per time slice the
//     full pairing sum of two tensors, FP64 accumulation in a fixed order:
//     per-CTA partials in scratch memory, then an ordered per-slice sum.
#include <algorithm>
#include <cstring>

#include "kernels.hpp"

namespace lqc {

namespace {

constexpr int kThreads = 256;
constexpr int kBK = 16;

__device__ __forceinline__ long long group_off(const Group& g, unsigned idx) {
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

__device__ __forceinline__ void cmac(double2& acc, const double2 a, const double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// C tile of (16*TM) x (16*TN) complex outputs per CTA, 16x16 threads, each
// thread a TM x TN register block; k-slabs of kBK staged in shared memory.
template <int TM, int TN>
__global__ void __launch_bounds__(kThreads)
k_contract_fp64(const double2* __restrict__ A, const double2* __restrict__ B,
                double2* __restrict__ C, const ContractDesc p) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  __shared__ double2 As[kBK][BM + 1];
  __shared__ double2 Bs[kBK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long long t = blockIdx.z;
  const unsigned m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const unsigned M = (unsigned)p.M, N = (unsigned)p.N, K = (unsigned)p.K;
  A += t * p.a_ts;
  B += t * p.b_ts;

  // fixed part of this thread's load coordinates
  int a_mm[TM], a_kk[TM], b_nn[TN], b_kk[TN];
  long long a_moff[TM], b_noff[TN];
#pragma unroll
  for (int j = 0; j < TM; ++j) {
    int e = tid + j * kThreads;
    if (p.a_kfast) { a_kk[j] = e % kBK; a_mm[j] = e / kBK; }
    else { a_mm[j] = e % BM; a_kk[j] = e / BM; }
    unsigned m = m0 + a_mm[j];
    a_moff[j] = m < M ? group_off(p.am, m) : 0;
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    int e = tid + j * kThreads;
    if (p.b_kfast) { b_kk[j] = e % kBK; b_nn[j] = e / kBK; }
    else { b_nn[j] = e % BN; b_kk[j] = e / BN; }
    unsigned n = n0 + b_nn[j];
    b_noff[j] = n < N ? group_off(p.bn, n) : 0;
  }

  double2 ra[TM], rb[TN];
  auto load_slab = [&](unsigned k0) {
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      unsigned m = m0 + a_mm[j], k = k0 + a_kk[j];
      ra[j] = (m < M && k < K) ? A[a_moff[j] + group_off(p.ak, k)] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      unsigned n = n0 + b_nn[j], k = k0 + b_kk[j];
      rb[j] = (n < N && k < K) ? B[b_noff[j] + group_off(p.bk, k)] : make_double2(0.0, 0.0);
    }
  };

  double2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = make_double2(0.0, 0.0);

  load_slab(0);
  for (unsigned k0 = 0; k0 < K; k0 += kBK) {
#pragma unroll
    for (int j = 0; j < TM; ++j) As[a_kk[j]][a_mm[j]] = ra[j];
#pragma unroll
    for (int j = 0; j < TN; ++j) Bs[b_kk[j]][b_nn[j]] = rb[j];
    __syncthreads();
    if (k0 + kBK < K) load_slab(k0 + kBK);  // prefetch overlaps the MACs below
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      double2 a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cmac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  double2* Ct = C + t * (long long)M * N;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    unsigned m = m0 + ty * TM + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      unsigned n = n0 + tx * TN + j;
      if (n < N) Ct[(long long)m * N + n] = acc[i][j];
    }
  }
}

// Per-CTA partial sums of one slice's pairing sum, fixed reduction order.
__global__ void __launch_bounds__(kThreads)
k_contract_all_partial(const double2* __restrict__ A, const double2* __restrict__ B,
                       double2* __restrict__ part, const ContractAllDesc p) {
  const long long t = blockIdx.y;
  const int c = blockIdx.x;
  const unsigned S = (unsigned)p.S;
  const unsigned lo = (unsigned)(((unsigned long long)S * c) / p.chunks);
  const unsigned hi = (unsigned)(((unsigned long long)S * (c + 1)) / p.chunks);
  A += t * p.S;
  B += t * p.S;
  double re = 0.0, im = 0.0;
  for (unsigned i = lo + threadIdx.x; i < hi; i += kThreads) {
    double2 a = A[i];
    double2 b = B[group_off(p.bp, i)];
    re = fma(a.x, b.x, re);
    re = fma(-a.y, b.y, re);
    im = fma(a.x, b.y, im);
    im = fma(a.y, b.x, im);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  __shared__ double2 w[kThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = make_double2(re, im);
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = w[0];
    for (int k = 1; k < kThreads / 32; ++k) { s.x += w[k].x; s.y += w[k].y; }
    part[t * p.chunks + c] = s;
  }
}

__global__ void k_contract_all_final(const double2* __restrict__ part, double2* __restrict__ C,
                                     long long lt, int chunks) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= lt) return;
  double2 s = make_double2(0.0, 0.0);
  for (int c = 0; c < chunks; ++c) {
    double2 v = part[t * chunks + c];
    s.x += v.x;
    s.y += v.y;
  }
  C[t] = s;
}

// Register-resident FMA chains (8 independent per thread) for the FP64
// throughput probe.
__global__ void k_fma_probe(double* out, int iters, double a, double b) {
  double acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = (double)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += acc[c];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_fill_nan(unsigned long long* p, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = 0x7FF8000000000000ull;
}

void row_major_strides(int rank, const int64_t* ext, long long* st) {
  long long s = 1;
  for (int a = rank - 1; a >= 0; --a) {
    st[a] = s;
    s *= ext[a];
  }
}

// merge neighbouring axes of a group that are contiguous with each other
void merge_group(Group* g) {
  int w = 0;
  for (int r = 0; r < g->n; ++r) {
    if (w > 0 && g->stride[w - 1] == g->stride[r] * (long long)g->ext[r]) {
      g->ext[w - 1] *= g->ext[r];
      g->stride[w - 1] = g->stride[r];
    } else {
      g->ext[w] = g->ext[r];
      g->stride[w] = g->stride[r];
      ++w;
    }
  }
  g->n = w;
}

bool check_pairs(int rank_a, const int64_t* ext_a, int rank_b, const int64_t* ext_b, int npairs,
                 const int* la, const int* ra, std::string* err) {
  if (rank_a < 1 || rank_b < 1 || rank_a > LQC_MAX_RANK || rank_b > LQC_MAX_RANK) {
    *err = "operand rank must be in [1, LQC_MAX_RANK]";
    return false;
  }
  if (npairs < 1 || npairs > LQC_MAX_RANK) {
    *err = "npairs out of range";
    return false;
  }
  bool ua[LQC_MAX_RANK] = {false}, ub[LQC_MAX_RANK] = {false};
  for (int j = 0; j < npairs; ++j) {
    if (la[j] < 0 || la[j] >= rank_a || ra[j] < 0 || ra[j] >= rank_b || ua[la[j]] || ub[ra[j]] ||
        ext_a[la[j]] != ext_b[ra[j]]) {
      *err = "invalid axis pairing";
      return false;
    }
    ua[la[j]] = ub[ra[j]] = true;
  }
  for (int a = 0; a < rank_a; ++a)
    if (ext_a[a] < 1) { *err = "extent < 1"; return false; }
  for (int b = 0; b < rank_b; ++b)
    if (ext_b[b] < 1) { *err = "extent < 1"; return false; }
  return true;
}

}  // namespace

bool make_contract_desc(int rank_a, const int64_t* ext_a, int rank_b, const int64_t* ext_b,
                        int npairs, const int* la, const int* ra, int64_t lt, ContractDesc* d,
                        std::string* err) {
  if (!check_pairs(rank_a, ext_a, rank_b, ext_b, npairs, la, ra, err)) return false;
  if (rank_a + rank_b - 2 * npairs < 1) {
    *err = "rank-0 output: use the contract-all kernel";
    return false;
  }
  long long sa[LQC_MAX_RANK], sb[LQC_MAX_RANK];
  row_major_strides(rank_a, ext_a, sa);
  row_major_strides(rank_b, ext_b, sb);
  bool pa[LQC_MAX_RANK] = {false}, pb[LQC_MAX_RANK] = {false};
  for (int j = 0; j < npairs; ++j) pa[la[j]] = pb[ra[j]] = true;
  std::memset(d, 0, sizeof(*d));
  d->lt = lt;
  d->M = d->N = d->K = 1;
  d->a_ts = d->b_ts = 1;
  for (int a = 0; a < rank_a; ++a) d->a_ts *= ext_a[a];
  for (int b = 0; b < rank_b; ++b) d->b_ts *= ext_b[b];
  for (int a = 0; a < rank_a; ++a)
    if (!pa[a]) {
      d->am.ext[d->am.n] = (int)ext_a[a];
      d->am.stride[d->am.n++] = sa[a];
      d->M *= ext_a[a];
    }
  for (int b = 0; b < rank_b; ++b)
    if (!pb[b]) {
      d->bn.ext[d->bn.n] = (int)ext_b[b];
      d->bn.stride[d->bn.n++] = sb[b];
      d->N *= ext_b[b];
    }
  // paired axes in pair order (k runs row-major over the pairs); each side
  // merges the neighbours that are contiguous on that side, so one operand
  // can be a single k group while the other is not (both still enumerate k
  // in the same order)
  d->ak.n = d->bk.n = npairs;
  for (int j = 0; j < npairs; ++j) {
    const int e = (int)ext_a[la[j]];
    d->ak.ext[j] = d->bk.ext[j] = e;
    d->ak.stride[j] = sa[la[j]];
    d->bk.stride[j] = sb[ra[j]];
    d->K *= e;
  }
  merge_group(&d->ak);
  merge_group(&d->bk);
  merge_group(&d->am);
  merge_group(&d->bn);
  d->a_kfast = pa[rank_a - 1] ? 1 : 0;
  d->b_kfast = pb[rank_b - 1] ? 1 : 0;
  if (d->M >= (1ll << 31) || d->N >= (1ll << 31) || d->K >= (1ll << 31)) {
    *err = "contraction extents exceed 2^31";
    return false;
  }
  return true;
}

int contract_all_chunks(int64_t lt, int64_t S) {
  // enough CTAs to cover the SMs a few times, at least 2048 elements each
  int64_t want = (4 * 148 + lt - 1) / lt;
  int64_t most = std::max<int64_t>(1, S / 2048);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, most));
}

bool make_contract_all_desc(int rank_a, const int64_t* ext_a, int rank_b, const int64_t* ext_b,
                            int npairs, const int* la, const int* ra, int64_t lt,
                            ContractAllDesc* d, std::string* err) {
  if (!check_pairs(rank_a, ext_a, rank_b, ext_b, npairs, la, ra, err)) return false;
  if (npairs != rank_a || npairs != rank_b) {
    *err = "contract-all needs every axis paired";
    return false;
  }
  long long sb[LQC_MAX_RANK];
  row_major_strides(rank_b, ext_b, sb);
  std::memset(d, 0, sizeof(*d));
  d->lt = lt;
  d->S = 1;
  for (int a = 0; a < rank_a; ++a) {
    int j = 0;
    while (la[j] != a) ++j;
    d->bp.ext[d->bp.n] = (int)ext_a[a];
    d->bp.stride[d->bp.n++] = sb[ra[j]];
    d->S *= ext_a[a];
  }
  merge_group(&d->bp);
  if (d->S >= (1ll << 31)) {
    *err = "contract-all extent exceeds 2^31";
    return false;
  }
  d->chunks = contract_all_chunks(lt, d->S);
  return true;
}

int64_t contract_all_scratch_bytes(const ContractAllDesc& d) {
  return d.lt * (int64_t)d.chunks * 16;
}

int launch_contract_fp64(const ContractDesc& d, const double* A, const double* B, double* C,
                         cudaStream_t s) {
  auto ctas = [&](int bm, int bn) {
    return ((d.M + bm - 1) / bm) * ((d.N + bn - 1) / bn) * d.lt;
  };
  const double2* a = reinterpret_cast<const double2*>(A);
  const double2* b = reinterpret_cast<const double2*>(B);
  double2* c = reinterpret_cast<double2*>(C);
  if (d.lt > 65535) return -1;
  if (d.M >= 64 && d.N >= 64 && ctas(64, 64) >= 4 * 148) {
    dim3 grid((unsigned)((d.N + 63) / 64), (unsigned)((d.M + 63) / 64), (unsigned)d.lt);
    k_contract_fp64<4, 4><<<grid, kThreads, 0, s>>>(a, b, c, d);
  } else if (d.M >= 32 && d.N >= 32 && ctas(32, 32) >= 2 * 148) {
    dim3 grid((unsigned)((d.N + 31) / 32), (unsigned)((d.M + 31) / 32), (unsigned)d.lt);
    k_contract_fp64<2, 2><<<grid, kThreads, 0, s>>>(a, b, c, d);
  } else {
    dim3 grid((unsigned)((d.N + 15) / 16), (unsigned)((d.M + 15) / 16), (unsigned)d.lt);
    k_contract_fp64<1, 1><<<grid, kThreads, 0, s>>>(a, b, c, d);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_contract_all_fp64(const ContractAllDesc& d, const double* A, const double* B,
                             double* C, double* scratch, cudaStream_t s) {
  if (d.lt > 65535) return -1;
  dim3 grid((unsigned)d.chunks, (unsigned)d.lt);
  double2* part = reinterpret_cast<double2*>(scratch);
  k_contract_all_partial<<<grid, kThreads, 0, s>>>(reinterpret_cast<const double2*>(A),
                                                    reinterpret_cast<const double2*>(B), part, d);
  k_contract_all_final<<<(unsigned)((d.lt + 127) / 128), 128, 0, s>>>(
      part, reinterpret_cast<double2*>(C), d.lt, d.chunks);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

int launch_fill_nan(void* p, int64_t bytes, cudaStream_t s) {
  long long n = bytes / 8;
  if (n <= 0) return 0;
  unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 4 * 148);
  k_fill_nan<<<blocks, 256, 0, s>>>(static_cast<unsigned long long*>(p), n);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace lqc

// ---------------------------------------------------------------- C ABI
extern "C" {

int lqc_contract_fp64(const double* A, int rank_a, const int64_t* ext_a, const double* B,
                      int rank_b, const int64_t* ext_b, int npairs, const int* la, const int* ra,
                      int64_t lt, double* C, void* stream) {
  if (!A || !B || !C || !ext_a || !ext_b || !la || !ra || lt < 1) return LQC_ERR_ARG;
  lqc::ContractDesc d;
  std::string err;
  if (!lqc::make_contract_desc(rank_a, ext_a, rank_b, ext_b, npairs, la, ra, lt, &d, &err))
    return LQC_ERR_ARG;
  lqc::clear_pending_error();
  int k = lqc::launch_contract_fp64(d, A, B, C, static_cast<cudaStream_t>(stream));
  return lqc::launch_status(k);
}

int lqc_measure_fp64_peak(double* tflops) {
  if (!tflops) return LQC_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LQC_ERR_CUDA;
  const int blocks = sms * 8, threads = 256, iters = 2048;
  double* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LQC_ERR_CUDA;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) == cudaSuccess &&
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, s);
      lqc::k_fma_probe<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);
    }
    if (cudaGetLastError() == cudaSuccess && best < 1e29f) {
      *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
      rc = LQC_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  return rc;
}

int64_t lqc_contract_all_scratch_bytes(int64_t lt, int64_t elems_per_slice) {
  if (lt < 1 || elems_per_slice < 1) return 0;
  return lt * (int64_t)lqc::contract_all_chunks(lt, elems_per_slice) * 16;
}

int lqc_contract_all_fp64(const double* A, int rank_a, const int64_t* ext_a, const double* B,
                          int rank_b, const int64_t* ext_b, int npairs, const int* la,
                          const int* ra, int64_t lt, double* C, void* scratch, void* stream) {
  if (!A || !B || !C || !scratch || !ext_a || !ext_b || !la || !ra || lt < 1) return LQC_ERR_ARG;
  lqc::ContractAllDesc d;
  std::string err;
  if (!lqc::make_contract_all_desc(rank_a, ext_a, rank_b, ext_b, npairs, la, ra, lt, &d, &err))
    return LQC_ERR_ARG;
  lqc::clear_pending_error();
  int k = lqc::launch_contract_all_fp64(d, A, B, C, static_cast<double*>(scratch),
                                         static_cast<cudaStream_t>(stream));
  return lqc::launch_status(k);
}

}  // extern "C"
