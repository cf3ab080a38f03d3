// C ABI: DAG construction with merging of identical requests (Sec. II-B),
// scheduling + planning, and the thin wrappers around the executor.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <string>

#include "internal.hpp"

#include <system_error>
#include <thread>
#include <type_traits>
#include <vector>

namespace {
// Host passes over leaf data (normalisation, conversion, copies): the range
// [0, n) in contiguous chunks on up to kMaxHostThreads threads (one chunk per
// thread, at least 2^20 values each); f(a, b) or f(a, b, chunk index).
constexpr int kMaxHostThreads = 32;
template <typename F>
void parallel_chunks(int64_t n, F f) {
  const int64_t per_min = 1 << 17;
  int t = (int)std::min<int64_t>(kMaxHostThreads, std::max<int64_t>(1, n / per_min));
  t = std::min<int>(t, std::max(1u, std::thread::hardware_concurrency()));
  auto call = [&](int64_t a, int64_t b, int i) {
    if constexpr (std::is_invocable_v<F, int64_t, int64_t, int>) f(a, b, i);
    else f(a, b);
  };
  if (t <= 1) {
    call(0, n, 0);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(t - 1);
  const int64_t per = (n + t - 1) / t;
  int started = 1;
  try {
    for (int i = 1; i < t; ++i, ++started) {
      const int64_t a = std::min(n, i * per), b = std::min(n, a + per);
      th.emplace_back(call, a, b, i);
    }
  } catch (const std::system_error&) {
    // no more threads: the calling thread takes the chunks not started
  }
  call(0, std::min(n, per), 0);
  for (int i = started; i < t; ++i) {
    const int64_t a = std::min(n, i * per), b = std::min(n, a + per);
    call(a, b, i);
  }
  for (auto& x : th) x.join();
}
}  // namespace

using lqc::Dag;
using lqc::Node;

namespace {

int fail(lqc_dag* h, int code, const std::string& msg) {
  if (h) h->d.err = msg;
  return code;
}

#define LQC_GUARD_BEGIN try {
#define LQC_GUARD_END(h)                                                  \
  }                                                                       \
  catch (const std::bad_alloc&) {                                         \
    return fail(h, LQC_ERR_HOST_MEM, "host allocation failed");           \
  }                                                                       \
  catch (const std::exception& e) {                                       \
    return fail(h, LQC_ERR_ARG, std::string("internal error: ") + e.what()); \
  }

std::string dedup_key(int64_t l, int64_t r, int np, const int* la, const int* ra) {
  std::string k;
  k.append(reinterpret_cast<const char*>(&l), sizeof l);
  k.append(reinterpret_cast<const char*>(&r), sizeof r);
  k.append(reinterpret_cast<const char*>(&np), sizeof np);
  k.append(reinterpret_cast<const char*>(la), sizeof(int) * np);
  k.append(reinterpret_cast<const char*>(ra), sizeof(int) * np);
  return k;
}

int finish_schedule(lqc_dag* h, std::vector<int64_t>&& order, lqc_evict evict,
                    uint64_t budget, lqc_stats* planned) {
  Dag& g = h->d;
  std::vector<lqc::Op> ops;
  lqc_stats st{};
  std::string err;
  lqc::exec_invalidate_plan(g);
  if (!lqc::plan_replay(g, order, budget, evict, &ops, &st, &err)) {
    g.scheduled = false;
    g.order.clear();
    g.ops.clear();
    return fail(h, LQC_ERR_BUDGET, err);
  }
  g.frozen = true;
  g.order = std::move(order);
  g.ops = std::move(ops);
  g.planned = st;
  g.budget = budget;
  g.evict = evict;
  g.scheduled = true;
  g.executed = false;
  if (planned) *planned = st;
  return LQC_OK;
}

template <typename T>
int copy_out(lqc_dag* h, const std::vector<T>& v, T* dst, int64_t cap, int64_t* n) {
  if (!n) return fail(h, LQC_ERR_ARG, "null length pointer");
  *n = (int64_t)v.size();
  if (cap < (int64_t)v.size() || (!dst && !v.empty())) {
    return fail(h, LQC_ERR_ARG, "output capacity too small");
  }
  if (!v.empty()) std::memcpy(dst, v.data(), sizeof(T) * v.size());
  return LQC_OK;
}

}  // namespace

// Size limits: a slice holds at most 2^40 elements; a tensor (all slices)
// at most 2^58, so byte sizes stay below 2^62; the batch extent fits the
// kernels' 32-bit slice index.
constexpr int64_t kMaxSliceElems = (int64_t)1 << 40;
constexpr int64_t kMaxTensorElems = (int64_t)1 << 58;
constexpr int64_t kMaxLt = ((int64_t)1 << 31) - 1;

namespace lqc {
namespace {
// per site: successful calls still to pass before the armed failure (-1 = none)
std::atomic<int64_t> g_inject_skip[INJ_SITES] = {{-1}, {-1}, {-1}};
}  // namespace

bool inject_fail(int site) {
  std::atomic<int64_t>& k = g_inject_skip[site];
  int64_t v = k.load();
  while (v >= 0) {
    if (k.compare_exchange_weak(v, v - 1)) return v == 0;  // 0 -> -1: this call fails
  }
  return false;
}
}  // namespace lqc

extern "C" {

int lqc_test_inject_failure(int site, int64_t skip_calls) {
  if (site == -1) {
    for (auto& k : lqc::g_inject_skip) k.store(-1);
    return LQC_OK;
  }
  if (site < 0 || site >= lqc::INJ_SITES || skip_calls < 0) return LQC_ERR_ARG;
  lqc::g_inject_skip[site].store(skip_calls);
  return LQC_OK;
}

int lqc_test_tamper_plan(lqc_dag* h, int what) {
  if (!h) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  Dag& g = h->d;
  if (!g.scheduled) return fail(h, LQC_ERR_STATE, "tamper before schedule");
  if (what != 1) return fail(h, LQC_ERR_ARG, "unknown plan change");
  // every FREE after all other ops, in their order: tensors stay resident to
  // the end (valid without a budget), the planned figures are kept
  if (g.budget != 0) return fail(h, LQC_ERR_ARG, "plan change needs an unlimited budget");
  std::stable_partition(g.ops.begin(), g.ops.end(),
                        [](const lqc::Op& op) { return op.kind != lqc::OP_FREE; });
  lqc::exec_invalidate_plan(g);
  return LQC_OK;
  LQC_GUARD_END(h)
}

int lqc_test_read_leaf_store(lqc_dag* h, int64_t id, void* out, int64_t cap_bytes,
                             int* scale_exp) {
  if (!h || !out || !scale_exp) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  Dag& g = h->d;
  if (id < 0 || id >= (int64_t)g.nodes.size() || !g.nodes[id].is_leaf())
    return fail(h, LQC_ERR_ARG, "not a leaf");
  const Node& n = g.nodes[id];
  if (!n.has_data || !n.host) return fail(h, LQC_ERR_STATE, "leaf has no data");
  const int64_t bytes = g.size_bytes(id);
  if (cap_bytes < bytes) return fail(h, LQC_ERR_ARG, "capacity too small");
  std::memcpy(out, n.host, (size_t)bytes);
  *scale_exp = n.scale_exp;
  return LQC_OK;
  LQC_GUARD_END(h)
}

int lqc_dag_create(lqc_dag** out, int64_t lt, lqc_precision prec) {
  if (!out || lt < 1 || lt > kMaxLt) return LQC_ERR_ARG;
  if (prec != LQC_PREC_FP64 && prec != LQC_PREC_TF32X3 && prec != LQC_PREC_BF16X3)
    return LQC_ERR_ARG;
  try {
    lqc_dag* h = new lqc_dag();
    h->d.lt = lt;
    h->d.prec = prec;
    h->d.elem_bytes = prec == LQC_PREC_FP64 ? 16 : 8;
    *out = h;
    return LQC_OK;
  } catch (...) {
    return LQC_ERR_HOST_MEM;
  }
}

int lqc_dag_set_batch(lqc_dag* h, int64_t lt) {
  if (!h) return LQC_ERR_ARG;
  if (h->d.frozen) return fail(h, LQC_ERR_STATE, "DAG is frozen by lqc_dag_schedule");
  if (lt < 1 || lt > kMaxLt) return fail(h, LQC_ERR_ARG, "batch extent must be in [1, 2^31)");
  h->d.lt = lt;
  return LQC_OK;
}

int lqc_dag_destroy(lqc_dag* h) {
  if (!h) return LQC_OK;
  lqc::exec_destroy(h->d);
  for (Node& n : h->d.nodes) lqc::host_store_free(n);
  delete h;
  return LQC_OK;
}

int lqc_dag_add_leaf_tensor(lqc_dag* h, int rank, const int64_t* extents, const double* data,
                            int64_t* node_id) {
  if (!h) return LQC_ERR_ARG;
  Dag& g = h->d;
  LQC_GUARD_BEGIN
  if (g.frozen) return fail(h, LQC_ERR_STATE, "DAG is frozen by lqc_dag_schedule");
  if (rank < 0 || rank > LQC_MAX_RANK || (rank > 0 && !extents) || !node_id)
    return fail(h, LQC_ERR_ARG, "bad leaf rank/extents");
  Node n;
  n.rank = rank;
  n.lt = g.lt;
  n.elems = 1;
  for (int i = 0; i < rank; ++i) {
    if (extents[i] < 1 || extents[i] > (int64_t)1 << 31)
      return fail(h, LQC_ERR_ARG, "leaf extent out of range");
    if (n.elems > kMaxSliceElems / extents[i]) return fail(h, LQC_ERR_ARG, "leaf too large");
    n.ext[i] = extents[i];
    n.elems *= extents[i];
  }
  if (n.elems > kMaxTensorElems / n.lt) return fail(h, LQC_ERR_ARG, "leaf too large");
  g.nodes.push_back(n);
  int64_t id = (int64_t)g.nodes.size() - 1;
  if (data) {
    int rc = lqc_dag_set_leaf_data(h, id, data);
    if (rc != LQC_OK) {
      g.nodes.pop_back();
      return rc;
    }
  }
  *node_id = id;
  return LQC_OK;
  LQC_GUARD_END(h)
}

int lqc_dag_add_contraction(lqc_dag* h, int64_t left, int64_t right, int npairs, const int* la,
                            const int* ra, int64_t* node_id) {
  if (!h) return LQC_ERR_ARG;
  Dag& g = h->d;
  LQC_GUARD_BEGIN
  if (g.frozen) return fail(h, LQC_ERR_STATE, "DAG is frozen by lqc_dag_schedule");
  const int64_t N = (int64_t)g.nodes.size();
  if (!node_id || left < 0 || right < 0 || left >= N || right >= N)
    return fail(h, LQC_ERR_ARG, "operand id out of range");
  if (npairs < 1 || npairs > LQC_MAX_RANK || !la || !ra)
    return fail(h, LQC_ERR_ARG, "npairs must be in [1, LQC_MAX_RANK]");
  const Node& L = g.nodes[left];
  const Node& R = g.nodes[right];
  if (L.rank == 0 || R.rank == 0)
    return fail(h, LQC_ERR_ARG, "a rank-0 correlator cannot be an operand");
  if (L.lt != R.lt) return fail(h, LQC_ERR_ARG, "operands differ in the batch extent");
  bool usedL[LQC_MAX_RANK] = {false}, usedR[LQC_MAX_RANK] = {false};
  for (int i = 0; i < npairs; ++i) {
    if (la[i] < 0 || la[i] >= L.rank || ra[i] < 0 || ra[i] >= R.rank)
      return fail(h, LQC_ERR_ARG, "axis index out of range");
    if (usedL[la[i]] || usedR[ra[i]]) return fail(h, LQC_ERR_ARG, "axis paired twice");
    usedL[la[i]] = usedR[ra[i]] = true;
    if (L.ext[la[i]] != R.ext[ra[i]]) return fail(h, LQC_ERR_ARG, "paired extents differ");
  }
  const int out_rank = L.rank + R.rank - 2 * npairs;
  if (out_rank > LQC_MAX_RANK) return fail(h, LQC_ERR_ARG, "output rank too large");
  std::string key = dedup_key(left, right, npairs, la, ra);
  auto it = g.dedup.find(key);
  if (it != g.dedup.end()) {
    *node_id = it->second;
    return LQC_OK;
  }
  Node n;
  n.left = left;
  n.right = right;
  n.npairs = npairs;
  for (int i = 0; i < npairs; ++i) {
    n.la[i] = la[i];
    n.ra[i] = ra[i];
  }
  n.scale_exp = L.scale_exp + R.scale_exp;
  n.lt = L.lt;
  n.rank = 0;
  n.elems = 1;
  bool fits = true;
  auto take = [&](int64_t e) {
    n.ext[n.rank++] = e;
    if (n.elems > kMaxSliceElems / e) fits = false;
    else n.elems *= e;
  };
  for (int a = 0; a < L.rank; ++a)
    if (!usedL[a]) take(L.ext[a]);
  for (int b = 0; b < R.rank; ++b)
    if (!usedR[b]) take(R.ext[b]);
  if (!fits || n.elems > kMaxTensorElems / n.lt) return fail(h, LQC_ERR_ARG, "output too large");
  g.nodes.push_back(n);
  const int64_t id = N;
  g.nodes[left].parents.push_back(id);
  if (right != left) g.nodes[right].parents.push_back(id);
  g.dedup.emplace(std::move(key), id);
  *node_id = id;
  return LQC_OK;
  LQC_GUARD_END(h)
}

int lqc_dag_add_contractions(lqc_dag* h, int64_t n, const int64_t* left, const int64_t* right,
                             const int* npairs, const int* la, const int* ra, int64_t* node_ids) {
  if (!h) return LQC_ERR_ARG;
  Dag& g = h->d;
  if (n < 0 || (n > 0 && (!left || !right || !npairs || !la || !ra || !node_ids)))
    return fail(h, LQC_ERR_ARG, "null or negative request arrays");
  const int64_t n0 = (int64_t)g.nodes.size();
  int64_t at = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int np = npairs[i];
    // -(j+1): the node request j of this call received
    // (x >= -i before negating: -x of INT64_MIN would overflow)
    auto resolve = [&](int64_t x) { return x >= 0 ? x : (x >= -i ? node_ids[-(x + 1)] : -1); };
    const int64_t l = resolve(left[i]), r = resolve(right[i]);
    const int rc = np < 1 || np > LQC_MAX_RANK
                       ? fail(h, LQC_ERR_ARG, "npairs must be in [1, LQC_MAX_RANK]")
                       : lqc_dag_add_contraction(h, l, r, np, la + at, ra + at, &node_ids[i]);
    if (rc != LQC_OK) {
      // remove what this call added, newest first (each is the last
      // consumer of its operands and owns one merge entry)
      for (int64_t u = (int64_t)g.nodes.size() - 1; u >= n0; --u) {
        const Node& nu = g.nodes[u];
        for (int c = 0; c < nu.n_children(); ++c) {
          auto& par = g.nodes[nu.child(c)].parents;
          if (!par.empty() && par.back() == u) par.pop_back();
        }
        g.nodes.pop_back();
      }
      for (auto it = g.dedup.begin(); it != g.dedup.end();)
        it = it->second >= n0 ? g.dedup.erase(it) : std::next(it);
      g.err = "request " + std::to_string(i) + ": " + g.err;
      return rc;
    }
    at += np;
  }
  return LQC_OK;
}

int lqc_dag_schedule(lqc_dag* h, lqc_policy policy, lqc_evict evict, uint64_t budget_bytes,
                     lqc_stats* planned) {
  if (!h) return LQC_ERR_ARG;
  Dag& g = h->d;
  LQC_GUARD_BEGIN
  if (evict != LQC_EVICT_LRU && evict != LQC_EVICT_NEXT_USE)
    return fail(h, LQC_ERR_ARG, "unknown eviction policy");
  std::vector<int64_t> order;
  switch (policy) {
    case LQC_SCHED_NAIVE_TOPO: order = lqc::schedule_naive(g); break;
    case LQC_SCHED_TREE: order = lqc::schedule_tree(g); break;
    case LQC_SCHED_SIBLING: order = lqc::schedule_sibling(g); break;
    case LQC_SCHED_NODE: order = lqc::schedule_node(g); break;
    case LQC_SCHED_RSGS: order = lqc::schedule_rsgs(g); break;
    default: return fail(h, LQC_ERR_ARG, "unknown scheduling policy");
  }
  return finish_schedule(h, std::move(order), evict, budget_bytes, planned);
  LQC_GUARD_END(h)
}

int lqc_dag_set_order(lqc_dag* h, const int64_t* order, int64_t n, lqc_evict evict,
                      uint64_t budget_bytes, lqc_stats* planned) {
  if (!h) return LQC_ERR_ARG;
  Dag& g = h->d;
  LQC_GUARD_BEGIN
  if (evict != LQC_EVICT_LRU && evict != LQC_EVICT_NEXT_USE)
    return fail(h, LQC_ERR_ARG, "unknown eviction policy");
  const int64_t N = (int64_t)g.nodes.size();
  int64_t n_contr = 0;
  for (const Node& x : g.nodes) n_contr += x.is_leaf() ? 0 : 1;
  if (n != n_contr || (n > 0 && !order)) return fail(h, LQC_ERR_ARG, "order length mismatch");
  std::vector<uint8_t> done(N, 0);
  for (int64_t i = 0; i < n; ++i) {
    int64_t u = order[i];
    if (u < 0 || u >= N || g.nodes[u].is_leaf() || done[u])
      return fail(h, LQC_ERR_ARG, "order entry invalid or repeated");
    const Node& x = g.nodes[u];
    for (int k = 0; k < x.n_children(); ++k) {
      int64_t c = x.child(k);
      if (!g.nodes[c].is_leaf() && !done[c]) return fail(h, LQC_ERR_ARG, "order not topological");
    }
    done[u] = 1;
  }
  return finish_schedule(h, std::vector<int64_t>(order, order + n), evict, budget_bytes, planned);
  LQC_GUARD_END(h)
}

int lqc_dag_get_order(lqc_dag* h, int64_t* order, int64_t cap, int64_t* n) {
  if (!h) return LQC_ERR_ARG;
  if (!h->d.scheduled) return fail(h, LQC_ERR_STATE, "not scheduled");
  return copy_out(h, h->d.order, order, cap, n);
}

int lqc_dag_get_plan(lqc_dag* h, int32_t* kind, int64_t* node, int32_t* flag, int64_t cap,
                     int64_t* n) {
  if (!h) return LQC_ERR_ARG;
  Dag& g = h->d;
  if (!g.scheduled) return fail(h, LQC_ERR_STATE, "not scheduled");
  if (!n) return fail(h, LQC_ERR_ARG, "null length pointer");
  *n = (int64_t)g.ops.size();
  if (cap < (int64_t)g.ops.size() || (!g.ops.empty() && (!kind || !node || !flag)))
    return fail(h, LQC_ERR_ARG, "output capacity too small");
  for (size_t k = 0; k < g.ops.size(); ++k) {
    kind[k] = g.ops[k].kind;
    node[k] = g.ops[k].node;
    flag[k] = g.ops[k].flag;
  }
  return LQC_OK;
}

int lqc_dag_set_option(lqc_dag* h, int option, int64_t value) {
  if (!h) return LQC_ERR_ARG;
  switch (option) {
    case LQC_OPT_CUDA_GRAPH: h->d.opt_graph = value ? 1 : 0; break;
    case LQC_OPT_POISON: h->d.opt_poison = value ? 1 : 0; break;
    case LQC_OPT_TIMING: h->d.opt_timing = value ? 1 : 0; break;
    case LQC_OPT_WINDOW:
      if (value < 0 || value > 4096) return fail(h, LQC_ERR_ARG, "window size out of range");
      h->d.opt_window = value;
      break;
    case LQC_OPT_FUSED_MAX_N:
      if (value < 0) return fail(h, LQC_ERR_ARG, "fused-form limit must be >= 0");
      h->d.opt_fused_max_n = value;
      break;
    case LQC_OPT_SPLIT_POLICY:
      if (value != 0 && value != 1) return fail(h, LQC_ERR_ARG, "split policy must be 0 or 1");
      h->d.opt_split_policy = value;
      break;
    case LQC_OPT_FUSED_KERNEL:
      if (value < 0 || value > 2) return fail(h, LQC_ERR_ARG, "fused kernel must be 0, 1 or 2");
      h->d.opt_fused_kernel = value;
      break;
    default: return fail(h, LQC_ERR_ARG, "unknown option");
  }
  lqc::exec_invalidate_plan(h->d);
  return LQC_OK;
}

int lqc_dag_get_roots(lqc_dag* h, int64_t* roots, int64_t cap, int64_t* n) {
  if (!h) return LQC_ERR_ARG;
  std::vector<int64_t> r;
  for (int64_t u = 0; u < (int64_t)h->d.nodes.size(); ++u) {
    const Node& x = h->d.nodes[u];
    if (!x.is_leaf() && x.parents.empty() && x.rank == 0) r.push_back(u);
  }
  return copy_out(h, r, roots, cap, n);
}

int lqc_dag_num_nodes(lqc_dag* h, int64_t* n) {
  if (!h || !n) return LQC_ERR_ARG;
  *n = (int64_t)h->d.nodes.size();
  return LQC_OK;
}

int lqc_dag_node_info(lqc_dag* h, int64_t id, int64_t* size_bytes, int* rank, int* is_leaf,
                      int64_t* lt) {
  if (!h) return LQC_ERR_ARG;
  if (id < 0 || id >= (int64_t)h->d.nodes.size()) return fail(h, LQC_ERR_ARG, "id out of range");
  if (size_bytes) *size_bytes = h->d.size_bytes(id);
  if (lt) *lt = h->d.nodes[id].lt;
  if (rank) *rank = h->d.nodes[id].rank;
  if (is_leaf) *is_leaf = h->d.nodes[id].is_leaf() ? 1 : 0;
  return LQC_OK;
}

int lqc_dag_node_operands(lqc_dag* h, int64_t id, int64_t* left, int64_t* right, int* npairs,
                          int* la, int* ra) {
  if (!h) return LQC_ERR_ARG;
  if (id < 0 || id >= (int64_t)h->d.nodes.size()) return fail(h, LQC_ERR_ARG, "id out of range");
  const Node& n = h->d.nodes[id];
  if (left) *left = n.left;
  if (right) *right = n.right;
  if (npairs) *npairs = n.npairs;
  for (int i = 0; i < n.npairs; ++i) {
    if (la) la[i] = n.la[i];
    if (ra) ra[i] = n.ra[i];
  }
  return LQC_OK;
}

int lqc_dag_set_leaf_data(lqc_dag* h, int64_t id, const double* data) {
  if (!h) return LQC_ERR_ARG;
  Dag& g = h->d;
  LQC_GUARD_BEGIN
  if (id < 0 || id >= (int64_t)g.nodes.size() || !g.nodes[id].is_leaf() || !data)
    return fail(h, LQC_ERR_ARG, "not a leaf / null data");
  int rc = lqc::exec_wait(g, 60000);
  if (rc != LQC_OK) return rc;
  std::string err;
  rc = lqc::host_store_alloc(g, id, &err);
  if (rc != LQC_OK) return fail(h, rc, err);
  Node& n = g.nodes[id];
  const int64_t cnt = n.lt * n.elems;  // complex values
  const int64_t nv = 2 * cnt;          // real components
  bool rescaled = false;
  if (g.prec == LQC_PREC_FP64) {
    parallel_chunks(nv, [&](int64_t a, int64_t b) {
      std::memcpy(static_cast<double*>(n.host) + a, data + a, (size_t)(b - a) * 8);
    });
  } else {
    // complex64 storage with FP64 normalisation: scale by the power of two
    // that brings the largest |component| into [0.5, 1), then round once
    // (x * 2^-e in FP64 is exact, as ldexp).  New data of a leaf keeps its
    // exponent while its largest component stays within (2^(e-32), 2^e]:
    // then no consumer's exponent changes and the program (and its CUDA
    // graph) stays valid.  With an exponent to keep, one pass converts and
    // finds the largest component; a second pass runs only if it changed.
    float* dst = static_cast<float*>(n.host);
    std::vector<double> part(kMaxHostThreads, 0.0);
    auto pass = [&](int e, bool convert) {
      const double sc = std::ldexp(1.0, -e);
      std::fill(part.begin(), part.end(), 0.0);
      parallel_chunks(nv, [&](int64_t a, int64_t b, int t) {
        // plain compares, which vectorise: a NaN component never wins (it is
        // stored as NaN), an infinite one does (then the exponent is 0)
        double m = 0.0;
        if (convert) {
          for (int64_t i = a; i < b; ++i) {
            const double x = data[i], ax = std::fabs(x);
            m = ax > m ? ax : m;
            dst[i] = (float)(x * sc);
          }
        } else {
          for (int64_t i = a; i < b; ++i) {
            const double ax = std::fabs(data[i]);
            m = ax > m ? ax : m;
          }
        }
        part[t] = m;
      });
      double mx = 0.0;
      for (double m : part) mx = m > mx ? m : mx;
      return mx;
    };
    const double mx = n.has_data ? pass(n.scale_exp, true) : pass(0, false);
    int e = 0;
    if (mx > 0.0 && std::isfinite(mx)) std::frexp(mx, &e);
    const bool keep = n.has_data && (mx == 0.0 || (std::isfinite(mx) &&
                                                   mx <= std::ldexp(1.0, n.scale_exp) &&
                                                   mx > std::ldexp(1.0, n.scale_exp - 32)));
    if (!keep) {
      rescaled = !n.has_data || e != n.scale_exp;
      n.scale_exp = e;
      pass(e, true);
    }
    // consumers registered before the data changed keep their exponents in sync
    if (rescaled)
      for (size_t u = (size_t)id + 1; u < g.nodes.size(); ++u) {
        Node& c = g.nodes[u];
        if (!c.is_leaf()) c.scale_exp = g.nodes[c.left].scale_exp + g.nodes[c.right].scale_exp;
      }
  }
  n.has_data = true;
  // a staged device copy takes the new values; a new exponent also changes
  // the correlators' scales, which the program holds
  if (rescaled) lqc::exec_invalidate_plan(g);
  return lqc::exec_refresh_staged_leaf(g, id);
  LQC_GUARD_END(h)
}

int lqc_dag_stage_leaves(lqc_dag* h, void* stream) {
  if (!h) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  return lqc::exec_stage_leaves(h->d, stream);
  LQC_GUARD_END(h)
}

int lqc_dag_unstage_leaves(lqc_dag* h) {
  if (!h) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  return lqc::exec_unstage_leaves(h->d);
  LQC_GUARD_END(h)
}

int lqc_dag_execute(lqc_dag* h, void* stream) {
  if (!h) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  if (!h->d.scheduled) return fail(h, LQC_ERR_STATE, "execute before schedule");
  return lqc::exec_run(h->d, stream);
  LQC_GUARD_END(h)
}

int lqc_dag_prepare(lqc_dag* h, void* stream) {
  if (!h) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  if (!h->d.scheduled) return fail(h, LQC_ERR_STATE, "prepare before schedule");
  return lqc::exec_prepare(h->d, stream);
  LQC_GUARD_END(h)
}

int lqc_dag_autotune(lqc_dag* h, void* stream, int reps, lqc_tune_entry* entries, int64_t cap,
                     int64_t* n) {
  if (!h || !n) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  if (!h->d.scheduled) return fail(h, LQC_ERR_STATE, "autotune before schedule");
  if (h->d.prec == LQC_PREC_FP64)
    return fail(h, LQC_ERR_ARG, "autotune applies to the mixed precisions");
  if (reps < 1 || reps > 1000) return fail(h, LQC_ERR_ARG, "reps out of range");
  return lqc::exec_autotune(h->d, stream, reps, entries, cap, n);
  LQC_GUARD_END(h)
}

int lqc_dag_wait(lqc_dag* h, int64_t timeout_ms) {
  if (!h) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  return lqc::exec_wait(h->d, timeout_ms <= 0 ? 60000 : timeout_ms);
  LQC_GUARD_END(h)
}

int lqc_dag_read_correlator(lqc_dag* h, int64_t root, double* out) {
  if (!h || !out) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  return lqc::exec_read(h->d, root, out);
  LQC_GUARD_END(h)
}

int lqc_dag_read_all_correlators(lqc_dag* h, double* out, int64_t cap) {
  if (!h || !out) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  return lqc::exec_read_all(h->d, out, cap);
  LQC_GUARD_END(h)
}

int lqc_dag_get_stats(lqc_dag* h, lqc_stats* s) {
  if (!h || !s) return LQC_ERR_ARG;
  if (!h->d.executed) return fail(h, LQC_ERR_STATE, "not executed");
  *s = h->d.measured;
  return LQC_OK;
}

int lqc_dag_get_exec_info(lqc_dag* h, lqc_exec_info* info) {
  if (!h || !info) return LQC_ERR_ARG;
  if (!h->d.executed) return fail(h, LQC_ERR_STATE, "not executed");
  LQC_GUARD_BEGIN
  int rc = lqc::exec_collect_timing(h->d);
  if (rc != LQC_OK) return rc;
  *info = h->d.info;
  return LQC_OK;
  LQC_GUARD_END(h)
}

int lqc_dag_get_kernel_times(lqc_dag* h, int64_t* node, double* ms, int64_t cap, int64_t* n) {
  if (!h || !n) return LQC_ERR_ARG;
  LQC_GUARD_BEGIN
  return lqc::exec_kernel_times(h->d, node, ms, cap, n);
  LQC_GUARD_END(h)
}

const char* lqc_last_error(const lqc_dag* h) {
  if (!h) return "null DAG handle";
  return h->d.err.c_str();
}

}  // extern "C"
