// Internal data structures of the contraction-DAG executor (host side).
#pragma once

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/lqc.h"

namespace lqc {

enum NodeType { LEAF = 0, INTERIOR = 1, ROOT = 2 };

// One DAG node (Sec. II-B): a leaf tensor, or a binary contraction together
// with its output tensor.
struct Node {
  int rank = 0;
  int64_t ext[LQC_MAX_RANK] = {0};
  int64_t elems = 1;            // per time slice
  int64_t lt = 1;               // batch (time-slice) extent, never contracted
  int64_t left = -1, right = -1;
  int npairs = 0;
  int la[LQC_MAX_RANK] = {0}, ra[LQC_MAX_RANK] = {0};
  std::vector<int64_t> parents; // distinct consumers, ascending id
  // leaves: host copy (pinned when a device is present), element layout of
  // the DAG's storage precision; nullptr until data is given
  void* host = nullptr;
  bool host_pinned = false;
  bool has_data = false;        // leaves: data given at least once
  // mixed precisions: stored values are the tensor times 2^-scale_exp
  // (leaves: FP64 normalisation; contractions: sum of the operands')
  int scale_exp = 0;
  bool is_leaf() const { return left < 0; }
  // distinct children: [left] or [left, right]
  int n_children() const { return is_leaf() ? 0 : (left == right ? 1 : 2); }
  int64_t child(int k) const { return k == 0 ? left : right; }
};

enum OpKind { OP_LOAD = 0, OP_EVICT = 1, OP_CONTRACT = 2, OP_FREE = 3 };

struct Op {
  int32_t kind;
  int32_t flag;   // EVICT: 1 = write back to the host
  int64_t node;
};

struct KeyHash {
  size_t operator()(const std::string& s) const { return std::hash<std::string>()(s); }
};

struct ExecState;  // device-side state (exec.cu)

struct Dag {
  int64_t lt = 1;               // batch extent given to leaves added next
  lqc_precision prec = LQC_PREC_FP64;
  int elem_bytes = 16;
  std::vector<Node> nodes;
  std::unordered_map<std::string, int64_t, KeyHash> dedup;
  bool frozen = false;
  // schedule + plan
  bool scheduled = false;
  std::vector<int64_t> order;
  std::vector<Op> ops;
  lqc_stats planned{};
  uint64_t budget = 0;
  lqc_evict evict = LQC_EVICT_LRU;
  // execution
  ExecState* ex = nullptr;
  int64_t opt_graph = 0, opt_poison = 0, opt_timing = 0, opt_window = 64;
  int64_t opt_fused_max_n = 64, opt_split_policy = 0;  // mixed GEMM choices
  int64_t opt_fused_kernel = 0;
  lqc_stats measured{};
  lqc_exec_info info{};
  bool executed = false;
  std::string err;

  int64_t size_bytes(int64_t u) const { return nodes[u].lt * nodes[u].elems * elem_bytes; }
  NodeType type(int64_t u) const {
    const Node& n = nodes[u];
    if (n.is_leaf()) return LEAF;
    return n.parents.empty() ? ROOT : INTERIOR;
  }
};

// ---- schedulers (sched.cpp) ----
std::vector<int64_t> schedule_naive(const Dag& g);
std::vector<int64_t> schedule_sibling(const Dag& g);
std::vector<int64_t> schedule_tree(const Dag& g);
std::vector<int64_t> schedule_node(const Dag& g);
std::vector<int64_t> schedule_rsgs(const Dag& g);

// ---- planner (plan.cpp): returns false and sets g.err on a budget error ----
bool plan_replay(const Dag& g, const std::vector<int64_t>& order, uint64_t budget,
                 lqc_evict evict, std::vector<Op>* ops, lqc_stats* st, std::string* err);
int64_t model_peak(const Dag& g, const std::vector<int64_t>& order);

// ---- failure injection for tests (api.cpp): the library's host-side CUDA
// allocations and copies ask this before the real call; true = behave as if
// the call had failed (one armed failure is consumed) ----
enum InjectSite { INJ_DEVICE_ALLOC = 0, INJ_PINNED_ALLOC = 1, INJ_COPY = 2, INJ_SITES = 3 };
bool inject_fail(int site);

// ---- executor (exec.cu) ----
int exec_run(Dag& g, void* stream);
int exec_prepare(Dag& g, void* stream);
int exec_autotune(Dag& g, void* stream, int reps, lqc_tune_entry* entries, int64_t cap,
                  int64_t* n);
int exec_wait(Dag& g, int64_t timeout_ms);
int exec_collect_timing(Dag& g);
int exec_kernel_times(Dag& g, int64_t* node, double* ms, int64_t cap, int64_t* n);
int exec_read(Dag& g, int64_t root, double* out);
int exec_read_all(Dag& g, double* out, int64_t cap);
int exec_stage_leaves(Dag& g, void* stream);
// after new data of leaf u with unchanged scale: refresh its staged device
// copy (if the leaves are staged); the program and its graph stay valid
int exec_refresh_staged_leaf(Dag& g, int64_t u);
int exec_unstage_leaves(Dag& g);
void exec_destroy(Dag& g);
void exec_invalidate_plan(Dag& g);   // plan changed: rebuild arena program on next run
int host_store_alloc(Dag& g, int64_t leaf, std::string* err);
void host_store_free(Node& n);

}  // namespace lqc

// The opaque handle of the C ABI.
struct lqc_dag {
  lqc::Dag d;
};
