// Executor: walks the planned op list (LOAD / EVICT / CONTRACT / FREE) on
// the device.
//
// Memory: one device arena sized by an offline placement of every planned
// residency interval (best fit with coalescing, 256-byte aligned); the plan's
// byte accounting is the paper's memory model (Sec. II-C) plus the budget
// rules, the arena is its physical image.  Streams: contractions run on the
// caller's stream; host-to-device loads and device-to-host write-backs run on
// two library-owned side streams.  Every cross-stream dependency (a load
// into memory last read by a kernel, a kernel reading a loaded tensor, a
// write-back of a tensor a kernel produced, a kernel writing memory a
// write-back is still reading) is computed once per plan and becomes an
// event wait, so copies overlap contractions wherever the plan allows.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <thread>

#include "internal.hpp"
#include "kernels.hpp"
#include "kernels_mixed.hpp"
#include "placer.hpp"

namespace lqc {

namespace {

enum Stream { S_COMPUTE = 0, S_H2D = 1, S_D2H = 2 };
enum IKind {
  I_LOAD = 0,
  I_WRITEBACK = 1,
  I_CONTRACT = 2,
  I_CONTRACT_ALL = 3,
  I_POISON = 4,
  I_WINDOW = 5  // a grouped window: its member contractions run as level launches
};

struct Instr {
  int kind;
  int stream;
  int64_t node;
  int64_t dst;        // arena offset (LOAD, CONTRACT) / -1 = results buffer
  int64_t src[2];     // arena offsets of the operands, -2 = staged leaf
  int64_t bytes;
  int32_t nwait = 0;
  int32_t wait[6];
  int32_t rec = -1;   // event slot recorded after this instruction
  int32_t root_slot = -1;
  int32_t win = -1;    // I_WINDOW: index of its window record
  bool member = false; // issued through its window, not on its own
  bool extra = false;  // LOAD / WRITEBACK made by placement within the budget, not by the plan
};

// A grouped window: up to W consecutive contractions of the plan whose frees
// are deferred to the window's end, run level by level (a level = members
// whose operands are all produced before it).
struct WinRec {
  std::vector<int32_t> members;              // instruction indices, plan order
  std::vector<std::vector<int32_t>> levels;  // members per level
  std::vector<int32_t> waits;                // cross-stream waits of the members
  std::vector<LevelDev> ldev;                // task tables per level
  std::vector<int32_t> lev_slot;             // LQC_OPT_TIMING: first mark slot per level
  int64_t flops = 0;
  bool any_exterior = false;
};

}  // namespace

struct ExecState {
  int64_t n_programs = 0;  // programs built (op list, task tables, graph)
  int device = -1;
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};  // [1] h2d, [2] d2h
  cudaEvent_t start_ev = nullptr, done_ev = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<Instr> prog;
  std::vector<ContractDesc> cdesc;        // per instruction (CONTRACT)
  std::vector<ContractAllDesc> adesc;     // per instruction (CONTRACT_ALL)
  std::vector<MixedDesc> mdesc;           // per instruction (CONTRACT, mixed precisions)
  std::vector<WinRec> wins;               // grouped windows
  char* wscratch = nullptr;               // planes / partials of one window level
  int64_t wscratch_bytes = 0;
  char* taskbuf = nullptr;                // task tables of every window level
  char* mscratch = nullptr;               // operand planes / split partials
  int64_t mscratch_bytes = 0;
  bool prog_valid = false;
  int64_t arena_bytes = 0;
  char* arena = nullptr;
  double* results = nullptr;
  int64_t n_results = 0;                  // rank-0 roots
  std::vector<int64_t> root_ids;          // ascending
  std::vector<int32_t> slot_of;           // node -> results slot (-1)
  std::vector<int64_t> res_off;           // slot -> offset in complex values
  int64_t n_result_vals = 0;              // sum of the roots' batch extents
  double* scratch = nullptr;
  int64_t scratch_bytes = 0;
  char* host_arena = nullptr;             // pinned write-back copies, placed per plan
  int64_t host_arena_bytes = 0;
  std::vector<void*> staged;              // node -> device copy of a leaf
  bool staged_valid = false;
  int64_t flops = 0, copy_h2d = 0, copy_d2h = 0, n_kernels = 0;
  lqc_stats counted{};
  bool ran = false;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  // LQC_OPT_TIMING: two sets (alternating executes) of begin/end event
  // pairs per contraction instruction; durations accumulate in g.info
  std::vector<cudaEvent_t> tev[2];
  std::vector<int32_t> tev_kind;
  std::vector<int64_t> tev_flops;
  std::vector<int64_t> tev_node;          // node of each timed instruction
  std::vector<double> tev_ms;             // summed duration per timed instruction
  // LQC_OPT_TIMING with windows: marks between the launches of every level
  // (two sets like tev); per slot the kind of the launch it opens (-1 after
  // a level's last launch) and, for GEMM launches, the level's flops
  std::vector<cudaEvent_t> kev[2];
  std::vector<int8_t> kev_kind;
  std::vector<int64_t> kev_flops;
  // figures of the executor's own walk of the op list
  int64_t walk_evict = 0, walk_peak = 0, resident_peak = 0;
  // moves made to keep the arena within the budget (not the plan's)
  int64_t extra_evict = 0, extra_h2d = 0, extra_d2h = 0;
  bool timing_pending[2] = {false, false};
  int tset = 0;
};

namespace {

// the library's allocations and copies, each open to a test's injected failure
cudaError_t dev_alloc(void** p, size_t n) {
  return inject_fail(INJ_DEVICE_ALLOC) ? cudaErrorMemoryAllocation : cudaMalloc(p, n);
}
cudaError_t pinned_alloc(void** p, size_t n) {
  return inject_fail(INJ_PINNED_ALLOC) ? cudaErrorMemoryAllocation
                                       : cudaHostAlloc(p, n, cudaHostAllocDefault);
}
cudaError_t copy_async(void* dst, const void* src, size_t n, cudaMemcpyKind kind,
                       cudaStream_t s) {
  return inject_fail(INJ_COPY) ? cudaErrorInvalidValue : cudaMemcpyAsync(dst, src, n, kind, s);
}

int cuda_fail(Dag& g, cudaError_t e, const char* what) {
  g.err = std::string(what) + ": " + cudaGetErrorString(e);
  return LQC_ERR_CUDA;
}

#define CK(call, what)                               \
  do {                                               \
    cudaError_t e__ = (call);                        \
    if (e__ != cudaSuccess) return cuda_fail(g, e__, what); \
  } while (0)

int ensure_state(Dag& g) {
  if (!g.ex) g.ex = new ExecState();
  ExecState& x = *g.ex;
  if (x.device < 0) {
    int dev = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    x.device = dev;
    CK(cudaStreamCreateWithFlags(&x.side[S_H2D], cudaStreamNonBlocking), "create h2d stream");
    CK(cudaStreamCreateWithFlags(&x.side[S_D2H], cudaStreamNonBlocking), "create d2h stream");
    CK(cudaEventCreateWithFlags(&x.start_ev, cudaEventDisableTiming), "event create");
    CK(cudaEventCreateWithFlags(&x.done_ev, cudaEventDisableTiming), "event create");
  }
  return LQC_OK;
}

void free_program(ExecState& x) {
  if (x.graph) { cudaGraphExecDestroy(x.graph); x.graph = nullptr; }
  for (int k = 0; k < 2; ++k) {
    for (cudaEvent_t e : x.tev[k]) cudaEventDestroy(e);
    x.tev[k].clear();
    for (cudaEvent_t e : x.kev[k]) cudaEventDestroy(e);
    x.kev[k].clear();
    x.timing_pending[k] = false;
  }
  x.tev_kind.clear();
  x.tev_node.clear();
  x.tev_ms.clear();
  x.tev_flops.clear();
  x.kev_kind.clear();
  x.kev_flops.clear();
  for (cudaEvent_t e : x.ev) cudaEventDestroy(e);
  x.ev.clear();
  if (x.arena) { cudaFree(x.arena); x.arena = nullptr; }
  if (x.results) { cudaFree(x.results); x.results = nullptr; }
  if (x.scratch) { cudaFree(x.scratch); x.scratch = nullptr; }
  if (x.mscratch) { cudaFree(x.mscratch); x.mscratch = nullptr; }
  x.mscratch_bytes = 0;
  if (x.wscratch) { cudaFree(x.wscratch); x.wscratch = nullptr; }
  x.wscratch_bytes = 0;
  if (x.taskbuf) { cudaFree(x.taskbuf); x.taskbuf = nullptr; }
  x.wins.clear();
  x.mdesc.clear();
  if (x.host_arena) { cudaFreeHost(x.host_arena); x.host_arena = nullptr; }
  x.host_arena_bytes = 0;
  x.prog.clear();
  x.cdesc.clear();
  x.adesc.clear();
  x.prog_valid = false;
  x.arena_bytes = 0;
}

// Translate the op list into stream instructions with event dependencies.
int build_program(Dag& g) {
  ExecState& x = *g.ex;
  free_program(x);
  const int64_t N = (int64_t)g.nodes.size();
  const bool staged = x.staged_valid;
  std::vector<int64_t> off(N, -1);
  std::vector<int32_t> last_compute(N, -1), last_h2d(N, -1), last_d2h(N, -1), writer(N, -1);
  std::vector<int32_t> wb_instr(N, -1);  // write-back that filled the node's host slot
  // host copies of written-back tensors live from their write-back to the
  // tensor's final release; their bytes are placed like the device arena, a
  // write-back into reused bytes waiting for the reloads of the previous owner
  std::vector<int64_t> hoff(N, -1);
  Placer hpl;
  std::vector<uint8_t> waited_for_load(N, 0);
  x.slot_of.assign(N, -1);
  x.root_ids.clear();
  for (int64_t u = 0; u < N; ++u)
    if (!g.nodes[u].is_leaf() && g.nodes[u].parents.empty() && g.nodes[u].rank == 0) {
      x.slot_of[u] = (int32_t)x.root_ids.size();
      x.root_ids.push_back(u);
    }
  x.n_results = (int64_t)x.root_ids.size();
  x.res_off.assign(x.n_results, 0);
  x.n_result_vals = 0;
  for (int64_t k = 0; k < x.n_results; ++k) {
    x.res_off[k] = x.n_result_vals;
    x.n_result_vals += g.nodes[x.root_ids[k]].lt;
  }
  Placer pl;
  int64_t scratch_need = 0, mscratch_need = 0;
  std::vector<Instr>& P = x.prog;
  bool evicts = false;
  for (const Op& op : g.ops) evicts = evicts || op.kind == OP_EVICT;
  // leaf region: when the plan evicts nothing and the budget has room, each
  // leaf gets bytes of its own at the bottom of the arena that no other
  // tensor reuses, so its H2D load waits for no kernel and the copy stream
  // runs ahead of the compute stream (loads keep their first-use order)
  std::vector<int64_t> leaf_slot(N, -1);
  if (!staged && !evicts) {
    int64_t total = 0;
    for (const Op& op : g.ops)
      if (op.kind == OP_LOAD && g.nodes[op.node].is_leaf() && leaf_slot[op.node] < 0) {
        leaf_slot[op.node] = total;
        total += (g.size_bytes(op.node) + 255) & ~int64_t(255);
      }
    if (g.budget == 0 || g.planned.peak_exec + total <= (int64_t)g.budget) pl.top = total;
    else std::fill(leaf_slot.begin(), leaf_slot.end(), -1);
  }
  // grouped windows: mixed precisions, plans without evictions
  const int W = (g.prec != LQC_PREC_FP64 && g.opt_window > 1 && !evicts) ? (int)g.opt_window : 0;
  std::vector<int32_t> win;            // open window: member instructions
  std::vector<int64_t> win_free;       // frees deferred to the window's end
  std::vector<int32_t> node_level(N, -1);
  std::vector<int64_t> lvl_need;       // scratch bytes per level of the open window
  std::vector<int32_t> owner;          // member instruction -> its window instruction
  const int64_t kLevelScratchCap = (int64_t)2 << 30;
  // the executor's own account of the device bytes it holds: `held` with
  // frees as they really happen (window frees at the window's end), `res`
  // with every EVICT / FREE at its op (the plan's model); a staged leaf
  // counts from the LOAD the executor skips to its release
  std::vector<uint8_t> holds(N, 0);
  int64_t held = 0, res = 0;
  x.walk_evict = x.walk_peak = x.resident_peak = 0;
  x.extra_evict = x.extra_h2d = x.extra_d2h = 0;
  std::map<int64_t, int64_t> live_at;        // arena offset -> resident node
  auto take_bytes = [&](int64_t u) {
    if (!holds[u]) { holds[u] = 1; held += g.size_bytes(u); }
  };
  auto drop_bytes = [&](int64_t u) {
    if (holds[u]) { holds[u] = 0; held -= g.size_bytes(u); }
  };
  auto add_wait = [&](Instr& in, int32_t on) {
    if (on < 0 || P[on].stream == in.stream) return;
    for (int k = 0; k < in.nwait; ++k)
      if (in.wait[k] == on) return;
    in.wait[in.nwait++] = on;
  };
  auto release = [&](int64_t u) {
    drop_bytes(u);
    if (off[u] < 0) return;
    if (leaf_slot[u] < 0) live_at.erase(off[u]);
    int32_t dep[3] = {last_compute[u], last_h2d[u], last_d2h[u]};
    if (g.opt_poison) {
      Instr in{};
      in.kind = I_POISON;
      in.stream = S_COMPUTE;
      in.node = u;
      in.dst = off[u];
      in.bytes = g.size_bytes(u);
      in.src[0] = in.src[1] = -1;
      add_wait(in, last_d2h[u]);
      add_wait(in, last_h2d[u]);
      P.push_back(in);
      x.cdesc.emplace_back();
      x.adesc.emplace_back();
      x.mdesc.emplace_back();
      dep[S_COMPUTE] = (int32_t)P.size() - 1;
    }
    if (leaf_slot[u] < 0) pl.release(off[u], g.size_bytes(u), dep);
    off[u] = -1;
  };
  auto member_need = [&](int32_t j) -> int64_t {
    if (P[j].kind == I_CONTRACT) return (x.mdesc[j].scratch_bytes + 255) & ~int64_t(255);
    return (contract_all_c64_scratch_bytes(x.adesc[j]) + 255) & ~int64_t(255);
  };
  auto flush = [&]() {
    if (win.empty()) return;
    WinRec rec;
    rec.members = win;
    int max_level = 0;
    for (int32_t m : win) max_level = std::max(max_level, node_level[P[m].node]);
    rec.levels.assign(max_level + 1, {});
    for (int32_t m : win) {
      rec.levels[node_level[P[m].node]].push_back(m);
      for (int k = 0; k < P[m].nwait; ++k)
        if (std::find(rec.waits.begin(), rec.waits.end(), P[m].wait[k]) == rec.waits.end())
          rec.waits.push_back(P[m].wait[k]);
      const ContractDesc& cd = x.cdesc[m];
      const ContractAllDesc& ad = x.adesc[m];
      if (P[m].kind == I_CONTRACT) {
        rec.flops += 8 * cd.lt * cd.M * cd.N * cd.K;
        rec.any_exterior = true;
      } else {
        rec.flops += 8 * ad.lt * ad.S;
      }
    }
    Instr wi{};
    wi.kind = I_WINDOW;
    wi.stream = S_COMPUTE;
    wi.node = P[win[0]].node;
    wi.src[0] = wi.src[1] = -1;
    wi.win = (int32_t)x.wins.size();
    x.wins.push_back(std::move(rec));
    P.push_back(wi);
    x.cdesc.emplace_back();
    x.adesc.emplace_back();
    x.mdesc.emplace_back();
    const int32_t wj = (int32_t)P.size() - 1;
    owner.resize(P.size(), -1);
    for (int32_t m : win) {
      owner[m] = wj;
      node_level[P[m].node] = -1;
    }
    win.clear();
    lvl_need.clear();
    for (int64_t u : win_free) release(u);
    win_free.clear();
  };
  // ---- placement within the budget.  The arena may not grow past the
  // budget: when a tensor's bytes fit nowhere below it (the freed ranges are
  // fragmented), live tensors the current contraction does not read move to
  // the host (written back when they have no host copy yet) and are loaded
  // again before their next use.  These moves are not the plan's: they are
  // reported apart (extra_*), so the counted figures stay the plan's.
  const int64_t limit = g.budget > 0 ? (int64_t)std::min<uint64_t>(g.budget, INT64_MAX) : 0;
  std::vector<uint8_t> out_of_place(N, 0);  // moved out by placement: load before its next use
  auto fits = [&](int64_t bytes) {
    const int64_t b = Placer::rounded(bytes);
    if (pl.by_size.lower_bound({b, INT64_MIN}) != pl.by_size.end()) return true;
    int64_t start = pl.top;
    if (!pl.free_.empty()) {
      auto last = std::prev(pl.free_.end());
      if (last->first + last->second.size == pl.top) start = last->first;
    }
    return start + b <= limit;
  };
  // the resident tensor (not p0 / p1, not in the leaf region) whose release
  // opens the largest free range below the limit
  auto pick_victim = [&](int64_t p0, int64_t p1) -> int64_t {
    int64_t best = -1, best_hole = -1;
    for (const auto& kv : live_at) {
      const int64_t v = kv.second;
      if (v == p0 || v == p1) continue;
      const int64_t o = kv.first, e = o + Placer::rounded(g.size_bytes(v));
      int64_t lo = o, hi = e;
      auto nx = pl.free_.find(e);
      if (nx != pl.free_.end()) hi = e + nx->second.size;
      auto pv = pl.free_.lower_bound(o);
      if (pv != pl.free_.begin()) {
        --pv;
        if (pv->first + pv->second.size == o) lo = pv->first;
      }
      if (hi == pl.top) hi = limit;
      if (hi - lo > best_hole) {
        best_hole = hi - lo;
        best = v;
      }
    }
    return best;
  };
  auto emit_writeback = [&](int64_t u, bool extra) {
    Instr in{};
    in.kind = I_WRITEBACK;
    in.stream = S_D2H;
    in.node = u;
    in.bytes = g.size_bytes(u);
    in.src[0] = off[u];
    in.src[1] = -1;
    in.extra = extra;
    int32_t hdep[3];
    in.dst = hpl.alloc(in.bytes, hdep);  // host offset
    hoff[u] = in.dst;
    add_wait(in, writer[u]);
    add_wait(in, hdep[S_H2D]);  // the previous owner's reloads have read these bytes
    P.push_back(in);
    x.cdesc.emplace_back();
    x.adesc.emplace_back();
    x.mdesc.emplace_back();
    last_d2h[u] = (int32_t)P.size() - 1;
    wb_instr[u] = last_d2h[u];
    if (extra) x.extra_d2h += in.bytes;
  };
  auto place = [&](int64_t u, int64_t bytes, int64_t p0, int64_t p1, int32_t dep[3]) {
    if (limit > 0 && !fits(bytes)) {
      flush();  // a window's members are issued before anything of theirs moves
      while (!fits(bytes)) {
        const int64_t v = pick_victim(p0, p1);
        if (v < 0) break;  // only this contraction's tensors left: the arena grows
        if (!g.nodes[v].is_leaf() && hoff[v] < 0) emit_writeback(v, true);
        release(v);
        out_of_place[v] = 1;
        ++x.extra_evict;
      }
    }
    const int64_t o = pl.alloc(bytes, dep);
    live_at[o] = u;
    return o;
  };
  // H2D load of u (a leaf on first use, or a reload of a written-back tensor)
  auto emit_load = [&](int64_t u, bool extra, int64_t p0, int64_t p1) {
    const Node& nu = g.nodes[u];
    Instr in{};
    in.kind = I_LOAD;
    in.stream = S_H2D;
    in.node = u;
    in.bytes = g.size_bytes(u);
    in.src[0] = in.src[1] = -1;
    in.extra = extra;
    int32_t dep[3];
    if (leaf_slot[u] >= 0) {
      in.dst = leaf_slot[u];  // own bytes: nothing to wait for
    } else {
      in.dst = place(u, in.bytes, p0, p1, dep);
      add_wait(in, dep[S_COMPUTE]);
      add_wait(in, dep[S_D2H]);
    }
    if (!nu.is_leaf()) {
      add_wait(in, wb_instr[u]);  // reload after the write-back landed
      in.src[0] = hoff[u];        // host offset of the copy
    }
    off[u] = in.dst;
    P.push_back(in);
    x.cdesc.emplace_back();
    x.adesc.emplace_back();
    x.mdesc.emplace_back();
    last_h2d[u] = (int32_t)P.size() - 1;
    last_compute[u] = -1;
    last_d2h[u] = -1;
    writer[u] = -1;
    waited_for_load[u] = 0;
    take_bytes(u);
    if (extra) x.extra_h2d += in.bytes;
  };
  // the contraction each op serves (a LOAD's operands are protected)
  std::vector<int64_t> serves(g.ops.size(), -1);
  for (int64_t k = (int64_t)g.ops.size() - 1, nxt = -1; k >= 0; --k) {
    if (g.ops[k].kind == OP_CONTRACT) nxt = g.ops[k].node;
    serves[k] = nxt;
  }
  int64_t opi = -1;
  for (const Op& op : g.ops) {
    ++opi;
    const int64_t u = op.node;
    const Node& n = g.nodes[u];
    if (op.kind == OP_LOAD) {
      take_bytes(u);
      res += g.size_bytes(u);
      if (staged && n.is_leaf()) continue;  // leaves already on the device
      const int64_t c = serves[opi];
      emit_load(u, false, c >= 0 ? g.nodes[c].left : -1, c >= 0 ? g.nodes[c].right : -1);
    } else if (op.kind == OP_EVICT) {
      ++x.walk_evict;
      res -= g.size_bytes(u);
      if (op.flag) {
        if (wb_instr[u] >= 0 && hoff[u] >= 0 && P[wb_instr[u]].extra) {
          // placement wrote it back already: that copy is the plan's write-back
          P[wb_instr[u]].extra = false;
          x.extra_d2h -= g.size_bytes(u);
        } else {
          emit_writeback(u, false);
        }
      }
      out_of_place[u] = 0;  // off the device in the plan too: the plan reloads it
      release(u);
    } else if (op.kind == OP_FREE && W > 0 && !win.empty()) {
      res -= g.size_bytes(u);
      win_free.push_back(u);  // no evictions in windowed plans: no host copy to drop
    } else if (op.kind == OP_FREE) {
      res -= g.size_bytes(u);
      if (hoff[u] >= 0) {  // final release: the host copy is dead too
        int32_t hdep[3] = {-1, last_h2d[u], wb_instr[u]};
        hpl.release(hoff[u], g.size_bytes(u), hdep);
        hoff[u] = -1;
      }
      release(u);
    } else {  // CONTRACT
      // a window holds at most W contractions, and closes (releasing its
      // deferred frees) before its arena would outgrow the budget
      if (W > 0 && !win.empty() &&
          ((int64_t)win.size() >= W ||
           (g.budget > 0 && n.rank != 0 &&
            pl.top + ((g.size_bytes(u) + 255) & ~int64_t(255)) > (int64_t)g.budget)))
        flush();
      // operands that placement moved out come back first
      for (int k = 0; k < n.n_children(); ++k) {
        const int64_t c = n.child(k);
        if (out_of_place[c]) {
          emit_load(c, true, n.left, n.right);
          out_of_place[c] = 0;
        }
      }
      Instr in{};
      in.stream = S_COMPUTE;
      in.node = u;
      in.bytes = g.size_bytes(u);
      for (int k = 0; k < 2; ++k) {
        int64_t c = n.child(k);
        const Node& cn = g.nodes[c];
        if (staged && cn.is_leaf()) {
          in.src[k] = -2;
        } else {
          in.src[k] = off[c];
          if (last_h2d[c] >= 0 && !waited_for_load[c]) {
            add_wait(in, last_h2d[c]);
            waited_for_load[c] = 1;
          }
        }
      }
      const Node& L = g.nodes[n.left];
      const Node& R = g.nodes[n.right];
      std::string err;
      ContractDesc cd{};
      ContractAllDesc ad{};
      if (n.rank == 0) {
        in.kind = I_CONTRACT_ALL;
        in.dst = -1;
        in.root_slot = x.slot_of[u];
        if (!make_contract_all_desc(L.rank, L.ext, R.rank, R.ext, n.npairs, n.la, n.ra, n.lt,
                                    &ad, &err)) {
          g.err = err;
          return LQC_ERR_ARG;
        }
        scratch_need = std::max(scratch_need, g.prec == LQC_PREC_FP64
                                                  ? contract_all_scratch_bytes(ad)
                                                  : contract_all_c64_scratch_bytes(ad));
      } else {
        in.kind = I_CONTRACT;
        if (!make_contract_desc(L.rank, L.ext, R.rank, R.ext, n.npairs, n.la, n.ra, n.lt, &cd,
                                &err)) {
          g.err = err;
          return LQC_ERR_ARG;
        }
        int32_t dep[3];
        in.dst = place(u, in.bytes, n.left, n.right, dep);
        add_wait(in, dep[S_H2D]);
        add_wait(in, dep[S_D2H]);
        off[u] = in.dst;
      }
      MixedDesc md{};
      if (g.prec != LQC_PREC_FP64 && in.kind == I_CONTRACT) {
        MixedTune tune;
        tune.fused_max_n = g.opt_fused_max_n;
        tune.split_policy = (int)g.opt_split_policy;
        tune.fused_kernel = (int)g.opt_fused_kernel;
        if (!make_mixed_desc(cd, g.prec == LQC_PREC_BF16X3, &md, tune)) {
          g.err = "contraction too large for the mixed-precision kernels";
          return LQC_ERR_ARG;
        }
        mscratch_need = std::max(mscratch_need, md.scratch_bytes);
      }
      if (W > 0) {
        int level = 0;
        for (int k = 0; k < n.n_children(); ++k) {
          const int lc = node_level[n.child(k)];
          if (lc >= 0) level = std::max(level, lc + 1);
        }
        const int64_t need = (in.kind == I_CONTRACT)
                                 ? ((md.scratch_bytes + 255) & ~int64_t(255))
                                 : ((contract_all_c64_scratch_bytes(ad) + 255) & ~int64_t(255));
        if (!win.empty() && level < (int)lvl_need.size() &&
            lvl_need[level] + need > std::max(kLevelScratchCap, need)) {
          flush();
          level = 0;
        }
        if ((int)lvl_need.size() <= level) lvl_need.resize(level + 1, 0);
        lvl_need[level] += need;
        in.member = true;
        node_level[u] = level;
      }
      P.push_back(in);
      x.cdesc.push_back(cd);
      x.adesc.push_back(ad);
      x.mdesc.push_back(md);
      const int32_t me = (int32_t)P.size() - 1;
      // the output's bytes (a root's: its Lt values, held only while it runs)
      x.walk_peak = std::max(x.walk_peak, res + g.size_bytes(u));
      x.resident_peak = std::max(x.resident_peak, held + g.size_bytes(u));
      res += g.size_bytes(u);        // a root's FREE op follows at once
      if (n.rank != 0) take_bytes(u);  // a root's values go to the results buffer
      if (W > 0) {
        win.push_back(me);
        (void)member_need;
      }
      for (int k = 0; k < n.n_children(); ++k) last_compute[n.child(k)] = me;
      if (n.rank != 0) {
        last_compute[u] = me;
        writer[u] = me;
        last_h2d[u] = -1;
        last_d2h[u] = -1;
      }
    }
  }
  flush();
  // waits on a window member wait on its window
  owner.resize(P.size(), -1);
  auto remap = [&](int32_t w) { return (w >= 0 && owner[w] >= 0) ? owner[w] : w; };
  for (Instr& in : P) {
    int nw = 0;
    for (int k = 0; k < in.nwait; ++k) {
      const int32_t w = remap(in.wait[k]);
      if (P[w].stream == in.stream) continue;
      bool dup = false;
      for (int q = 0; q < nw; ++q) dup = dup || in.wait[q] == w;
      if (!dup) in.wait[nw++] = w;
    }
    in.nwait = nw;
  }
  for (WinRec& r : x.wins) {
    std::vector<int32_t> ws;
    for (int32_t w : r.waits) {
      w = remap(w);
      if (P[w].stream != S_COMPUTE && std::find(ws.begin(), ws.end(), w) == ws.end())
        ws.push_back(w);
    }
    r.waits = ws;
  }
  // event slots for every instruction somebody waits on
  std::vector<int32_t> slot(P.size(), -1);
  int32_t n_ev = 0;
  auto need_slot = [&](int32_t j) {
    if (slot[j] < 0) slot[j] = n_ev++;
  };
  for (Instr& in : P)
    if (!in.member)
      for (int k = 0; k < in.nwait; ++k) need_slot(in.wait[k]);
  for (WinRec& r : x.wins)
    for (int32_t w : r.waits) need_slot(w);
  for (size_t j = 0; j < P.size(); ++j) P[j].rec = slot[j];
  for (Instr& in : P)
    if (!in.member)
      for (int k = 0; k < in.nwait; ++k) in.wait[k] = slot[in.wait[k]];
  for (WinRec& r : x.wins)
    for (int32_t& w : r.waits) w = slot[w];
  x.ev.resize(n_ev, nullptr);
  for (int32_t k = 0; k < n_ev; ++k)
    CK(cudaEventCreateWithFlags(&x.ev[k], cudaEventDisableTiming), "event create");
  if (g.opt_timing) {
    for (size_t j = 0; j < P.size(); ++j) {
      if (P[j].member) continue;
      if (P[j].kind != I_CONTRACT && P[j].kind != I_CONTRACT_ALL && P[j].kind != I_WINDOW)
        continue;
      for (int k = 0; k < 2; ++k) {
        cudaEvent_t b, e;
        CK(cudaEventCreate(&b), "timing event");
        CK(cudaEventCreate(&e), "timing event");
        x.tev[k].push_back(b);
        x.tev[k].push_back(e);
      }
      const ContractDesc& cd = x.cdesc[j];
      const ContractAllDesc& ad = x.adesc[j];
      x.tev_node.push_back(P[j].node);
      x.tev_ms.push_back(0.0);
      if (P[j].kind == I_WINDOW) {
        const WinRec& r = x.wins[P[j].win];
        x.tev_kind.push_back(r.any_exterior ? I_CONTRACT : I_CONTRACT_ALL);
        x.tev_flops.push_back(r.flops);
      } else {
        x.tev_kind.push_back(P[j].kind);
        x.tev_flops.push_back(P[j].kind == I_CONTRACT ? 8 * cd.lt * cd.M * cd.N * cd.K
                                                        : 8 * ad.lt * ad.S);
      }
    }
  }
  x.arena_bytes = pl.top;
  if (x.arena_bytes > 0) CK(dev_alloc((void**)&x.arena, (size_t)x.arena_bytes), "arena cudaMalloc");
  if (x.n_results > 0)
    CK(dev_alloc((void**)&x.results, (size_t)(x.n_result_vals * 16)), "results cudaMalloc");
  x.scratch_bytes = scratch_need;
  if (scratch_need > 0) CK(dev_alloc((void**)&x.scratch, (size_t)scratch_need), "scratch cudaMalloc");
  x.mscratch_bytes = mscratch_need;
  if (mscratch_need > 0)
    CK(dev_alloc((void**)&x.mscratch, (size_t)mscratch_need), "plane scratch cudaMalloc");
  // window levels: scratch sized by the largest level, task tables built with
  // the final device addresses
  for (const WinRec& r : x.wins)
    for (const auto& lv : r.levels) {
      int64_t sum = 0;
      for (int32_t m : lv) sum += member_need(m);
      x.wscratch_bytes = std::max(x.wscratch_bytes, sum);
    }
  if (x.wscratch_bytes > 0)
    CK(dev_alloc((void**)&x.wscratch, (size_t)x.wscratch_bytes), "window scratch cudaMalloc");
  if (!x.wins.empty()) {
    std::vector<char> tbuf;
    auto operand = [&](const Instr& in, int k) -> const float* {
      const int64_t c = g.nodes[in.node].child(k);
      return in.src[k] == -2 ? static_cast<const float*>(x.staged[c])
                             : reinterpret_cast<const float*>(x.arena + in.src[k]);
    };
    for (WinRec& r : x.wins) {
      r.ldev.resize(r.levels.size());
      for (size_t l = 0; l < r.levels.size(); ++l) {
        std::vector<GroupExt> ext;
        std::vector<GroupRoot> roots;
        int64_t so = 0;
        for (int32_t m : r.levels[l]) {
          const Instr& in = P[m];
          const Node& nn = g.nodes[in.node];
          if (in.kind == I_CONTRACT) {
            ext.push_back(GroupExt{&x.mdesc[m], operand(in, 0), operand(in, 1),
                                   reinterpret_cast<float*>(x.arena + in.dst), x.wscratch + so});
          } else {
            roots.push_back(GroupRoot{
                &x.adesc[m], operand(in, 0), operand(in, 1), x.results + 2 * x.res_off[in.root_slot],
                reinterpret_cast<double*>(x.wscratch + so),
                std::ldexp(1.0, g.nodes[nn.left].scale_exp + g.nodes[nn.right].scale_exp)});
          }
          so += member_need(m);
        }
        if (!append_level_tasks(ext, roots, g.prec == LQC_PREC_BF16X3, &tbuf, &r.ldev[l])) {
          g.err = "TMA tensor map encoding failed";
          return LQC_ERR_CUDA;
        }
      }
    }
    CK(dev_alloc((void**)&x.taskbuf, tbuf.size() + 64), "task table cudaMalloc");
    CK(cudaMemcpy(x.taskbuf, tbuf.data(), tbuf.size(), cudaMemcpyHostToDevice), "task tables");
    for (WinRec& r : x.wins)
      for (LevelDev& d : r.ldev) rebase_level(&d, x.taskbuf);
    if (g.opt_timing) {
      for (WinRec& r : x.wins) {
        r.lev_slot.resize(r.levels.size());
        for (size_t l = 0; l < r.levels.size(); ++l) {
          int kinds[LQC_NUM_KINDS];
          const int nk = level_launch_kinds(r.ldev[l], kinds);
          // each GEMM launch of the level carries the flops of its own tasks:
          // plane form, CTA-pair fused form (launched first), one-CTA fused form
          int64_t fl_planes = 0, fl_pair = 0, fl_single = 0;
          for (int32_t m : r.levels[l])
            if (P[m].kind == I_CONTRACT) {
              const ContractDesc& cd = x.cdesc[m];
              const MixedDesc& md = x.mdesc[m];
              const int64_t f = 8 * cd.lt * cd.M * cd.N * cd.K;
              (md.fused ? (md.pair ? fl_pair : fl_single) : fl_planes) += f;
            }
          r.lev_slot[l] = (int32_t)x.kev_kind.size();
          bool pair_next = r.ldev[l].ngemm_pair > 0;
          for (int k = 0; k < nk; ++k) {
            x.kev_kind.push_back((int8_t)kinds[k]);
            int64_t f = 0;
            if (kinds[k] == LQC_KIND_GEMM_PLANES) {
              f = fl_planes;
            } else if (kinds[k] == LQC_KIND_GEMM_FUSED) {
              f = pair_next ? fl_pair : fl_single;
              pair_next = false;
            }
            x.kev_flops.push_back(f);
          }
          x.kev_kind.push_back(-1);
          x.kev_flops.push_back(0);
        }
      }
      for (int k = 0; k < 2; ++k) {
        x.kev[k].resize(x.kev_kind.size(), nullptr);
        for (cudaEvent_t& e : x.kev[k]) CK(cudaEventCreate(&e), "timing event");
      }
    }
  }
  x.host_arena_bytes = hpl.top;
  if (hpl.top > 0)
    CK(pinned_alloc((void**)&x.host_arena, (size_t)hpl.top),
       "pinned write-back arena");
  x.prog_valid = true;
  ++x.n_programs;
  x.tset = 0;
  g.info.n_contract = g.info.n_contract_all = 0;
  g.info.ms_contract = g.info.ms_contract_all = 0.0;
  g.info.flops_contract = g.info.flops_contract_all = 0;
  for (int k = 0; k < LQC_NUM_KINDS; ++k) {
    g.info.n_kind[k] = 0;
    g.info.ms_kind[k] = 0.0;
  }
  g.info.flops_gemm = 0;
  return LQC_OK;
}

// Issue the program on the streams (also used under graph capture).
int issue(Dag& g, cudaStream_t cs, bool capturing) {
  // timing events inside a stream capture must become event-record nodes
  const unsigned tflag = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  ExecState& x = *g.ex;
  cudaStream_t st[3] = {cs, x.side[S_H2D], x.side[S_D2H]};
  // side streams start after everything already queued on the compute stream
  CK(cudaEventRecord(x.start_ev, cs), "record start");
  CK(cudaStreamWaitEvent(st[S_H2D], x.start_ev, 0), "wait start");
  CK(cudaStreamWaitEvent(st[S_D2H], x.start_ev, 0), "wait start");
  x.flops = 0;
  x.copy_h2d = x.copy_d2h = 0;
  x.n_kernels = 0;
  lqc_stats c{};
  size_t tk = 0;  // timing pair cursor
  for (size_t j = 0; j < x.prog.size(); ++j) {
    const Instr& in = x.prog[j];
    if (in.member) continue;  // runs inside its window
    cudaStream_t s = st[in.stream];
    for (int k = 0; k < in.nwait; ++k) CK(cudaStreamWaitEvent(s, x.ev[in.wait[k]], 0), "wait");
    if (in.kind == I_WINDOW) {
      const WinRec& r = x.wins[in.win];
      for (int32_t w : r.waits) CK(cudaStreamWaitEvent(s, x.ev[w], 0), "wait");
      const bool timed = g.opt_timing && tk < x.tev_kind.size();
      if (timed) CK(cudaEventRecordWithFlags(x.tev[x.tset][2 * tk], s, tflag), "timing record");
      for (size_t l = 0; l < r.ldev.size(); ++l) {
        cudaEvent_t* marks = timed && !r.lev_slot.empty() ? &x.kev[x.tset][r.lev_slot[l]]
                                                          : nullptr;
        const int nk = launch_level(r.ldev[l], s, marks, tflag);
        if (nk < 0) return cuda_fail(g, cudaGetLastError(), "window level launch");
        x.n_kernels += nk;
      }
      if (timed) {
        CK(cudaEventRecordWithFlags(x.tev[x.tset][2 * tk + 1], s, tflag), "timing record");
        ++tk;
      }
      x.flops += r.flops;
      if (in.rec >= 0) CK(cudaEventRecord(x.ev[in.rec], s), "record");
      continue;
    }
    const Node& n = g.nodes[in.node];
    switch (in.kind) {
      case I_LOAD: {
        const void* src = n.is_leaf() ? n.host : (const void*)(x.host_arena + in.src[0]);
        CK(copy_async(x.arena + in.dst, src, (size_t)in.bytes, cudaMemcpyHostToDevice, s),
           "H2D load");
        x.copy_h2d += in.bytes;
        if (!in.extra) {  // the plan's loads (placement's are reported apart)
          c.n_h2d++;
          c.h2d_bytes += in.bytes;
        }
        break;
      }
      case I_WRITEBACK: {
        CK(copy_async(x.host_arena + in.dst, x.arena + in.src[0], (size_t)in.bytes,
                           cudaMemcpyDeviceToHost, s),
           "D2H write-back");
        x.copy_d2h += in.bytes;
        if (!in.extra) {
          c.n_d2h++;
          c.d2h_bytes += in.bytes;
        }
        break;
      }
      case I_POISON: {
        if (launch_fill_nan(x.arena + in.dst, in.bytes, s) < 0)
          return cuda_fail(g, cudaGetLastError(), "poison launch");
        x.n_kernels += 1;
        break;
      }
      case I_CONTRACT:
      case I_CONTRACT_ALL: {
        const void* op[2];
        for (int k = 0; k < 2; ++k) {
          int64_t ch = n.child(k);
          op[k] = in.src[k] == -2 ? x.staged[ch] : (const void*)(x.arena + in.src[k]);
        }
        int nk;
        const bool timed = g.opt_timing && tk < x.tev_kind.size();
        if (timed) CK(cudaEventRecordWithFlags(x.tev[x.tset][2 * tk], s, tflag), "timing record");
        const bool mixed = g.prec != LQC_PREC_FP64;
        if (in.kind == I_CONTRACT) {
          const ContractDesc& d = x.cdesc[j];
          if (mixed)
            nk = launch_contract_mixed(x.mdesc[j], (const float*)op[0], (const float*)op[1],
                                       (float*)(x.arena + in.dst), x.mscratch, s);
          else
            nk = launch_contract_fp64(d, (const double*)op[0], (const double*)op[1],
                                      (double*)(x.arena + in.dst), s);
          x.flops += 8 * d.lt * d.M * d.N * d.K;
        } else {
          const ContractAllDesc& d = x.adesc[j];
          if (mixed)
            nk = launch_contract_all_c64(d, (const float*)op[0], (const float*)op[1],
                                         x.results + 2 * x.res_off[in.root_slot], x.scratch,
                                         std::ldexp(1.0, g.nodes[n.left].scale_exp +
                                                             g.nodes[n.right].scale_exp),
                                         s);
          else
            nk = launch_contract_all_fp64(d, (const double*)op[0], (const double*)op[1],
                                          x.results + 2 * x.res_off[in.root_slot], x.scratch, s);
          x.flops += 8 * d.lt * d.S;
        }
        if (nk == -2) {
          g.err = "TMA tensor map encoding failed";
          return LQC_ERR_CUDA;
        }
        if (nk < 0) return cuda_fail(g, cudaGetLastError(), "contraction launch");
        if (timed) {
          CK(cudaEventRecordWithFlags(x.tev[x.tset][2 * tk + 1], s, tflag), "timing record");
          ++tk;
        }
        x.n_kernels += nk;
        break;
      }
    }
    if (in.rec >= 0) CK(cudaEventRecord(x.ev[in.rec], s), "record");
  }
  // join the side streams back into the compute stream
  for (int k = 1; k < 3; ++k) {
    CK(cudaEventRecord(x.start_ev, st[k]), "record join");
    CK(cudaStreamWaitEvent(cs, x.start_ev, 0), "wait join");
  }
  // counted figures: copies from this walk; evictions and the op-level peak
  // from the program build's walk of the op list; peak_paper is the plan's
  // model figure of the order (the executor runs the order as planned)
  c.n_evict = x.walk_evict;
  c.peak_exec = x.walk_peak;
  c.peak_paper = g.planned.peak_paper;
  // with staged leaves the leaf loads are served on the device: c counts
  // only what really crossed the host link
  x.counted = c;
  return LQC_OK;
}

}  // namespace

int host_store_alloc(Dag& g, int64_t leaf, std::string* err) {
  Node& n = g.nodes[leaf];
  if (n.host) return LQC_OK;
  const size_t bytes = (size_t)(n.lt * n.elems * g.elem_bytes);
  void* p = nullptr;
  if (pinned_alloc(&p, bytes) == cudaSuccess) {
    n.host = p;
    n.host_pinned = true;
    return LQC_OK;
  }
  cudaGetLastError();  // no device (or pinned memory exhausted): pageable store
  p = std::malloc(bytes);
  if (!p) {
    *err = "host store allocation failed";
    return LQC_ERR_HOST_MEM;
  }
  n.host = p;
  n.host_pinned = false;
  return LQC_OK;
}

void host_store_free(Node& n) {
  if (!n.host) return;
  if (n.host_pinned) cudaFreeHost(n.host);
  else std::free(n.host);
  n.host = nullptr;
}

void exec_invalidate_plan(Dag& g) {
  if (!g.ex) return;
  exec_wait(g, 60000);
  free_program(*g.ex);
}

// Times whole executions of the scheduled DAG (as it stands: staged or host
// leaves, graph or not) for every candidate of window x fused-form limit x
// split policy, `reps` executes each after one that builds the program; the
// fastest is kept.  Windows only where the plan evicts nothing.
int exec_autotune(Dag& g, void* stream, int reps, lqc_tune_entry* entries, int64_t cap,
                  int64_t* n) {
  std::vector<lqc_tune_entry> cand;
  const bool windows_ok = g.planned.n_evict == 0;
  // the GEMM tile (one CTA or a CTA pair) is a candidate with every width
  // fused; the A-in-TMEM kernel, when chosen, is kept as it is
  const bool tmem_a = g.opt_fused_kernel == 1;
  for (int64_t w : {int64_t(0), int64_t(64), int64_t(512), int64_t(4096)}) {
    if (w && !windows_ok) continue;
    for (int64_t f : {int64_t(0), int64_t(64), int64_t(1) << 30}) {
      if (g.prec == LQC_PREC_BF16X3 && f) continue;  // no fused form for BF16
      for (int64_t sp : {int64_t(0), int64_t(1)}) {
        if (tmem_a || f != (int64_t(1) << 30)) {
          cand.push_back(lqc_tune_entry{w, f, sp, g.opt_fused_kernel, 0.0});
        } else {
          for (int64_t k : {int64_t(0), int64_t(2)}) cand.push_back(lqc_tune_entry{w, f, sp, k, 0.0});
        }
      }
    }
  }
  if (cap < (int64_t)cand.size() && entries) {
    g.err = "tune entry capacity too small";
    return LQC_ERR_ARG;
  }
  const int64_t save[4] = {g.opt_window, g.opt_fused_max_n, g.opt_split_policy,
                           g.opt_fused_kernel};
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0), "tune event");
  if (cudaError_t e = cudaEventCreate(&e1); e != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(g, e, "tune event");
  }
  int rc = LQC_OK;
  size_t best = 0;
  for (size_t c = 0; c < cand.size() && rc == LQC_OK; ++c) {
    g.opt_window = cand[c].window;
    g.opt_fused_max_n = cand[c].fused_max_n;
    g.opt_split_policy = cand[c].split_policy;
    g.opt_fused_kernel = cand[c].fused_kernel;
    exec_invalidate_plan(g);
    rc = exec_run(g, stream);  // builds the program (and the graph)
    if (rc != LQC_OK) break;
    cudaEventRecord(e0, cs);
    for (int r = 0; r < reps && rc == LQC_OK; ++r) rc = exec_run(g, stream);
    cudaEventRecord(e1, cs);
    if (rc != LQC_OK) break;
    rc = exec_wait(g, 600000);
    if (rc != LQC_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) rc = cuda_fail(g, e, "tune timing");
    cand[c].ms = ms / reps;
    if (cand[c].ms < cand[best].ms) best = c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LQC_OK) {
    g.opt_window = save[0];
    g.opt_fused_max_n = save[1];
    g.opt_split_policy = save[2];
    g.opt_fused_kernel = save[3];
    exec_invalidate_plan(g);
    return rc;
  }
  g.opt_window = cand[best].window;
  g.opt_fused_max_n = cand[best].fused_max_n;
  g.opt_split_policy = cand[best].split_policy;
  g.opt_fused_kernel = cand[best].fused_kernel;
  exec_invalidate_plan(g);
  *n = (int64_t)cand.size();
  if (entries) std::copy(cand.begin(), cand.end(), entries);
  return LQC_OK;
}

namespace {
int collect_set(Dag& g, int set) {
  ExecState& x = *g.ex;
  const std::vector<cudaEvent_t>& ev = x.tev[set];
  if (ev.empty()) return LQC_OK;
  auto t0 = std::chrono::steady_clock::now();
  while (true) {  // bounded wait for the set's last event
    cudaError_t e = cudaEventQuery(ev.back());
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_fail(g, e, "timing wait");
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60)) {
      g.err = "timing events not complete after the wait limit";
      return LQC_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  for (size_t k = 0; k < x.tev_kind.size(); ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]), "timing elapsed");
    x.tev_ms[k] += ms;
    if (x.tev_kind[k] == I_CONTRACT) {
      g.info.n_contract++;
      g.info.ms_contract += ms;
      g.info.flops_contract += x.tev_flops[k];
    } else {
      g.info.n_contract_all++;
      g.info.ms_contract_all += ms;
      g.info.flops_contract_all += x.tev_flops[k];
    }
  }
  const std::vector<cudaEvent_t>& kv = x.kev[set];
  for (size_t k = 0; k + 1 < kv.size(); ++k) {
    const int kind = x.kev_kind[k];
    if (kind < 0) continue;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, kv[k], kv[k + 1]), "timing elapsed");
    g.info.n_kind[kind]++;
    g.info.ms_kind[kind] += ms;
    g.info.flops_gemm += x.kev_flops[k];
  }
  x.timing_pending[set] = false;
  return LQC_OK;
}
}  // namespace

namespace {
// capture the whole issue into a graph for stream `cs` (once per stream)
int ensure_graph(Dag& g, cudaStream_t cs) {
  ExecState& x = *g.ex;
  if (x.graph && x.graph_stream == cs) return LQC_OK;
  if (x.graph) { cudaGraphExecDestroy(x.graph); x.graph = nullptr; }
  cudaStream_t cap = cs;
  bool own = false;
  if (cap == nullptr) {  // the legacy stream cannot be captured
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    own = true;
  }
  CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  int rc = issue(g, cap, true);
  if (rc != LQC_OK) {  // an issue that stopped early: join the forked side streams
    for (int k = 1; k < 3; ++k) {  // so that the capture ends on every stream
      cudaEventRecord(x.start_ev, x.side[k]);
      cudaStreamWaitEvent(cap, x.start_ev, 0);
    }
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cap, &graph);
  if (rc != LQC_OK) {
    if (graph) cudaGraphDestroy(graph);
    if (own) cudaStreamDestroy(cap);
    return rc;
  }
  if (e != cudaSuccess) {
    if (own) cudaStreamDestroy(cap);
    return cuda_fail(g, e, "end capture");
  }
  e = cudaGraphInstantiate(&x.graph, graph, 0);
  cudaGraphDestroy(graph);
  if (own) cudaStreamDestroy(cap);
  if (e != cudaSuccess) return cuda_fail(g, e, "graph instantiate");
  x.graph_stream = cs;
  return LQC_OK;
}
}  // namespace

int exec_prepare(Dag& g, void* stream) {
  clear_pending_error();  // an earlier, unrelated error must not fail this DAG's launches
  int rc = ensure_state(g);
  if (rc != LQC_OK) return rc;
  ExecState& x = *g.ex;
  for (const Op& op : g.ops)
    if (op.kind == OP_LOAD && g.nodes[op.node].is_leaf() && !g.nodes[op.node].host &&
        !x.staged_valid) {
      g.err = "leaf " + std::to_string(op.node) + " has no data";
      return LQC_ERR_STATE;
    }
  if (!x.prog_valid) {
    rc = build_program(g);
    if (rc != LQC_OK) {
      free_program(x);
      return rc;
    }
  }
  if (g.opt_graph) return ensure_graph(g, static_cast<cudaStream_t>(stream));
  return LQC_OK;
}

int exec_run(Dag& g, void* stream) {
  int rc = exec_prepare(g, stream);
  if (rc != LQC_OK) return rc;
  ExecState& x = *g.ex;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (g.opt_graph) x.tset = 0;  // a captured graph always records timing set 0
  if (g.opt_timing && x.timing_pending[x.tset]) {
    // the execute that last recorded this set: two steps back (normally long
    // done), or the previous graph replay
    rc = collect_set(g, x.tset);
    if (rc != LQC_OK) return rc;
  }
  if (g.opt_graph) {
    CK(cudaGraphLaunch(x.graph, cs), "graph launch");
  } else {
    rc = issue(g, cs, false);
    if (rc != LQC_OK) return rc;
  }
  CK(cudaEventRecord(x.done_ev, cs), "record done");
  x.ran = true;
  if (g.opt_timing && !x.tev_kind.empty()) {
    x.timing_pending[x.tset] = true;
    if (!g.opt_graph) x.tset ^= 1;
  }
  g.measured = x.counted;
  g.info.n_kernels = x.n_kernels;
  g.info.flops = x.flops;
  g.info.arena_bytes = x.arena_bytes;
  g.info.host_arena_bytes = x.host_arena_bytes;
  g.info.copied_h2d = x.copy_h2d;
  g.info.copied_d2h = x.copy_d2h;
  g.info.n_ops = (int64_t)g.ops.size();
  g.info.resident_peak_bytes = x.resident_peak;
  g.info.extra_evictions = x.extra_evict;
  g.info.extra_h2d_bytes = x.extra_h2d;
  g.info.extra_d2h_bytes = x.extra_d2h;
  g.info.n_programs = x.n_programs;
  g.executed = true;
  return LQC_OK;
}

int exec_wait(Dag& g, int64_t timeout_ms) {
  if (!g.ex || !g.ex->ran) return LQC_OK;
  ExecState& x = *g.ex;
  auto t0 = std::chrono::steady_clock::now();
  int sleep_us = 20;
  while (true) {
    cudaError_t e = cudaEventQuery(x.done_ev);
    if (e == cudaSuccess) {
      if (g.prec != LQC_PREC_FP64) {
        int st = mixed_error_status(true);
        if (st != 0) {
          g.err = st < 0 ? "cannot read the device error word"
                         : "a tensor-core kernel gave up on a bounded wait";
          return st < 0 ? LQC_ERR_CUDA : LQC_ERR_TIMEOUT;
        }
      }
      return LQC_OK;
    }
    if (e != cudaErrorNotReady) return cuda_fail(g, e, "execution failed");
    auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                  std::chrono::steady_clock::now() - t0).count();
    if (ms >= timeout_ms) {
      g.err = "execution still running after the wait limit";
      return LQC_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(sleep_us));
    sleep_us = std::min(sleep_us * 2, 2000);
  }
}

int exec_collect_timing(Dag& g) {
  if (!g.ex) return LQC_OK;
  ExecState& x = *g.ex;
  // older set first (the one the next execute would reuse), then the newer
  for (int k = 0; k < 2; ++k) {
    int set = x.tset ^ (k == 0 ? 0 : 1);
    if (!x.timing_pending[set]) continue;
    int rc = collect_set(g, set);
    if (rc != LQC_OK) return rc;
  }
  return LQC_OK;
}

int exec_kernel_times(Dag& g, int64_t* node, double* ms, int64_t cap, int64_t* n) {
  int rc = exec_collect_timing(g);
  if (rc != LQC_OK) return rc;
  if (!g.ex) {
    *n = 0;
    return LQC_OK;
  }
  ExecState& x = *g.ex;
  *n = (int64_t)x.tev_node.size();
  if (cap < *n || (*n > 0 && (!node || !ms))) {
    g.err = "output capacity too small";
    return LQC_ERR_ARG;
  }
  for (int64_t k = 0; k < *n; ++k) {
    node[k] = x.tev_node[k];
    ms[k] = x.tev_ms[k];
  }
  return LQC_OK;
}

int exec_read(Dag& g, int64_t root, double* out) {
  if (root < 0 || root >= (int64_t)g.nodes.size()) {
    g.err = "root id out of range";
    return LQC_ERR_ARG;
  }
  if (!g.executed || !g.ex || !g.ex->results) {
    g.err = "not executed";
    return LQC_ERR_STATE;
  }
  ExecState& x = *g.ex;
  if (x.slot_of[root] < 0) {
    g.err = "node is not a rank-0 root";
    return LQC_ERR_ARG;
  }
  int rc = exec_wait(g, 60000);
  if (rc != LQC_OK) return rc;
  CK(cudaMemcpy(out, x.results + 2 * x.res_off[x.slot_of[root]], (size_t)(g.nodes[root].lt * 16),
                cudaMemcpyDeviceToHost),
     "read correlator");
  return LQC_OK;
}

int exec_read_all(Dag& g, double* out, int64_t cap) {
  if (!g.executed || !g.ex) {
    g.err = "not executed";
    return LQC_ERR_STATE;
  }
  ExecState& x = *g.ex;
  if (cap < x.n_result_vals * 2) {
    g.err = "output capacity too small";
    return LQC_ERR_ARG;
  }
  int rc = exec_wait(g, 60000);
  if (rc != LQC_OK) return rc;
  if (x.n_results > 0)
    CK(cudaMemcpy(out, x.results, (size_t)(x.n_result_vals * 16), cudaMemcpyDeviceToHost),
       "read correlators");
  return LQC_OK;
}

int exec_stage_leaves(Dag& g, void* stream) {
  int rc = ensure_state(g);
  if (rc != LQC_OK) return rc;
  ExecState& x = *g.ex;
  rc = exec_wait(g, 60000);
  if (rc != LQC_OK) return rc;
  exec_unstage_leaves(g);
  const int64_t N = (int64_t)g.nodes.size();
  x.staged.assign(N, nullptr);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int64_t u = 0; u < N; ++u) {
    Node& n = g.nodes[u];
    if (!n.is_leaf() || n.parents.empty()) continue;
    if (!n.host) {
      g.err = "leaf " + std::to_string(u) + " has no data";
      exec_unstage_leaves(g);
      return LQC_ERR_STATE;
    }
    size_t bytes = (size_t)g.size_bytes(u);
    CK(dev_alloc(&x.staged[u], bytes), "staged leaf cudaMalloc");
    CK(copy_async(x.staged[u], n.host, bytes, cudaMemcpyHostToDevice, s), "stage leaf");
  }
  CK(cudaStreamSynchronize(s), "stage sync");
  x.staged_valid = true;
  free_program(x);
  return LQC_OK;
}

int exec_refresh_staged_leaf(Dag& g, int64_t u) {
  if (!g.ex) return LQC_OK;
  ExecState& x = *g.ex;
  if (!x.staged_valid || u < 0 || u >= (int64_t)x.staged.size() || !x.staged[u]) return LQC_OK;
  CK(cudaMemcpy(x.staged[u], g.nodes[u].host, (size_t)g.size_bytes(u), cudaMemcpyHostToDevice),
     "refresh staged leaf");
  return LQC_OK;
}

int exec_unstage_leaves(Dag& g) {
  if (!g.ex) return LQC_OK;
  ExecState& x = *g.ex;
  exec_wait(g, 60000);
  for (void* p : x.staged)
    if (p) cudaFree(p);
  x.staged.clear();
  if (x.staged_valid) {
    x.staged_valid = false;
    free_program(x);
  }
  return LQC_OK;
}

void exec_destroy(Dag& g) {
  if (!g.ex) return;
  ExecState& x = *g.ex;
  if (x.ran) exec_wait(g, 60000);
  exec_unstage_leaves(g);
  free_program(x);
  for (int k = 1; k < 3; ++k)
    if (x.side[k]) cudaStreamDestroy(x.side[k]);
  if (x.start_ev) cudaEventDestroy(x.start_ev);
  if (x.done_ev) cudaEventDestroy(x.done_ev);
  delete g.ex;
  g.ex = nullptr;
}

}  // namespace lqc
