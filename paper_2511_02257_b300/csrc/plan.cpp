// Budgeted replay of a contraction order (the planner).
//
// Memory model of Sec. II-C: leaves live on the host and occupy device memory
// from their first use; step i loads the leaves c_i needs, performs c_i and
// releases every tensor without remaining consumers (a root's output at
// once).  peak_paper = max_i M_i of that model.
//
// Budget rules (the paper delegates eviction to MemHC's "pre-protected LRU",
// Sec. II-A; these are the executor's rules):
//  * need_i = bytes of c_i's inputs not on the device + bytes of its output;
//    if inputs + output alone exceed the budget -> budget error.
//  * while resident + need_i > budget, evict one resident non-operand:
//    LRU = least recent touch (load, production, use), ties -> smaller id;
//    NEXT_USE = farthest next use in the order, ties -> larger size, then
//    smaller id.  A tensor without a host copy (an intermediate never
//    evicted before) is written back (D2H) once; others are dropped.
//  * missing inputs are loaded (H2D), left operand first; the contraction
//    runs with resident + output bytes on the device (peak_exec); releases
//    follow the model.
#include <algorithm>
#include <set>
#include <tuple>

#include "internal.hpp"

namespace lqc {

int64_t model_peak(const Dag& g, const std::vector<int64_t>& order) {
  const int64_t N = (int64_t)g.nodes.size();
  std::vector<int64_t> remaining(N);
  std::vector<uint8_t> on(N, 0);
  for (int64_t u = 0; u < N; ++u) remaining[u] = (int64_t)g.nodes[u].parents.size();
  int64_t mem = 0, peak = 0;
  for (int64_t c : order) {
    const Node& n = g.nodes[c];
    for (int k = 0; k < n.n_children(); ++k) {
      int64_t x = n.child(k);
      if (!on[x]) { on[x] = 1; mem += g.size_bytes(x); }  // leaves on first use
    }
    on[c] = 1;
    mem += g.size_bytes(c);
    for (int k = 0; k < n.n_children(); ++k) {
      int64_t x = n.child(k);
      if (--remaining[x] == 0) { on[x] = 0; mem -= g.size_bytes(x); }
    }
    if (n.parents.empty()) { on[c] = 0; mem -= g.size_bytes(c); }
    peak = std::max(peak, mem);
  }
  return peak;
}

bool plan_replay(const Dag& g, const std::vector<int64_t>& order, uint64_t budget,
                 lqc_evict evict, std::vector<Op>* ops_out, lqc_stats* st_out,
                 std::string* err) {
  const int64_t N = (int64_t)g.nodes.size();
  const bool limited = budget != 0;
  const int64_t B = limited ? (int64_t)std::min<uint64_t>(budget, (uint64_t)INT64_MAX) : 0;
  std::vector<int64_t> pos(N, -1);
  for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int64_t)i;
  // consumer positions of each tensor, ascending, and a cursor into them
  std::vector<std::vector<int64_t>> uses(N);
  for (int64_t u = 0; u < N; ++u)
    for (int64_t p : g.nodes[u].parents) uses[u].push_back(pos[p]);
  for (auto& v : uses) std::sort(v.begin(), v.end());
  std::vector<size_t> cursor(N, 0);
  std::vector<int64_t> remaining(N), touch(N, -1);
  for (int64_t u = 0; u < N; ++u) remaining[u] = (int64_t)g.nodes[u].parents.size();
  std::vector<uint8_t> resident(N, 0), host_copy(N, 0);
  for (int64_t u = 0; u < N; ++u) host_copy[u] = g.nodes[u].is_leaf() ? 1 : 0;

  // candidate sets ordered by victim preference (first = victim)
  typedef std::pair<int64_t, int64_t> LKey;                    // (touch, id)
  typedef std::tuple<int64_t, int64_t, int64_t> NKey;          // (-next, -size, id)
  std::set<LKey> lru;
  std::set<NKey> nxt;
  auto next_use = [&](int64_t x) -> int64_t {
    return cursor[x] < uses[x].size() ? uses[x][cursor[x]] : (int64_t)order.size();
  };
  auto key_add = [&](int64_t x) {
    if (evict == LQC_EVICT_LRU) lru.insert({touch[x], x});
    else nxt.insert(NKey{-next_use(x), -g.size_bytes(x), x});
  };
  auto key_del = [&](int64_t x) {
    if (evict == LQC_EVICT_LRU) lru.erase({touch[x], x});
    else nxt.erase(NKey{-next_use(x), -g.size_bytes(x), x});
  };

  std::vector<Op> ops;
  ops.reserve(order.size() * 4);
  lqc_stats st{};
  int64_t res_bytes = 0;
  for (size_t i = 0; i < order.size(); ++i) {
    const int64_t c = order[i];
    const Node& n = g.nodes[c];
    const int64_t out_b = g.size_bytes(c);
    int64_t in_b = 0, miss_b = 0;
    for (int k = 0; k < n.n_children(); ++k) {
      int64_t x = n.child(k);
      in_b += g.size_bytes(x);
      if (!resident[x]) miss_b += g.size_bytes(x);
    }
    if (limited && in_b + out_b > B) {
      *err = "contraction " + std::to_string(c) + " needs " + std::to_string(in_b + out_b) +
             " bytes (inputs + output), more than the budget " + std::to_string(B);
      return false;
    }
    const int64_t need = miss_b + out_b;
    if (limited) {
      while (res_bytes + need > B) {
        // operands of c are protected: pick the first candidate that is not one
        int64_t victim = -1;
        if (evict == LQC_EVICT_LRU) {
          for (auto it = lru.begin(); it != lru.end(); ++it)
            if (it->second != n.left && it->second != n.right) { victim = it->second; break; }
        } else {
          for (auto it = nxt.begin(); it != nxt.end(); ++it)
            if (std::get<2>(*it) != n.left && std::get<2>(*it) != n.right) {
              victim = std::get<2>(*it);
              break;
            }
        }
        if (victim < 0) {  // cannot happen when inputs + output <= budget
          *err = "no eviction candidate";
          return false;
        }
        int32_t wb = 0;
        if (!host_copy[victim]) {
          wb = 1;
          host_copy[victim] = 1;
          st.n_d2h += 1;
          st.d2h_bytes += g.size_bytes(victim);
        }
        ops.push_back(Op{OP_EVICT, wb, victim});
        st.n_evict += 1;
        key_del(victim);
        resident[victim] = 0;
        res_bytes -= g.size_bytes(victim);
      }
    }
    for (int k = 0; k < n.n_children(); ++k) {
      int64_t x = n.child(k);
      if (!resident[x]) {
        ops.push_back(Op{OP_LOAD, 0, x});
        st.n_h2d += 1;
        st.h2d_bytes += g.size_bytes(x);
        resident[x] = 1;
        res_bytes += g.size_bytes(x);
        touch[x] = (int64_t)i;
        key_add(x);
      }
    }
    ops.push_back(Op{OP_CONTRACT, 0, c});
    st.peak_exec = std::max(st.peak_exec, res_bytes + out_b);
    for (int k = 0; k < n.n_children(); ++k) {  // touch + consume the inputs
      int64_t x = n.child(k);
      key_del(x);
      touch[x] = (int64_t)i;
      cursor[x] += 1;
    }
    resident[c] = 1;
    touch[c] = (int64_t)i;
    res_bytes += out_b;
    for (int k = 0; k < n.n_children(); ++k) {
      int64_t x = n.child(k);
      if (--remaining[x] == 0) {
        ops.push_back(Op{OP_FREE, 0, x});
        resident[x] = 0;
        res_bytes -= g.size_bytes(x);
      } else {
        key_add(x);
      }
    }
    if (n.parents.empty()) {
      ops.push_back(Op{OP_FREE, 0, c});
      resident[c] = 0;
      res_bytes -= out_b;
    } else {
      key_add(c);
    }
  }
  st.peak_paper = model_peak(g, order);
  *ops_out = std::move(ops);
  *st_out = st;
  return true;
}

}  // namespace lqc
