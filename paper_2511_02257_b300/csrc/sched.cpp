// Contraction orders: naive topological order, the sibling scheduler
// (Sec. III-A, Alg. 1 SB-SCHEDULER, Alg. 2 SB-PROCESS, Alg. 3 SB-PROP-DOWN)
// and the tree scheduler (Sec. III-B, Alg. 4 TR-SCHEDULER, Alg. 5 TR-INIT,
// Alg. 6 PROCESS-CTREE, Alg. 7 PROCESS-CHILD, Alg. 8 PROCESS-NODE).
//
// Each scheduler returns the order of the non-leaf nodes.  Deterministic
// readings of the points the paper leaves open:
//  * sibling: the "random" WAITING leaf is the smallest-id WAITING leaf that
//    has a consumer; queues are FIFO; parents are visited in ascending id;
//    children and parents are sets of distinct nodes.
//  * tree: T_i = descendant closure of the i-th root (ascending root id);
//    the initial tgain is the sum of the individual gains (the text's
//    definition); ties of max tgain go to the smallest tree index;
//    PROCESS-CHILD updates x.outAv (the printed "v.outAv" is a typo); the
//    nodes of a tree are visited by a post-order walk from its root, left
//    operand first, skipping nodes (and their sub-trees) that an earlier
//    tree already processed.
// Two schedulers the paper only names, with these readings:
//  * node (Sec. VI, future work: a node-based scheduler using the tree
//    scheduler's gain concept): each step takes, among the contractions whose
//    non-leaf inputs are computed, the one whose processing lowers the
//    resident memory of the model (Sec. II-C) the most: gain = bytes of the
//    inputs it releases (their last pending consumer) - bytes of the leaves
//    it loads - its output bytes (none for a root); ties to the smallest id.
//  * rsgs (Sec. II-A, Redstar's trees sorted by similarity): the first tree
//    (smallest root id), then repeatedly the unprocessed tree sharing the
//    most contractions with the tree processed last (ties to the smallest
//    index); each tree's not yet processed contractions in the same
//    post-order walk as the tree scheduler's.
#include <pthread.h>

#include <algorithm>
#include <deque>
#include <queue>
#include <stdexcept>

#include "internal.hpp"

namespace lqc {

std::vector<int64_t> schedule_naive(const Dag& g) {
  std::vector<int64_t> o;
  for (int64_t u = 0; u < (int64_t)g.nodes.size(); ++u)
    if (!g.nodes[u].is_leaf()) o.push_back(u);
  return o;
}

// ---------------------------------------------------------------- sibling
namespace {

enum SibState : uint8_t { SB_WAITING, SB_QUEUED, SB_INMEM, SB_RELEASED };

struct Sibling {
  const Dag& g;
  std::vector<int32_t> rank;
  std::vector<int32_t> rs, rp;
  std::vector<uint8_t> st;
  std::vector<std::deque<int64_t>> Q;  // Q[r]: contractions of rank r
  std::vector<int64_t> order;
  bool failed = false;

  explicit Sibling(const Dag& d) : g(d) {}

  void process(int64_t u) {  // Alg. 2
    const Node& n = g.nodes[u];
    if (!n.is_leaf()) order.push_back(u);  // perform the contraction
    st[u] = SB_INMEM;
    if (!n.is_leaf()) {
      for (int c = 0; c < n.n_children(); ++c) {
        int64_t v = n.child(c);
        if (--rs[v] == 0) st[v] = SB_RELEASED;
      }
      if (n.parents.empty()) st[u] = SB_RELEASED;  // ROOT
    }
    for (int64_t v : n.parents) {
      --rp[v];
      if (rp[v] == 1) {
        const Node& pv = g.nodes[v];
        int64_t w = (pv.left == u) ? pv.right : pv.left;  // the sibling of u
        if (st[w] == SB_WAITING) prop_down(w);
      } else if (rp[v] == 0) {
        Q[rank[v]].push_back(v);
        st[v] = SB_QUEUED;
      }
    }
  }

  void prop_down(int64_t u) {  // Alg. 3
    if (st[u] != SB_WAITING) return;
    const Node& n = g.nodes[u];
    if (n.is_leaf()) {
      process(u);
      return;
    }
    prop_down(n.left);
    prop_down(n.right);
  }

  void run() {  // Alg. 1
    const int64_t N = (int64_t)g.nodes.size();
    rank.assign(N, 0);
    rs.assign(N, 0);
    rp.assign(N, 0);
    st.assign(N, SB_WAITING);
    int32_t q = 0;
    int64_t n_contr = 0;
    std::vector<int64_t> leaves;
    for (int64_t u = 0; u < N; ++u) {
      const Node& n = g.nodes[u];
      rs[u] = (int32_t)n.parents.size();
      rp[u] = n.n_children();
      if (n.is_leaf()) {
        if (!n.parents.empty()) leaves.push_back(u);
      } else {
        int32_t r = 0;
        for (int c = 0; c < n.n_children(); ++c) r = std::max(r, rank[n.child(c)]);
        rank[u] = r + 1;  // Eq. (1)
        q = std::max(q, rank[u]);
        ++n_contr;
      }
    }
    Q.assign(q + 1, std::deque<int64_t>());
    size_t leaf_ptr = 0;
    while ((int64_t)order.size() < n_contr) {
      int32_t top = -1;
      for (int32_t r = q; r >= 1; --r)
        if (!Q[r].empty()) { top = r; break; }
      int64_t u;
      if (top < 0) {
        while (leaf_ptr < leaves.size() && st[leaves[leaf_ptr]] != SB_WAITING) ++leaf_ptr;
        if (leaf_ptr >= leaves.size()) { failed = true; return; }
        u = leaves[leaf_ptr];
      } else {
        u = Q[top].front();
        Q[top].pop_front();
      }
      process(u);
    }
  }
};

void* sibling_thread(void* p) {
  Sibling* s = static_cast<Sibling*>(p);
  try {
    s->run();
  } catch (...) {
    s->failed = true;
  }
  return nullptr;
}

}  // namespace

std::vector<int64_t> schedule_sibling(const Dag& g) {
  // The paper's routines recurse (PROCESS -> PROP-DOWN -> PROCESS ...); the
  // depth grows with the sharing in the DAG, so run them on a thread with a
  // large stack.
  Sibling s(g);
  pthread_attr_t attr;
  pthread_attr_init(&attr);
  pthread_attr_setstacksize(&attr, (size_t)1 << 30);
  pthread_t th;
  if (pthread_create(&th, &attr, sibling_thread, &s) != 0) {
    pthread_attr_destroy(&attr);
    throw std::runtime_error("sibling scheduler: cannot start worker thread");
  }
  pthread_join(th, nullptr);
  pthread_attr_destroy(&attr);
  if (s.failed) throw std::runtime_error("sibling scheduler failed");
  return s.order;
}

// ------------------------------------------------------------------- tree
namespace {

enum TrState : uint8_t { TR_AVAIL, TR_INMEM, TR_RELEASED };

struct TreeSched {
  const Dag& g;
  int64_t N = 0;
  int32_t K = 0;
  std::vector<int64_t> root;                  // root of tree i
  std::vector<std::vector<int32_t>> ctree;    // u.ctree, ascending
  std::vector<std::vector<int64_t>> igain;    // T_i.u.igain aligned with ctree[u]
  std::vector<int64_t> cgain, tgain;
  std::vector<uint8_t> state;
  std::vector<int64_t> outav;                 // |u.outAv|
  // tau/delta of a node x per tree (Alg. 7-8), kept implicitly: tau =
  // tau0 - in (parents of x in the tree processed so far), delta = delta0 -
  // (pc - in) with pc = parents of x processed so far.  A tree's "delta
  // reaches 0" event (case 2b) fires at the call that makes pc equal
  // th = delta0 + in, so each entry waits in the bucket of its threshold
  // and a call visits only the trees of its parent u (cases 1a-1c) and the
  // bucket of the new pc, instead of every tree of x.
  struct Ent {       // one per tree of x, aligned with ctree[x]
    int32_t tau;     // tau0 - in; tau0 = parents of x in the tree
    int32_t delta0;
    int32_t in;
    uint8_t inpred;  // x in T_tree.pred (a tree without parents of x never is)
  };
  struct XState {
    std::vector<Ent> ent;
    std::vector<int32_t> head;                  // threshold -> first pool link, -1 = none
    std::vector<std::pair<int32_t, int32_t>> pool;  // (entry, next link)
    int32_t pc = 0;
    void bucket_push(int32_t th, int32_t k) {
      pool.push_back({k, head[th]});
      head[th] = (int32_t)pool.size() - 1;
    }
  };
  std::vector<XState> S;                      // set by PROCESS-NODE
  std::vector<int32_t> pos_of;                // scratch: tree -> index in ctree[u]
  std::vector<uint8_t> alive, dirty_flag;
  std::vector<int32_t> dirty;
  std::vector<int64_t> visit_stamp;
  std::vector<int64_t> order;

  explicit TreeSched(const Dag& d) : g(d) {}

  void touch(int32_t i) {
    if (!dirty_flag[i]) { dirty_flag[i] = 1; dirty.push_back(i); }
  }

  void init() {  // Alg. 5 TR-INIT
    N = (int64_t)g.nodes.size();
    for (int64_t u = 0; u < N; ++u)
      if (!g.nodes[u].is_leaf() && g.nodes[u].parents.empty()) root.push_back(u);
    K = (int32_t)root.size();
    ctree.assign(N, {});
    igain.assign(N, {});
    state.assign(N, TR_AVAIL);
    outav.assign(N, 0);
    for (int64_t u = 0; u < N; ++u) outav[u] = (int64_t)g.nodes[u].parents.size();
    cgain.assign(K, 0);
    tgain.assign(K, 0);
    std::vector<int64_t> mark(N, -1), stack;
    for (int32_t i = 0; i < K; ++i) {  // u.ctree: descendant closure of each root
      stack.clear();
      stack.push_back(root[i]);
      mark[root[i]] = i;
      while (!stack.empty()) {
        int64_t u = stack.back();
        stack.pop_back();
        ctree[u].push_back(i);
        const Node& n = g.nodes[u];
        for (int c = 0; c < n.n_children(); ++c) {
          int64_t v = n.child(c);
          if (mark[v] != i) { mark[v] = i; stack.push_back(v); }
        }
      }
    }
    // individual gains: g(u, T_i) = |outAv(u)| - #{parents of u in T_i};
    // the parents in each tree are counted in one pass over the parents'
    // tree lists (a parent's trees all contain u)
    std::vector<int32_t> in_count(K, 0);
    for (int64_t u = 0; u < N; ++u) {
      const auto& cu = ctree[u];
      const auto& par = g.nodes[u].parents;
      for (int64_t v : par)
        for (int32_t i : ctree[v]) ++in_count[i];
      igain[u].assign(cu.size(), 0);
      for (size_t k = 0; k < cu.size(); ++k) {
        const int64_t gcount = (int64_t)par.size() - in_count[cu[k]];
        igain[u][k] = gcount == 0 ? 0 : -g.size_bytes(u);
        tgain[cu[k]] += igain[u][k];
      }
      for (int64_t v : par)
        for (int32_t i : ctree[v]) in_count[i] = 0;
    }
    S.assign(N, {});
    pos_of.assign(K, -1);
    alive.assign(K, 1);
    dirty_flag.assign(K, 0);
    visit_stamp.assign(N, -1);
  }

  void process_child(int64_t u, int64_t x) {  // Alg. 7
    const int64_t sz = g.size_bytes(x);
    XState& xs = S[x];
    const int32_t pc_before = xs.pc++;
    // cases 1a-1c: the trees of u (each is a tree of x)
    const auto& cx = ctree[x];
    for (int32_t i : ctree[u]) {
      const int32_t k = (int32_t)(std::lower_bound(cx.begin(), cx.end(), i) - cx.begin());
      Ent& e = xs.ent[k];
      if (!e.inpred) continue;
      const int32_t delta = e.delta0 - (pc_before - e.in);
      if (e.tau == 1 && delta == 0) {
        cgain[i] -= sz;
        tgain[i] -= sz;
        touch(i);
      }
      ++e.in;
      if (--e.tau == 0) {
        e.inpred = 0;
      } else {
        // delta = th - pc: only a threshold still ahead can fire later (a
        // tree whose outside parents are all processed has delta 0 for good)
        const int32_t th = e.delta0 + e.in;
        if (th > xs.pc && th < (int32_t)xs.head.size()) xs.bucket_push(th, k);
      }
    }
    // cases 2a-2b: every other live tree loses one outside parent; delta
    // goes 1 -> 0 for those whose threshold is the new pc
    if (xs.pc < (int32_t)xs.head.size()) {
      for (int32_t l = xs.head[xs.pc]; l >= 0; l = xs.pool[l].second) {
        const int32_t k = xs.pool[l].first;
        const Ent& e = xs.ent[k];
        if (e.inpred && e.delta0 + e.in == xs.pc) {
          const int32_t i = cx[k];
          cgain[i] += sz;
          tgain[i] += sz;
          touch(i);
        }
      }
    }
    if (--outav[x] == 0) {
      state[x] = TR_RELEASED;
      XState().ent.swap(xs.ent);
      std::vector<int32_t>().swap(xs.head);
      std::vector<std::pair<int32_t, int32_t>>().swap(xs.pool);
    }
  }

  void process_node(int64_t u) {  // Alg. 8
    const int64_t sz = g.size_bytes(u);
    const auto& cu = ctree[u];
    for (size_t k = 0; k < cu.size(); ++k) {
      if (igain[u][k] != 0) {
        tgain[cu[k]] -= igain[u][k];
        touch(cu[k]);
      }
    }
    // every consumer of an AVAIL node is AVAIL, so u.outAv = u.parents here
    const int32_t n_out = (int32_t)outav[u];
    XState& xs = S[u];
    std::vector<Ent>& su = xs.ent;
    su.assign(cu.size(), Ent{0, n_out, 0, 0});
    for (size_t k = 0; k < cu.size(); ++k) pos_of[cu[k]] = (int32_t)k;
    for (int64_t v : g.nodes[u].parents) {
      for (int32_t i : ctree[v]) {  // a parent's trees all hold u
        Ent& e = su[pos_of[i]];
        --e.delta0;
        ++e.tau;
      }
    }
    for (int32_t i : cu) pos_of[i] = -1;
    xs.pc = 0;
    xs.head.assign((size_t)n_out + 1, -1);
    xs.pool.clear();
    for (size_t k = 0; k < cu.size(); ++k) {
      Ent& e = su[k];
      if (e.tau == 0) continue;  // no parent of u in this tree: no entry
      e.inpred = 1;
      if (e.delta0 == 0) {
        cgain[cu[k]] += sz;
        tgain[cu[k]] += sz;
        touch(cu[k]);
      } else {
        xs.bucket_push(e.delta0, (int32_t)k);
      }
    }
    state[u] = outav[u] == 0 ? TR_RELEASED : TR_INMEM;
  }

  void process_ctree(int32_t i) {  // Alg. 6
    // post-order from the root, left operand first, AVAIL nodes only
    struct Frame { int64_t u; int c; };
    std::vector<Frame> st;
    int64_t r = root[i];
    if (state[r] != TR_AVAIL) return;
    visit_stamp[r] = i;
    st.push_back({r, 0});
    while (!st.empty()) {
      Frame& f = st.back();
      const Node& n = g.nodes[f.u];
      if (f.c < n.n_children()) {
        int64_t v = n.child(f.c++);
        if (state[v] == TR_AVAIL && visit_stamp[v] != i) {
          visit_stamp[v] = i;
          st.push_back({v, 0});
        }
        continue;
      }
      int64_t u = f.u;
      st.pop_back();
      if (!n.is_leaf())
        for (int c = 0; c < n.n_children(); ++c) process_child(u, n.child(c));
      process_node(u);
      if (!n.is_leaf()) order.push_back(u);
    }
  }

  // indexed binary max-heap of the alive trees on (tgain, -index): a
  // changed gain is sifted in place, so the heap never holds stale entries.
  // The heap compares its own copy of the gains (hkey), brought up to date
  // one tree at a time, so every sift runs on a valid heap.
  std::vector<int32_t> heap, hpos;
  std::vector<int64_t> hkey;
  bool above(int32_t a, int32_t b) const {  // a before b
    return hkey[a] != hkey[b] ? hkey[a] > hkey[b] : a < b;
  }
  void hswap(size_t x, size_t y) {
    std::swap(heap[x], heap[y]);
    hpos[heap[x]] = (int32_t)x;
    hpos[heap[y]] = (int32_t)y;
  }
  void sift_up(size_t x) {
    while (x > 0 && above(heap[x], heap[(x - 1) / 2])) {
      hswap(x, (x - 1) / 2);
      x = (x - 1) / 2;
    }
  }
  void sift_down(size_t x) {
    for (;;) {
      size_t b = x, l = 2 * x + 1, r = l + 1;
      if (l < heap.size() && above(heap[l], heap[b])) b = l;
      if (r < heap.size() && above(heap[r], heap[b])) b = r;
      if (b == x) return;
      hswap(x, b);
      x = b;
    }
  }

  void run() {  // Alg. 4
    init();
    heap.resize(K);
    hpos.resize(K);
    hkey = tgain;
    for (int32_t i = 0; i < K; ++i) { heap[i] = i; hpos[i] = i; }
    for (int32_t x = K / 2 - 1; x >= 0; --x) sift_down((size_t)x);
    for (int32_t step = 0; step < K; ++step) {
      for (int32_t i : dirty) {
        dirty_flag[i] = 0;
        if (alive[i] && hkey[i] != tgain[i]) {
          hkey[i] = tgain[i];
          sift_up((size_t)hpos[i]);
          sift_down((size_t)hpos[i]);
        }
      }
      dirty.clear();
      if (heap.empty()) throw std::runtime_error("tree scheduler: empty selection");
      const int32_t best = heap[0];
      hswap(0, heap.size() - 1);
      heap.pop_back();
      if (!heap.empty()) sift_down(0);
      alive[best] = 0;
      process_ctree(best);
    }
  }
};

}  // namespace

// ------------------------------------------------------------------- node
std::vector<int64_t> schedule_node(const Dag& g) {
  const int64_t N = (int64_t)g.nodes.size();
  std::vector<int64_t> pending(N), missing(N, 0), version(N, 0), order;
  std::vector<uint8_t> resident(N, 0), done(N, 0);
  for (int64_t u = 0; u < N; ++u) {
    const Node& n = g.nodes[u];
    pending[u] = (int64_t)n.parents.size();
    for (int k = 0; k < n.n_children(); ++k)
      if (!g.nodes[n.child(k)].is_leaf()) ++missing[u];
  }
  auto gain = [&](int64_t u) {
    const Node& n = g.nodes[u];
    int64_t v = 0;
    for (int k = 0; k < n.n_children(); ++k) {
      const int64_t x = n.child(k);
      if (g.nodes[x].is_leaf() && !resident[x]) v -= g.size_bytes(x);
      if (pending[x] == 1) v += g.size_bytes(x);
    }
    if (!n.parents.empty()) v -= g.size_bytes(u);
    return v;
  };
  struct Ent {
    int64_t gain, id, ver;
    bool operator<(const Ent& o) const {  // max gain first, then smallest id
      return gain != o.gain ? gain < o.gain : id > o.id;
    }
  };
  std::priority_queue<Ent> heap;
  auto push = [&](int64_t u) { heap.push(Ent{gain(u), u, ++version[u]}); };
  for (int64_t u = 0; u < N; ++u)
    if (!g.nodes[u].is_leaf() && missing[u] == 0) push(u);
  // a node's gain changes only when one of its children changes residency
  // or reaches one pending consumer: re-key the available parents
  auto rekey_parents = [&](int64_t x) {
    for (int64_t p : g.nodes[x].parents)
      if (!done[p] && missing[p] == 0) push(p);
  };
  while (!heap.empty()) {
    const Ent e = heap.top();
    heap.pop();
    if (done[e.id] || e.ver != version[e.id]) continue;  // stale entry
    const int64_t u = e.id;
    const Node& n = g.nodes[u];
    done[u] = 1;
    order.push_back(u);
    for (int k = 0; k < n.n_children(); ++k) {
      const int64_t x = n.child(k);
      const bool was_resident = resident[x];
      if (g.nodes[x].is_leaf()) resident[x] = 1;
      if (--pending[x] == 0) resident[x] = 0;
      if ((g.nodes[x].is_leaf() && !was_resident) || pending[x] == 1) rekey_parents(x);
    }
    if (!n.parents.empty()) resident[u] = 1;
    for (int64_t p : n.parents)
      if (--missing[p] == 0 && !done[p]) push(p);
  }
  return order;
}

// ------------------------------------------------------------------- rsgs
std::vector<int64_t> schedule_rsgs(const Dag& g) {
  const int64_t N = (int64_t)g.nodes.size();
  std::vector<int64_t> roots;
  for (int64_t u = 0; u < N; ++u)
    if (!g.nodes[u].is_leaf() && g.nodes[u].parents.empty()) roots.push_back(u);
  const int64_t K = (int64_t)roots.size();
  // trees containing each contraction (descendant closures of the roots)
  std::vector<std::vector<int32_t>> trees_of(N);
  std::vector<int64_t> stamp(N, -1), stack;
  for (int64_t i = 0; i < K; ++i) {
    stack.assign(1, roots[i]);
    while (!stack.empty()) {
      const int64_t u = stack.back();
      stack.pop_back();
      if (stamp[u] == i || g.nodes[u].is_leaf()) continue;
      stamp[u] = i;
      trees_of[u].push_back((int32_t)i);
      for (int k = 0; k < g.nodes[u].n_children(); ++k) stack.push_back(g.nodes[u].child(k));
    }
  }
  std::vector<uint8_t> done(N, 0), used(K, 0);
  std::vector<int64_t> order, shared(K, 0), seen(N, -1);
  std::vector<int32_t> touched;
  int64_t next_unused = 0;
  std::vector<std::pair<int64_t, bool>> walk;
  int64_t cur = K ? 0 : -1;
  while (cur >= 0) {
    used[cur] = 1;
    walk.assign(1, {roots[cur], false});  // post-order, left operand first
    while (!walk.empty()) {
      auto [u, expanded] = walk.back();
      walk.pop_back();
      const Node& n = g.nodes[u];
      if (n.is_leaf() || done[u]) continue;
      if (expanded) {
        done[u] = 1;
        order.push_back(u);
        continue;
      }
      walk.push_back({u, true});
      for (int k = n.n_children() - 1; k >= 0; --k) walk.push_back({n.child(k), false});
    }
    // contractions shared by the tree just processed and every other tree;
    // only trees met here can share any, the rest count 0
    touched.clear();
    stack.assign(1, roots[cur]);
    while (!stack.empty()) {
      const int64_t u = stack.back();
      stack.pop_back();
      if (seen[u] == cur || g.nodes[u].is_leaf()) continue;
      seen[u] = cur;
      for (int32_t j : trees_of[u])
        if (shared[j]++ == 0) touched.push_back(j);
      for (int k = 0; k < g.nodes[u].n_children(); ++k) stack.push_back(g.nodes[u].child(k));
    }
    // the unused tree sharing the most, ties to the smallest index; with
    // none sharing, the smallest unused index
    int64_t best = -1;
    for (int32_t j : touched)
      if (!used[j] && (best < 0 || shared[j] > shared[best] ||
                       (shared[j] == shared[best] && j < best)))
        best = j;
    for (int32_t j : touched) shared[j] = 0;
    while (next_unused < K && used[next_unused]) ++next_unused;
    if (best < 0 && next_unused < K) best = next_unused;
    cur = best;
  }
  return order;
}

std::vector<int64_t> schedule_tree(const Dag& g) {
  TreeSched t(g);
  t.run();
  return t.order;
}

}  // namespace lqc
