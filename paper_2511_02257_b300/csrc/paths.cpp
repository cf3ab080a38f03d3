// Contraction-path selection (Sec. II-A: the step Redstar runs before the
// scheduler).  The terms of the correlation functions are graphs -- vertices
// are tensors (existing DAG nodes), edges are index pairs -- and each is
// reduced to one vertex by binary contractions added to the DAG.  Redstar
// counts how often each edge occurs across all contraction trees and weighs
// it with the cost of its contraction, preferring edges that recur and
// contractions that are expensive, so that a costly contraction is done once
// and reused.  Reading used:
//  * a candidate of a graph is a pair of its current vertices joined by at
//    least one edge; contracting it pairs every edge between the two.  Its
//    key is the DAG's merge key (left node, right node, left axes, right
//    axes): left = the vertex whose tensor has more elements, so that the
//    larger free extent runs over the output's rows (M >= N: full 128-row
//    GEMM tiles), ties to the smaller node id, then to the vertex whose
//    smallest axis label is smaller; pairs sorted by the left axis;
//  * value of a key = (graphs holding a candidate with that key) x (complex
//    multiply-adds, Lt * M * N * K); outputs with more elements than the
//    graph's largest input tensor are not candidates unless the graph has no
//    other;
//  * each step takes the key of largest value (ties: the smallest key,
//    compared field by field, axis lists lexicographically) and contracts it
//    in every graph that holds it, first pair first, while it does;
//    identical contractions of different graphs become one DAG node;
//  * a graph is done when one vertex is left: its root.
#include <algorithm>
#include <cstring>
#include <set>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "internal.hpp"

namespace {

// an axis of one of the graph's original vertices: vertex * LQC_MAX_RANK +
// axis, so that code order is (vertex, axis) order
using Label = int32_t;
using Wide = __int128;  // costs and values: exact for any extents (no overflow)

// (left node, right node, left axes, right axes), ordered like the tuple
// (l, r, la, ra) with the axis lists compared lexicographically
struct Key {
  int64_t l = 0, r = 0;
  int32_t n = 0;
  int8_t la[LQC_MAX_RANK] = {0}, ra[LQC_MAX_RANK] = {0};
  friend bool operator<(const Key& a, const Key& b) {
    if (a.l != b.l) return a.l < b.l;
    if (a.r != b.r) return a.r < b.r;
    const int m = std::min(a.n, b.n);
    for (int i = 0; i < m; ++i)
      if (a.la[i] != b.la[i]) return a.la[i] < b.la[i];
    if (a.n != b.n) return a.n < b.n;
    for (int i = 0; i < a.n; ++i)
      if (a.ra[i] != b.ra[i]) return a.ra[i] < b.ra[i];
    return false;
  }
  friend bool operator==(const Key& a, const Key& b) {
    return a.l == b.l && a.r == b.r && a.n == b.n && std::memcmp(a.la, b.la, a.n) == 0 &&
           std::memcmp(a.ra, b.ra, a.n) == 0;
  }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = (uint64_t)k.l * 0x9E3779B97F4A7C15ULL ^ ((uint64_t)k.r + 0x632BE59BD9B4E019ULL);
    for (int i = 0; i < k.n; ++i) h = (h ^ (uint64_t)(k.la[i] * 8 + k.ra[i] + 1)) * 0x100000001B3ULL;
    return (size_t)(h ^ (h >> 29));
  }
};

struct Vertex {
  int64_t node;
  int32_t nl = 0;
  Label labels[LQC_MAX_RANK];  // every axis of the node, in axis order
  Label min_label() const { return *std::min_element(labels, labels + nl); }
};

struct Cand {
  int x, y;     // vertex indices, x < y
  bool x_left;  // the x vertex is the left operand
  Key key;
  Wide cost;
  int64_t out_elems;
};

struct Graph {
  std::vector<Vertex> verts;
  std::vector<Label> partner;  // label -> paired label, -1 = open axis
  int64_t cap = 0;
};

bool candidate(const lqc::Dag& g, const Vertex& p, const Vertex& q,
               const std::vector<Label>& partner, Cand* c) {
  int pi[LQC_MAX_RANK], qj[LQC_MAX_RANK], np = 0;
  for (int i = 0; i < p.nl; ++i) {
    const Label other = partner[p.labels[i]];
    if (other < 0) continue;
    for (int j = 0; j < q.nl; ++j)
      if (q.labels[j] == other) {
        pi[np] = i;
        qj[np++] = j;
        break;
      }
  }
  if (np == 0) return false;
  const int64_t pe = g.nodes[p.node].elems, qe = g.nodes[q.node].elems;
  const Label pmin = p.min_label(), qmin = q.min_label();
  const bool p_left = pe != qe ? pe > qe : (p.node != q.node ? p.node < q.node : pmin <= qmin);
  const Vertex& L = p_left ? p : q;
  const Vertex& R = p_left ? q : p;
  Key& k = c->key;
  k = Key();
  k.l = L.node;
  k.r = R.node;
  k.n = np;
  for (int t = 0; t < np; ++t) {  // pairs by ascending left axis
    k.la[t] = (int8_t)(p_left ? pi[t] : qj[t]);
    k.ra[t] = (int8_t)(p_left ? qj[t] : pi[t]);
  }
  for (int t = 1; t < np; ++t)
    for (int s = t; s > 0 && k.la[s - 1] > k.la[s]; --s) {
      std::swap(k.la[s - 1], k.la[s]);
      std::swap(k.ra[s - 1], k.ra[s]);
    }
  const lqc::Node& ln = g.nodes[L.node];
  const lqc::Node& rn = g.nodes[R.node];
  int64_t kext = 1;
  for (int t = 0; t < np; ++t) kext *= ln.ext[k.la[t]];
  const int64_t m = ln.elems / kext, n = rn.elems / kext;
  c->cost = (Wide)ln.lt * m * n * kext;
  c->out_elems = m * n;
  c->x_left = p_left;
  return true;
}

void candidates(const lqc::Dag& g, const Graph& G, std::vector<Cand>* out) {
  out->clear();
  for (int x = 0; x < (int)G.verts.size(); ++x)
    for (int y = x + 1; y < (int)G.verts.size(); ++y) {
      Cand c;
      if (candidate(g, G.verts[x], G.verts[y], G.partner, &c)) {
        c.x = x;
        c.y = y;
        out->push_back(c);
      }
    }
  bool any_fits = false;
  for (const Cand& c : *out) any_fits |= c.out_elems <= G.cap;
  if (any_fits)
    out->erase(std::remove_if(out->begin(), out->end(),
                              [&](const Cand& c) { return c.out_elems > G.cap; }),
               out->end());
}

// true when every vertex of the graph is reached from vertex 0 by its edges
bool connected(int nv, const int32_t* edges, int64_t ne) {
  std::vector<int> parent(nv);
  for (int v = 0; v < nv; ++v) parent[v] = v;
  auto find = [&](int v) {
    while (parent[v] != v) v = parent[v] = parent[parent[v]];
    return v;
  };
  int parts = nv;
  for (int64_t e = 0; e < ne; ++e) {
    const int a = find(edges[4 * e]), b = find(edges[4 * e + 2]);
    if (a != b) {
      parent[a] = b;
      --parts;
    }
  }
  return parts == 1;
}

// remove the nodes from id n0 on (the contractions one call added), newest
// first: each is the last consumer of its operands and has a merge entry
void roll_back(lqc::Dag& g, int64_t n0) {
  for (int64_t u = (int64_t)g.nodes.size() - 1; u >= n0; --u) {
    const lqc::Node& n = g.nodes[u];
    for (int c = 0; c < n.n_children(); ++c) {
      auto& par = g.nodes[n.child(c)].parents;
      if (!par.empty() && par.back() == u) par.pop_back();
    }
    g.nodes.pop_back();
  }
  for (auto it = g.dedup.begin(); it != g.dedup.end();)
    it = it->second >= n0 ? g.dedup.erase(it) : std::next(it);
}

}  // namespace

extern "C" int lqc_dag_add_graphs(lqc_dag* h, int64_t n_graphs, const int64_t* vert_off,
                                  const int64_t* vert_nodes, const int64_t* edge_off,
                                  const int32_t* edges, int64_t* roots) {
  if (!h) return LQC_ERR_ARG;
  lqc::Dag& g = h->d;
  int64_t n0 = -1;  // first node this call adds, once validation passed
  try {
    if (g.frozen) {
      g.err = "DAG is frozen by lqc_dag_schedule";
      return LQC_ERR_STATE;
    }
    if (n_graphs < 0 || (n_graphs > 0 && (!vert_off || !vert_nodes || !edge_off || !roots))) {
      g.err = "null graph arrays";
      return LQC_ERR_ARG;
    }
    const int64_t N = (int64_t)g.nodes.size();
    std::vector<Graph> graphs((size_t)n_graphs);
    for (int64_t gi = 0; gi < n_graphs; ++gi) {
      Graph& G = graphs[gi];
      const int64_t v0 = vert_off[gi], v1 = vert_off[gi + 1];
      const int64_t e0 = edge_off[gi], e1 = edge_off[gi + 1];
      if (v0 < 0 || e0 < 0 || v1 <= v0 || e1 < e0 || (e1 > e0 && !edges) ||
          v1 - v0 > ((int64_t)1 << 24)) {
        g.err = "graph " + std::to_string(gi) + ": empty or bad offsets";
        return LQC_ERR_ARG;
      }
      const int nv = (int)(v1 - v0);
      G.partner.assign((size_t)nv * LQC_MAX_RANK, -1);
      for (int64_t v = v0; v < v1; ++v) {
        const int64_t u = vert_nodes[v];
        if (u < 0 || u >= N || g.nodes[u].rank == 0) {
          g.err = "graph " + std::to_string(gi) + ": vertex is no tensor node";
          return LQC_ERR_ARG;
        }
        Vertex vx;
        vx.node = u;
        vx.nl = g.nodes[u].rank;
        for (int a = 0; a < vx.nl; ++a) vx.labels[a] = (Label)((v - v0) * LQC_MAX_RANK + a);
        G.cap = std::max(G.cap, g.nodes[u].elems);
        G.verts.push_back(vx);
      }
      for (int64_t e = e0; e < e1; ++e) {
        const int32_t* q = edges + 4 * e;
        if (q[0] < 0 || q[0] >= nv || q[2] < 0 || q[2] >= nv || q[0] == q[2] || q[1] < 0 ||
            q[1] >= g.nodes[vert_nodes[v0 + q[0]]].rank || q[3] < 0 ||
            q[3] >= g.nodes[vert_nodes[v0 + q[2]]].rank) {
          g.err = "graph " + std::to_string(gi) + ": edge out of range";
          return LQC_ERR_ARG;
        }
        const Label a = q[0] * LQC_MAX_RANK + q[1], b = q[2] * LQC_MAX_RANK + q[3];
        if (G.partner[a] >= 0 || G.partner[b] >= 0) {
          g.err = "graph " + std::to_string(gi) + ": an axis is paired twice";
          return LQC_ERR_ARG;
        }
        if (g.nodes[vert_nodes[v0 + q[0]]].ext[q[1]] != g.nodes[vert_nodes[v0 + q[2]]].ext[q[3]]) {
          g.err = "graph " + std::to_string(gi) + ": paired extents differ";
          return LQC_ERR_ARG;
        }
        G.partner[a] = b;
        G.partner[b] = a;
      }
      if (!connected(nv, edges + 4 * e0, e1 - e0)) {
        g.err = "graph " + std::to_string(gi) + " is not connected";
        return LQC_ERR_ARG;
      }
    }
    // from here on contractions are added; a failure removes them again
    n0 = (int64_t)g.nodes.size();
    // Key values are kept incrementally: a step changes the candidates of
    // only the graphs it contracts in, and of those only the keys that
    // appear or disappear are recounted.  The result equals recounting
    // every graph at every step.
    struct KeyStat {
      int64_t count = 0;
      Wide cost = 0;
      std::set<int64_t> graphs;
    };
    std::unordered_map<Key, KeyStat, KeyHash> stat;
    // max-heap on (value, -key) with lazy invalidation: every change of a
    // key's value pushes its new value; an entry whose value is no longer
    // the key's is dropped when it reaches the top
    typedef std::pair<Wide, Key> HE;
    auto worse = [](const HE& a, const HE& b) {
      if (a.first != b.first) return a.first < b.first;
      return b.second < a.second;
    };
    std::vector<HE> heap;
    auto push = [&](const Key& k, const KeyStat& ks) {
      heap.push_back({ks.count * ks.cost, k});
      std::push_heap(heap.begin(), heap.end(), worse);
    };
    std::vector<std::vector<std::pair<Key, Wide>>> held((size_t)n_graphs);  // sorted keys
    std::vector<Cand> cs;
    std::vector<std::pair<Key, Wide>> now;
    auto add_key = [&](int64_t gi, const Key& k, Wide cost) {
      KeyStat& ks = stat[k];
      ks.count += 1;
      ks.cost = cost;
      ks.graphs.insert(gi);
      push(k, ks);
    };
    auto drop_key = [&](int64_t gi, const Key& k) {
      auto it = stat.find(k);
      KeyStat& ks = it->second;
      ks.count -= 1;
      ks.graphs.erase(gi);
      if (ks.count)
        push(k, ks);
      else
        stat.erase(it);
    };
    // the graph's current keys replace held[gi]: only the difference is
    // applied to the counts
    auto refresh = [&](int64_t gi, bool cs_current) {
      const Graph& G = graphs[gi];
      now.clear();
      if (G.verts.size() >= 2) {
        if (!cs_current) candidates(g, G, &cs);
        for (const Cand& c : cs) now.push_back({c.key, c.cost});
        std::sort(now.begin(), now.end(),
                  [](const std::pair<Key, Wide>& a, const std::pair<Key, Wide>& b) {
                    return a.first < b.first;
                  });
        now.erase(std::unique(now.begin(), now.end(),
                              [](const std::pair<Key, Wide>& a, const std::pair<Key, Wide>& b) {
                                return a.first == b.first;
                              }),
                  now.end());
      }
      auto& old = held[gi];
      size_t i = 0, j = 0;
      while (i < old.size() || j < now.size()) {
        if (j == now.size() || (i < old.size() && old[i].first < now[j].first)) {
          drop_key(gi, old[i++].first);
        } else if (i == old.size() || now[j].first < old[i].first) {
          add_key(gi, now[j].first, now[j].second);
          ++j;
        } else {
          ++i;
          ++j;
        }
      }
      old.swap(now);
    };
    for (int64_t gi = 0; gi < n_graphs; ++gi) refresh(gi, false);
    std::vector<int64_t> hold;
    for (;;) {
      if (heap.size() > 2 * stat.size() + 4096) {  // drop stale entries
        heap.clear();
        for (auto& kv : stat) heap.push_back({kv.second.count * kv.second.cost, kv.first});
        std::make_heap(heap.begin(), heap.end(), worse);
      }
      bool found = false;
      while (!heap.empty()) {
        std::pop_heap(heap.begin(), heap.end(), worse);
        const HE top = heap.back();
        heap.pop_back();
        auto it = stat.find(top.second);
        if (it != stat.end() && it->second.count * it->second.cost == top.first) {
          heap.push_back(top);  // still current: keep it until the key is used up
          std::push_heap(heap.begin(), heap.end(), worse);
          found = true;
          break;
        }
      }
      if (!found) break;
      const Key bk = heap.front().second;
      const std::set<int64_t>& holders = stat[bk].graphs;
      hold.assign(holders.begin(), holders.end());
      for (int64_t gi : hold) {
        Graph& G = graphs[gi];
        bool cs_current = false;
        while (G.verts.size() >= 2) {
          candidates(g, G, &cs);
          cs_current = true;
          const Cand* hit = nullptr;
          for (const Cand& c : cs)
            if (c.key == bk) {
              hit = &c;
              break;
            }
          if (!hit) break;
          int la[LQC_MAX_RANK], ra[LQC_MAX_RANK];
          for (int t = 0; t < bk.n; ++t) {
            la[t] = bk.la[t];
            ra[t] = bk.ra[t];
          }
          int64_t node = -1;
          const int rc = lqc_dag_add_contraction(h, bk.l, bk.r, bk.n, la, ra, &node);
          if (rc != LQC_OK) {
            const std::string why = g.err;
            roll_back(g, n0);
            g.err = "graph " + std::to_string(gi) + ": " + why + " (no contraction added)";
            return rc;
          }
          const Vertex& Lv = G.verts[hit->x_left ? hit->x : hit->y];
          const Vertex& Rv = G.verts[hit->x_left ? hit->y : hit->x];
          Vertex nv;
          nv.node = node;
          for (int i = 0; i < Lv.nl; ++i)
            if (std::find(la, la + bk.n, i) == la + bk.n) nv.labels[nv.nl++] = Lv.labels[i];
          for (int j = 0; j < Rv.nl; ++j)
            if (std::find(ra, ra + bk.n, j) == ra + bk.n) nv.labels[nv.nl++] = Rv.labels[j];
          const int x = hit->x, y = hit->y;
          G.verts[x] = nv;
          G.verts.erase(G.verts.begin() + y);
          cs_current = false;
        }
        refresh(gi, cs_current);
      }
    }
    for (int64_t gi = 0; gi < n_graphs; ++gi) {
      if (graphs[gi].verts.size() != 1) {  // not reached for connected graphs
        roll_back(g, n0);
        g.err = "graph " + std::to_string(gi) + " was not reduced to one node";
        return LQC_ERR_ARG;
      }
    }
    for (int64_t gi = 0; gi < n_graphs; ++gi) roots[gi] = graphs[gi].verts[0].node;
    return LQC_OK;
  } catch (const std::bad_alloc&) {
    if (n0 >= 0) roll_back(g, n0);
    g.err = "host allocation failed";
    return LQC_ERR_HOST_MEM;
  }
}
