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
#include <map>
#include <set>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "internal.hpp"

namespace {

using Label = std::pair<int32_t, int32_t>;  // (vertex of the graph, axis)
using Key = std::tuple<int64_t, int64_t, std::vector<int>, std::vector<int>>;
using Wide = __int128;  // costs and values: exact for any extents (no overflow)

struct Vertex {
  int64_t node;
  std::vector<Label> labels;  // every axis of the node, in axis order
};

struct Cand {
  int x, y;  // vertex indices, x < y
  Key key;
  Wide cost;
  int64_t out_elems;
  const Vertex* left;
  const Vertex* right;
};

struct Graph {
  std::vector<Vertex> verts;
  std::map<Label, Label> partner;
  int64_t cap = 0;
};

bool candidate(const lqc::Dag& g, const Vertex& p, const Vertex& q,
               const std::map<Label, Label>& partner, Cand* c) {
  std::map<Label, int> qpos;
  for (int j = 0; j < (int)q.labels.size(); ++j) qpos[q.labels[j]] = j;
  std::vector<std::pair<int, int>> pairs;
  for (int i = 0; i < (int)p.labels.size(); ++i) {
    auto it = partner.find(p.labels[i]);
    if (it == partner.end()) continue;
    auto jt = qpos.find(it->second);
    if (jt != qpos.end()) pairs.push_back({i, jt->second});
  }
  if (pairs.empty()) return false;
  const Label pmin = *std::min_element(p.labels.begin(), p.labels.end());
  const Label qmin = *std::min_element(q.labels.begin(), q.labels.end());
  const int64_t pe = g.nodes[p.node].elems, qe = g.nodes[q.node].elems;
  const bool p_left = std::make_tuple(-pe, p.node, pmin) <= std::make_tuple(-qe, q.node, qmin);
  if (!p_left)
    for (auto& pr : pairs) std::swap(pr.first, pr.second);
  std::sort(pairs.begin(), pairs.end());
  const Vertex& L = p_left ? p : q;
  const Vertex& R = p_left ? q : p;
  std::vector<int> la, ra;
  for (auto& pr : pairs) {
    la.push_back(pr.first);
    ra.push_back(pr.second);
  }
  const lqc::Node& ln = g.nodes[L.node];
  const lqc::Node& rn = g.nodes[R.node];
  int64_t k = 1;
  for (int a : la) k *= ln.ext[a];
  const int64_t m = ln.elems / k, n = rn.elems / k;
  c->key = Key(L.node, R.node, la, ra);
  c->cost = (Wide)ln.lt * m * n * k;
  c->out_elems = m * n;
  c->left = &L;
  c->right = &R;
  return true;
}

std::vector<Cand> candidates(const lqc::Dag& g, const Graph& G) {
  std::vector<Cand> out;
  for (int x = 0; x < (int)G.verts.size(); ++x)
    for (int y = x + 1; y < (int)G.verts.size(); ++y) {
      Cand c;
      if (candidate(g, G.verts[x], G.verts[y], G.partner, &c)) {
        c.x = x;
        c.y = y;
        out.push_back(std::move(c));
      }
    }
  std::vector<Cand> ok;
  for (const Cand& c : out)
    if (c.out_elems <= G.cap) ok.push_back(c);
  return ok.empty() ? out : ok;
}

}  // namespace

extern "C" int lqc_dag_add_graphs(lqc_dag* h, int64_t n_graphs, const int64_t* vert_off,
                                  const int64_t* vert_nodes, const int64_t* edge_off,
                                  const int32_t* edges, int64_t* roots) {
  if (!h) return LQC_ERR_ARG;
  lqc::Dag& g = h->d;
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
      if (v0 < 0 || e0 < 0 || v1 <= v0 || e1 < e0 || (e1 > e0 && !edges)) {
        g.err = "graph " + std::to_string(gi) + ": empty or bad offsets";
        return LQC_ERR_ARG;
      }
      for (int64_t v = v0; v < v1; ++v) {
        const int64_t u = vert_nodes[v];
        if (u < 0 || u >= N || g.nodes[u].rank == 0) {
          g.err = "graph " + std::to_string(gi) + ": vertex is no tensor node";
          return LQC_ERR_ARG;
        }
        Vertex vx;
        vx.node = u;
        for (int a = 0; a < g.nodes[u].rank; ++a) vx.labels.push_back({(int32_t)(v - v0), a});
        G.cap = std::max(G.cap, g.nodes[u].elems);
        G.verts.push_back(std::move(vx));
      }
      for (int64_t e = e0; e < e1; ++e) {
        const int32_t* q = edges + 4 * e;
        const int nv = (int)(v1 - v0);
        if (q[0] < 0 || q[0] >= nv || q[2] < 0 || q[2] >= nv || q[0] == q[2] || q[1] < 0 ||
            q[1] >= g.nodes[vert_nodes[v0 + q[0]]].rank || q[3] < 0 ||
            q[3] >= g.nodes[vert_nodes[v0 + q[2]]].rank) {
          g.err = "graph " + std::to_string(gi) + ": edge out of range";
          return LQC_ERR_ARG;
        }
        const Label a{q[0], q[1]}, b{q[2], q[3]};
        if (G.partner.count(a) || G.partner.count(b)) {
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
    }
    // Key values are kept incrementally: a step changes the candidates of
    // only the graphs it contracts in, so only their keys are recounted.
    // The result equals recounting every graph at every step.
    struct KeyStat {
      int64_t count = 0;
      Wide cost = 0;
      std::set<int64_t> graphs;
    };
    std::map<Key, KeyStat> stat;
    std::set<std::pair<Wide, Key>> by_value;  // (-value, key): first = best
    std::vector<std::vector<Key>> held((size_t)n_graphs);
    auto enter = [&](int64_t gi) {
      const Graph& G = graphs[gi];
      held[gi].clear();
      if (G.verts.size() < 2) return;
      std::map<Key, Wide> seen;
      for (const Cand& c : candidates(g, G)) seen[c.key] = c.cost;
      for (auto& kv : seen) {
        KeyStat& ks = stat[kv.first];
        if (ks.count) by_value.erase({-(ks.count * ks.cost), kv.first});
        ks.count += 1;
        ks.cost = kv.second;
        ks.graphs.insert(gi);
        by_value.insert({-(ks.count * ks.cost), kv.first});
        held[gi].push_back(kv.first);
      }
    };
    auto leave = [&](int64_t gi) {
      for (const Key& k : held[gi]) {
        auto it = stat.find(k);
        KeyStat& ks = it->second;
        by_value.erase({-(ks.count * ks.cost), k});
        ks.count -= 1;
        ks.graphs.erase(gi);
        if (ks.count)
          by_value.insert({-(ks.count * ks.cost), k});
        else
          stat.erase(it);
      }
      held[gi].clear();
    };
    for (int64_t gi = 0; gi < n_graphs; ++gi) enter(gi);
    while (!by_value.empty()) {
      const Key bk = by_value.begin()->second;
      const std::vector<int64_t> hold(stat[bk].graphs.begin(), stat[bk].graphs.end());
      for (int64_t gi : hold) {
        Graph& G = graphs[gi];
        leave(gi);
        while (G.verts.size() >= 2) {
          std::vector<Cand> cs = candidates(g, G);
          const Cand* hit = nullptr;
          for (const Cand& c : cs)
            if (c.key == bk) {
              hit = &c;
              break;
            }
          if (!hit) break;
          const std::vector<int>& la = std::get<2>(hit->key);
          const std::vector<int>& ra = std::get<3>(hit->key);
          int64_t node = -1;
          const int rc = lqc_dag_add_contraction(h, std::get<0>(hit->key), std::get<1>(hit->key),
                                                 (int)la.size(), la.data(), ra.data(), &node);
          if (rc != LQC_OK) return rc;
          Vertex nv;
          nv.node = node;
          for (int i = 0; i < (int)hit->left->labels.size(); ++i)
            if (std::find(la.begin(), la.end(), i) == la.end()) nv.labels.push_back(hit->left->labels[i]);
          for (int j = 0; j < (int)hit->right->labels.size(); ++j)
            if (std::find(ra.begin(), ra.end(), j) == ra.end()) nv.labels.push_back(hit->right->labels[j]);
          const int x = hit->x, y = hit->y;
          G.verts[x] = std::move(nv);
          G.verts.erase(G.verts.begin() + y);
        }
        enter(gi);
      }
    }
    for (int64_t gi = 0; gi < n_graphs; ++gi) {
      if (graphs[gi].verts.size() != 1) {
        g.err = "graph " + std::to_string(gi) + " is not connected";
        return LQC_ERR_ARG;
      }
    }
    for (int64_t gi = 0; gi < n_graphs; ++gi) roots[gi] = graphs[gi].verts[0].node;
    return LQC_OK;
  } catch (const std::bad_alloc&) {
    g.err = "host allocation failed";
    return LQC_ERR_HOST_MEM;
  }
}
