// Algebraic ordering for matrices without a grid (Section 2.2): nested
// dissection of graph(A^T A), the interfaces of the modified nested dissection
// and the merge hierarchy (Section 2.6), and a maximum-weight row-to-column
// matching.  Host only.
//
// Readings (the paper relies on third-party partitioners and matchings here):
//  * graph(A^T A): columns i != j adjacent when a row has entries in both;
//  * nested dissection to depth L, heap numbering: a node's vertex set V is cut
//    by a level structure.  r0 = min(V); a breadth-first search of the
//    subgraph induced by V from r0; u = the vertex of its last level with the
//    smallest induced degree (then smallest id); a second search from u gives
//    levels L_0..L_h of u's component, the rest of V comes after.  The
//    separator is the first L_j (j >= 1) whose prefix holds at least half of
//    V (none if h = 0: the left child takes V); separator vertices without a
//    neighbour beyond L_j move to the left child; the right child takes the
//    levels beyond j and the other components.  Level-L nodes keep their set;
//  * interfaces: at stage k a label is (t, -1) for a vertex in the subtree of
//    a level-k node t (or deeper) and (t, i) for the i-th interface of a
//    separator t of level < k; a separator vertex's key is the set of labels
//    of its neighbours in proper descendants of its node; a separator's
//    interfaces are its vertices with equal keys, ranked by key, computed
//    deepest node first.  Every stage-k interface lies in one stage-(k-1)
//    interface (the merge).  On grids with the geometric tree this gives the
//    geometric interfaces of symbolic.cpp;
//  * matching: the row-to-column matching that maximises sum log|a_ij| (a
//    maximum-product matching), by successive shortest augmenting paths with
//    Dijkstra and dual potentials on the costs log(max_i |a_ij|) - log|a_ij|.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <limits>
#include <map>
#include <queue>
#include <stdexcept>
#include <utility>
#include <vector>

#include "symbolic.h"

namespace spaqr {
namespace {

int lvl_of(int t) {
  int l = 1;
  for (int x = t + 1; x > 1; x >>= 1) ++l;
  return l;
}

int anc_at(int t, int level) {
  while (lvl_of(t) > level) t = (t - 1) / 2;
  return t;
}

bool proper_desc(int t, int s) {
  while (t > s) {
    t = (t - 1) / 2;
    if (t == s) return true;
  }
  return false;
}

struct Graph {
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj;  // ascending per vertex
};

Graph column_graph(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colidx) {
  // rows of each column
  std::vector<int64_t> cptr((size_t)n + 1, 0);
  for (int64_t e = 0; e < rowptr[m]; ++e) cptr[(size_t)colidx[e] + 1]++;
  for (int64_t j = 0; j < n; ++j) cptr[(size_t)j + 1] += cptr[(size_t)j];
  std::vector<int64_t> crow((size_t)rowptr[m]);
  {
    std::vector<int64_t> pos(cptr.begin(), cptr.end() - 1);
    for (int64_t r = 0; r < m; ++r)
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) crow[(size_t)pos[(size_t)colidx[e]]++] = r;
  }
  Graph g;
  g.ptr.assign((size_t)n + 1, 0);
  std::vector<int64_t> mark((size_t)n, -1);
  std::vector<int32_t> tmp;
  for (int64_t j = 0; j < n; ++j) {
    tmp.clear();
    for (int64_t q = cptr[(size_t)j]; q < cptr[(size_t)j + 1]; ++q) {
      const int64_t r = crow[(size_t)q];
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        const int32_t i = colidx[e];
        if (i != j && mark[(size_t)i] != j) {
          mark[(size_t)i] = j;
          tmp.push_back(i);
        }
      }
    }
    std::sort(tmp.begin(), tmp.end());
    g.adj.insert(g.adj.end(), tmp.begin(), tmp.end());
    g.ptr[(size_t)j + 1] = (int64_t)g.adj.size();
  }
  return g;
}

// breadth-first levels of the subgraph induced by the vertices with in[v] == stamp
void bfs_levels(const Graph& g, const std::vector<int64_t>& in, int64_t stamp, int32_t root,
                std::vector<int64_t>& seen, int64_t seen_stamp, std::vector<std::vector<int32_t>>& lev) {
  lev.clear();
  lev.push_back({root});
  seen[(size_t)root] = seen_stamp;
  for (;;) {
    std::vector<int32_t> nxt;
    for (int32_t v : lev.back())
      for (int64_t q = g.ptr[(size_t)v]; q < g.ptr[(size_t)v + 1]; ++q) {
        const int32_t w = g.adj[(size_t)q];
        if (in[(size_t)w] == stamp && seen[(size_t)w] != seen_stamp) {
          seen[(size_t)w] = seen_stamp;
          nxt.push_back(w);
        }
      }
    if (nxt.empty()) return;
    std::sort(nxt.begin(), nxt.end());
    lev.push_back(std::move(nxt));
  }
}

}  // namespace

Analysis* build_analysis_matrix(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colidx, int depth) {
  if (n <= 0 || m < 0) throw std::invalid_argument("matrix sizes must be positive");
  if (depth < 1 || depth > 30) throw std::invalid_argument("depth must be in [1, 30]");
  const auto t0 = std::chrono::steady_clock::now();
  const Graph g = column_graph(m, n, rowptr, colidx);
  Analysis* an = new Analysis();
  an->nx = (int)n;
  an->ny = an->nz = 1;
  an->depth = depth;
  an->n = n;
  const int L = depth;
  const int nnodes = (1 << L) - 1;
  an->nodes.assign((size_t)nnodes, NdNode());
  // ---- nested dissection
  std::vector<std::vector<int32_t>> work((size_t)nnodes);
  work[0].resize((size_t)n);
  for (int64_t v = 0; v < n; ++v) work[0][(size_t)v] = (int32_t)v;
  std::vector<int64_t> in((size_t)n, -1), seen((size_t)n, -1), beyond((size_t)n, -1);
  int64_t stamp = 0;
  std::vector<std::vector<int32_t>> lev;
  for (int t = 0; t < nnodes; ++t) {
    NdNode& nd = an->nodes[(size_t)t];
    nd.id = t;
    nd.level = lvl_of(t);
    std::vector<int32_t> V;
    V.swap(work[(size_t)t]);
    if (nd.level == L || V.empty()) {
      nd.verts = V;
      nd.empty = V.empty();
      continue;
    }
    const int64_t in_stamp = ++stamp;
    for (int32_t v : V) in[(size_t)v] = in_stamp;
    const int64_t first_seen = ++stamp;
    bfs_levels(g, in, in_stamp, V.front(), seen, first_seen, lev);
    auto deg = [&](int32_t v) {
      int d = 0;
      for (int64_t q = g.ptr[(size_t)v]; q < g.ptr[(size_t)v + 1]; ++q) d += in[(size_t)g.adj[(size_t)q]] == in_stamp;
      return d;
    };
    int32_t u = lev.back().front();
    int du = deg(u);
    for (int32_t v : lev.back()) {
      const int dv = deg(v);
      if (dv < du || (dv == du && v < u)) {
        u = v;
        du = dv;
      }
    }
    const int64_t sst = ++stamp;
    bfs_levels(g, in, in_stamp, u, seen, sst, lev);
    std::vector<int32_t> left, right, sep;
    if (lev.size() == 1) {
      left = V;
    } else {
      size_t j = lev.size() - 1;
      int64_t cum = 0;
      for (size_t q = 0; q < lev.size(); ++q) {
        cum += (int64_t)lev[q].size();
        if (q >= 1 && 2 * cum >= (int64_t)V.size()) {
          j = q;
          break;
        }
      }
      const int64_t bst = ++stamp;
      for (size_t q = j + 1; q < lev.size(); ++q)
        for (int32_t v : lev[q]) beyond[(size_t)v] = bst;
      for (size_t q = 0; q < j; ++q) left.insert(left.end(), lev[q].begin(), lev[q].end());
      for (int32_t v : lev[j]) {
        bool far = false;
        for (int64_t q = g.ptr[(size_t)v]; q < g.ptr[(size_t)v + 1] && !far; ++q)
          far = beyond[(size_t)g.adj[(size_t)q]] == bst;
        (far ? sep : left).push_back(v);
      }
      for (int32_t v : V)
        if (seen[(size_t)v] != sst || beyond[(size_t)v] == bst) right.push_back(v);
    }
    std::sort(left.begin(), left.end());
    std::sort(right.begin(), right.end());
    std::sort(sep.begin(), sep.end());
    nd.verts = sep;
    nd.empty = sep.empty();
    if (2 * t + 2 < nnodes) {
      work[(size_t)(2 * t + 1)] = std::move(left);
      work[(size_t)(2 * t + 2)] = std::move(right);
    }
  }
  std::vector<int32_t> node_of((size_t)n, -1);
  for (const NdNode& nd : an->nodes)
    for (int32_t v : nd.verts) node_of[(size_t)v] = nd.id;
  for (int64_t v = 0; v < n; ++v)
    if (node_of[(size_t)v] < 0) throw std::logic_error("nested dissection lost a vertex");
  // ---- interfaces of every stage
  using Label = std::pair<int, int>;
  using Key = std::vector<Label>;
  std::vector<int> order((size_t)nnodes);
  for (int t = 0; t < nnodes; ++t) order[(size_t)t] = t;
  std::sort(order.begin(), order.end(), [](int a, int b) {
    const int la = lvl_of(a), lb = lvl_of(b);
    return la != lb ? la > lb : a < b;
  });
  an->stages.assign((size_t)L + 1, StageClusters());
  std::vector<Label> label((size_t)n);
  std::vector<Key> key((size_t)n);
  std::vector<int32_t> cluster_prev;  // cluster of every vertex at the previous (finer) stage
  for (int k = L; k >= 1; --k) {
    for (int t : order) {
      const NdNode& nd = an->nodes[(size_t)t];
      if (nd.verts.empty()) continue;
      if (nd.level >= k) {
        const int a = anc_at(t, k);
        for (int32_t v : nd.verts) label[(size_t)v] = Label(a, -1);
        continue;
      }
      for (int32_t v : nd.verts) {
        Key& kv = key[(size_t)v];
        kv.clear();
        for (int64_t q = g.ptr[(size_t)v]; q < g.ptr[(size_t)v + 1]; ++q) {
          const int32_t w = g.adj[(size_t)q];
          if (proper_desc(node_of[(size_t)w], t)) kv.push_back(label[(size_t)w]);
        }
        std::sort(kv.begin(), kv.end());
        kv.erase(std::unique(kv.begin(), kv.end()), kv.end());
      }
      std::map<Key, int> rank;
      for (int32_t v : nd.verts) rank.emplace(key[(size_t)v], 0);
      int r = 0;
      for (auto& kv : rank) kv.second = r++;
      for (int32_t v : nd.verts) label[(size_t)v] = Label(t, rank[key[(size_t)v]]);
    }
    StageClusters& st = an->stages[(size_t)k];
    st.stage = k;
    st.vptr.assign(1, 0);
    std::vector<int32_t> cluster_of((size_t)n, -1);
    for (const NdNode& nd : an->nodes) {
      if (nd.verts.empty() || nd.level > k) continue;
      std::map<Key, std::vector<int32_t>> groups;
      if (nd.level == k)
        groups[Key()] = nd.verts;
      else
        for (int32_t v : nd.verts) groups[key[(size_t)v]].push_back(v);
      for (auto& kv : groups) {
        const int c = (int)st.node.size();
        st.node.push_back(nd.id);
        st.level.push_back(nd.level);
        for (int32_t v : kv.second) cluster_of[(size_t)v] = c;
        st.verts.insert(st.verts.end(), kv.second.begin(), kv.second.end());  // ascending: nd.verts is
        st.vptr.push_back((int64_t)st.verts.size());
      }
    }
    if (k < L) {  // parents of the finer stage's clusters
      StageClusters& fine = an->stages[(size_t)k + 1];
      fine.parent.assign(fine.node.size(), -1);
      for (size_t c = 0; c < fine.node.size(); ++c) {
        if (fine.level[c] >= k + 1) continue;  // eliminated at stage k + 1
        const int32_t v0 = fine.verts[(size_t)fine.vptr[c]];
        const int32_t p = cluster_of[(size_t)v0];
        for (int64_t q = fine.vptr[c]; q < fine.vptr[c + 1]; ++q)
          if (cluster_of[(size_t)fine.verts[(size_t)q]] != p) throw std::logic_error("interfaces do not nest");
        fine.parent[c] = p;
      }
    }
    cluster_prev.swap(cluster_of);
  }
  an->stages[1].parent.assign(an->stages[1].node.size(), -1);
  an->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return an;
}

// Maximum-weight column-perfect matching: match[j] = row of column j.  Returns
// false when A has no such matching (structurally rank deficient).
bool max_weight_matching(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* vals,
                         int32_t* match) {
  // columns in CSC with costs c = log(max_i |a_ij|) - log|a_ij| >= 0 (entries that are zero are not edges)
  std::vector<int64_t> cptr((size_t)n + 1, 0);
  for (int64_t e = 0; e < rowptr[m]; ++e)
    if (vals[e] != 0.0) cptr[(size_t)colidx[e] + 1]++;
  for (int64_t j = 0; j < n; ++j) cptr[(size_t)j + 1] += cptr[(size_t)j];
  std::vector<int32_t> crow((size_t)cptr[(size_t)n]);
  std::vector<double> cost((size_t)cptr[(size_t)n]);
  {
    std::vector<int64_t> pos(cptr.begin(), cptr.end() - 1);
    for (int64_t r = 0; r < m; ++r)
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e)
        if (vals[e] != 0.0) {
          const int64_t q = pos[(size_t)colidx[e]]++;
          crow[(size_t)q] = (int32_t)r;
          cost[(size_t)q] = std::log(std::fabs(vals[e]));
        }
    for (int64_t j = 0; j < n; ++j) {
      double mx = -std::numeric_limits<double>::infinity();
      for (int64_t q = cptr[(size_t)j]; q < cptr[(size_t)j + 1]; ++q) mx = std::max(mx, cost[(size_t)q]);
      for (int64_t q = cptr[(size_t)j]; q < cptr[(size_t)j + 1]; ++q) cost[(size_t)q] = mx - cost[(size_t)q];
    }
  }
  const double inf = std::numeric_limits<double>::infinity();
  std::vector<double> u((size_t)n, 0.0), v((size_t)m, 0.0);  // duals: reduced cost c - u_j - v_r >= 0
  std::vector<int32_t> col_of((size_t)m, -1), row_of((size_t)n, -1);
  for (int64_t j = 0; j < n; ++j) {  // u_j = min cost of column j
    double mn = inf;
    for (int64_t q = cptr[(size_t)j]; q < cptr[(size_t)j + 1]; ++q) mn = std::min(mn, cost[(size_t)q]);
    u[(size_t)j] = mn == inf ? 0.0 : mn;
  }
  std::vector<double> dist((size_t)m, inf);
  std::vector<int32_t> pred((size_t)m, -1);  // column from which a row was reached
  std::vector<char> done((size_t)m, 0);
  std::vector<int32_t> touched;
  using QE = std::pair<double, int32_t>;
  for (int64_t j0 = 0; j0 < n; ++j0) {
    // Dijkstra over rows: from column c to row r at reduced cost; a matched row
    // continues from its column at distance dist[r]
    std::priority_queue<QE, std::vector<QE>, std::greater<QE>> pq;
    touched.clear();
    auto relax_from = [&](int32_t c, double base) {
      for (int64_t q = cptr[(size_t)c]; q < cptr[(size_t)c + 1]; ++q) {
        const int32_t r = crow[(size_t)q];
        if (done[(size_t)r]) continue;
        const double d = base + std::max(0.0, cost[(size_t)q] - u[(size_t)c] - v[(size_t)r]);
        if (d < dist[(size_t)r]) {
          if (dist[(size_t)r] == inf) touched.push_back(r);
          dist[(size_t)r] = d;
          pred[(size_t)r] = c;
          pq.emplace(d, r);
        }
      }
    };
    relax_from((int32_t)j0, 0.0);
    int32_t free_row = -1;
    double dfree = inf;
    std::vector<int32_t> settled;
    while (!pq.empty()) {
      const auto [d, r] = pq.top();
      pq.pop();
      if (done[(size_t)r] || d > dist[(size_t)r]) continue;
      done[(size_t)r] = 1;
      settled.push_back(r);
      if (col_of[(size_t)r] < 0) {
        free_row = r;
        dfree = d;
        break;
      }
      relax_from(col_of[(size_t)r], d);
    }
    if (free_row < 0) {
      for (int32_t r : touched) {
        dist[(size_t)r] = inf;
        done[(size_t)r] = 0;
      }
      return false;
    }
    // dual update (keeps reduced costs non-negative and tight on the matching)
    for (int32_t r : settled) {
      if (dist[(size_t)r] < dfree) {
        const int32_t c = col_of[(size_t)r];
        v[(size_t)r] -= dfree - dist[(size_t)r];
        if (c >= 0) u[(size_t)c] += dfree - dist[(size_t)r];
      }
    }
    u[(size_t)j0] += dfree;
    // augment along the predecessor chain
    int32_t r = free_row;
    while (r >= 0) {
      const int32_t c = pred[(size_t)r];
      const int32_t prev = row_of[(size_t)c];
      row_of[(size_t)c] = r;
      col_of[(size_t)r] = c;
      r = c == (int32_t)j0 ? -1 : prev;
    }
    for (int32_t t : touched) {
      dist[(size_t)t] = inf;
      done[(size_t)t] = 0;
      pred[(size_t)t] = -1;
    }
  }
  for (int64_t j = 0; j < n; ++j) match[j] = row_of[(size_t)j];
  return true;
}

}  // namespace spaqr
