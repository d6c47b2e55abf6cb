// Host symbolic analysis (Section 2.2 nested dissection + modified nested
// dissection interfaces; Section 2.6 cluster hierarchy).  See symbolic.h for
// the readings taken for structured grids.
#include "symbolic.h"

#include <algorithm>
#include <chrono>
#include <map>
#include <stdexcept>

namespace spaqr {

namespace {

using Key = std::vector<std::pair<int, int>>;  // sorted (D node id, sign)

int level_of(int id) {
  int l = 0;
  unsigned v = (unsigned)id + 1u;
  while (v) {
    ++l;
    v >>= 1;
  }
  return l;
}

void build_tree(Analysis& an) {
  const int L = an.depth;
  const int64_t nnodes = (int64_t(1) << L) - 1;
  an.nodes.assign((size_t)nnodes, NdNode());
  const int nx = an.nx, ny = an.ny;
  auto vid = [&](int x, int y, int z) { return (int32_t)(x + (int64_t)nx * (y + (int64_t)ny * z)); };
  NdNode& root = an.nodes[0];
  root.id = 0;
  root.level = 1;
  root.hi[0] = an.nx;
  root.hi[1] = an.ny;
  root.hi[2] = an.nz;
  for (int64_t i = 0; i < nnodes; ++i) {
    NdNode& nd = an.nodes[(size_t)i];
    nd.id = (int)i;
    nd.level = level_of((int)i);
    nd.empty = false;
    for (int a = 0; a < 3; ++a)
      if (nd.hi[a] <= nd.lo[a]) nd.empty = true;
    if (nd.level == L) {
      if (!nd.empty) {
        for (int z = nd.lo[2]; z < nd.hi[2]; ++z)
          for (int y = nd.lo[1]; y < nd.hi[1]; ++y)
            for (int x = nd.lo[0]; x < nd.hi[0]; ++x) nd.verts.push_back(vid(x, y, z));
        std::sort(nd.verts.begin(), nd.verts.end());
      }
      continue;
    }
    NdNode& lc = an.nodes[(size_t)(2 * i + 1)];
    NdNode& rc = an.nodes[(size_t)(2 * i + 2)];
    if (nd.empty) {
      nd.axis = 0;
      nd.mid = nd.lo[0];
      for (int a = 0; a < 3; ++a) {
        lc.lo[a] = lc.hi[a] = nd.lo[a];
        rc.lo[a] = rc.hi[a] = nd.lo[a];
      }
      continue;
    }
    int ax = 0;
    for (int a = 1; a < 3; ++a)
      if (nd.hi[a] - nd.lo[a] > nd.hi[ax] - nd.lo[ax]) ax = a;
    const int mid = (nd.lo[ax] + nd.hi[ax]) / 2;
    nd.axis = ax;
    nd.mid = mid;
    int slo[3], shi[3];
    for (int a = 0; a < 3; ++a) {
      slo[a] = nd.lo[a];
      shi[a] = nd.hi[a];
    }
    slo[ax] = mid;
    shi[ax] = mid + 1;
    for (int z = slo[2]; z < shi[2]; ++z)
      for (int y = slo[1]; y < shi[1]; ++y)
        for (int x = slo[0]; x < shi[0]; ++x) nd.verts.push_back(vid(x, y, z));
    std::sort(nd.verts.begin(), nd.verts.end());
    for (int a = 0; a < 3; ++a) {
      lc.lo[a] = nd.lo[a];
      lc.hi[a] = nd.hi[a];
      rc.lo[a] = nd.lo[a];
      rc.hi[a] = nd.hi[a];
    }
    lc.hi[ax] = mid;
    rc.lo[ax] = mid + 1;
  }
}

// Interface keys of every vertex of separator S (all descendant levels).
void separator_keys(const Analysis& an, const NdNode& S, std::vector<Key>& keys) {
  const int nv = (int)S.verts.size();
  keys.assign((size_t)nv, Key());
  std::vector<int> coord((size_t)nv * 3);
  for (int t = 0; t < nv; ++t) {
    int64_t v = S.verts[(size_t)t];
    coord[3 * t + 0] = (int)(v % an.nx);
    coord[3 * t + 1] = (int)((v / an.nx) % an.ny);
    coord[3 * t + 2] = (int)(v / ((int64_t)an.nx * an.ny));
  }
  const int64_t nnodes = (int64_t)an.nodes.size();
  std::vector<int> stack;
  stack.push_back(2 * S.id + 1);
  stack.push_back(2 * S.id + 2);
  std::vector<int> inside;
  while (!stack.empty()) {
    const int d = stack.back();
    stack.pop_back();
    if (d >= nnodes) continue;
    const NdNode& D = an.nodes[(size_t)d];
    if (D.empty) continue;
    inside.clear();
    for (int t = 0; t < nv; ++t) {
      bool in = true;
      for (int b = 0; b < 3 && in; ++b) {
        const int c = coord[3 * t + b];
        in = (c >= D.lo[b] - 1) && (c <= D.hi[b]);
      }
      if (in) inside.push_back(t);
    }
    if (inside.empty()) continue;  // no descendant of D can touch S either
    if (D.level < an.depth && D.axis != S.axis) {
      for (int t : inside) {
        const int diff = coord[3 * t + D.axis] - D.mid;
        keys[(size_t)t].emplace_back(d, (diff > 0) - (diff < 0));
      }
    }
    stack.push_back(2 * d + 1);
    stack.push_back(2 * d + 2);
  }
  for (auto& k : keys) std::sort(k.begin(), k.end());
}

}  // namespace

Analysis* build_analysis(int nx, int ny, int nz, int depth) {
  if (nx <= 0 || ny <= 0 || nz <= 0) throw std::invalid_argument("grid extents must be positive");
  if (depth < 1 || depth > 30) throw std::invalid_argument("depth must be in [1, 30]");
  auto t0 = std::chrono::steady_clock::now();
  Analysis* an = new Analysis();
  an->nx = nx;
  an->ny = ny;
  an->nz = nz;
  an->depth = depth;
  an->n = (int64_t)nx * ny * nz;
  build_tree(*an);
  const int L = depth;
  an->stages.assign((size_t)L + 1, StageClusters());

  // ---- stage L: leaves whole, separators split by their full keys
  std::vector<Key> ckeys;  // key of each stage-L cluster
  {
    StageClusters& st = an->stages[(size_t)L];
    st.stage = L;
    st.vptr.push_back(0);
    std::vector<Key> vkeys;
    std::vector<int> order;
    for (const NdNode& nd : an->nodes) {
      if (nd.verts.empty()) continue;
      if (nd.level == L) {
        st.node.push_back(nd.id);
        st.level.push_back(nd.level);
        st.verts.insert(st.verts.end(), nd.verts.begin(), nd.verts.end());
        st.vptr.push_back((int64_t)st.verts.size());
        ckeys.emplace_back();
        continue;
      }
      separator_keys(*an, nd, vkeys);
      order.resize(nd.verts.size());
      for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return vkeys[(size_t)a] < vkeys[(size_t)b]; });
      size_t t = 0;
      while (t < order.size()) {
        size_t e = t;
        while (e < order.size() && vkeys[(size_t)order[e]] == vkeys[(size_t)order[t]]) ++e;
        std::vector<int32_t> vs;
        for (size_t u = t; u < e; ++u) vs.push_back(nd.verts[(size_t)order[u]]);
        std::sort(vs.begin(), vs.end());
        st.node.push_back(nd.id);
        st.level.push_back(nd.level);
        st.verts.insert(st.verts.end(), vs.begin(), vs.end());
        st.vptr.push_back((int64_t)st.verts.size());
        ckeys.push_back(vkeys[(size_t)order[t]]);
        t = e;
      }
    }
  }

  // ---- stages L-1 .. 1 by merging: drop the pairs of level k-1
  for (int k = L; k >= 2; --k) {
    StageClusters& cur = an->stages[(size_t)k];
    StageClusters& nxt = an->stages[(size_t)k - 1];
    nxt.stage = k - 1;
    const int nc = (int)cur.node.size();
    cur.parent.assign((size_t)nc, -1);
    std::map<std::pair<int, Key>, std::vector<int>> groups;
    for (int c = 0; c < nc; ++c) {
      if (cur.level[(size_t)c] >= k) continue;  // eliminated at stage k
      Key pk;
      for (const auto& pr : ckeys[(size_t)c])
        if (an->nodes[(size_t)pr.first].level < k - 1) pk.push_back(pr);
      groups[{cur.node[(size_t)c], pk}].push_back(c);
    }
    std::vector<Key> nkeys;
    nxt.vptr.push_back(0);
    int pid = 0;
    for (auto& kv : groups) {
      std::vector<int32_t> vs;
      for (int c : kv.second) {
        cur.parent[(size_t)c] = pid;
        vs.insert(vs.end(), cur.verts.begin() + cur.vptr[(size_t)c], cur.verts.begin() + cur.vptr[(size_t)c + 1]);
      }
      std::sort(vs.begin(), vs.end());
      nxt.node.push_back(kv.first.first);
      nxt.level.push_back(an->nodes[(size_t)kv.first.first].level);
      nxt.verts.insert(nxt.verts.end(), vs.begin(), vs.end());
      nxt.vptr.push_back((int64_t)nxt.verts.size());
      nkeys.push_back(kv.first.second);
      ++pid;
    }
    ckeys.swap(nkeys);
  }
  an->stages[1].parent.assign(an->stages[1].node.size(), -1);
  an->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return an;
}

}  // namespace spaqr
