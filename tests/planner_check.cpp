// Host-side check of the launch planners in csrc/kernels.h (plan_qrcp,
// plan_fronts, the grid-mode exchange layout): for seeded random batches it
// verifies that every matrix is planned exactly once and that every launch the
// plans imply stays within its shared memory, its co-resident CTA budget and
// its buffers (the index ranges the kernels touch).  Built and run by
// tests/test_planner.py with the host compiler; prints "OK ..." or the first
// violations.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "kernels.h"

namespace spaqr {
int qrcp_tuned_choice(int, int, int) { return 0; }  // no tuning table in this check
}  // namespace spaqr

using namespace spaqr;

namespace {

uint64_t g_state = 0x9E3779B97F4A7C15ull;
int draw(int lo, int hi) {  // uniform in [lo, hi], splitmix64
  uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return lo + (int)(z % (uint64_t)(hi - lo + 1));
}

int g_bad = 0;
void fail(const char* what, int a = 0, int b = 0) {
  if (g_bad < 20) std::printf("FAIL %s (%d, %d)\n", what, a, b);
  ++g_bad;
}

constexpr int kLimit = 232448 - 1024;  // GB300 opt-in shared memory less the static margin
constexpr int kGrid = 152;             // one CTA per SM

void check_qrcp(const std::vector<int>& ms, const std::vector<int>& ns, int elem, int grid_ctas, bool force,
                long long& ngroups, long long& ngrid) {
  std::vector<QrcpGroup> groups;
  std::vector<char> work;
  if (!plan_qrcp(ms, ns, elem, kLimit, groups, work, grid_ctas, force)) return;  // capacity error: reported
  std::vector<int> seen(ms.size(), 0);
  int big_fp64 = 0;
  for (const auto& g : groups) {
    ++ngroups;
    for (int i : g.idx) seen[(size_t)i]++;
    if (g.grid) {
      ++ngrid;
      if (g.ctas.size() != g.idx.size()) fail("grid ctas size");
      int tot = 0;
      for (size_t q = 0; q < g.idx.size(); ++q) {
        const int i = g.idx[q], G = g.ctas[q], m = ms[(size_t)i], n = ns[(size_t)i];
        tot += G;
        if (G < 1 || G > 256 || (g.slab && G < 17)) fail("grid CTA count", G, n);
        const int nl = (n + G - 1) / G;
        if (nl > g.nl_max || m > g.m_max) fail("grid footprint", nl, g.nl_max);
        if (n > 0 && (n - 1) / nl >= G) fail("pivot owner out of range", n, G);
        if (work[(size_t)i] != (g.slab ? 0 : 1)) fail("grid work flag", i, g.slab);
        if (g.slab && elem == 8 && !force) ++big_fp64;
      }
      if (tot > grid_ctas) fail("grid CTAs over the co-resident budget", tot, grid_ctas);
      // spare CTAs are spread until every member has at most 8 columns per CTA
      // (one per warp) or the co-resident budget is used up
      if (g.slab && tot < grid_ctas)
        for (size_t q = 0; q < g.idx.size(); ++q) {
          const int n = ns[(size_t)g.idx[q]], G = g.ctas[q];
          if ((n + G - 1) / G > 8) fail("grid CTAs not spread", n, G);
        }
      if (qrcp_grid_smem_bytes(g.m_max, g.nl_max, elem, g.slab) > kLimit) fail("grid shared memory");
      // exchange areas: back to back, each access range inside its own area
      std::vector<QrcpGridDesc> gd;
      unsigned char* base = nullptr;
      const int total = qrcp_grid_descs(g.ctas, g.m_max, elem, base, gd);
      if (total != tot) fail("grid total CTAs", total, tot);
      size_t off = 0;
      int cta0 = 0;
      for (size_t q = 0; q < gd.size(); ++q) {
        const int G = g.ctas[q];
        const size_t area = qrcp_grid_xchg_bytes(G, g.m_max, elem);
        const size_t t0 = (size_t)(reinterpret_cast<unsigned char*>(gd[q].tags) - base);
        const size_t s0 = (size_t)(reinterpret_cast<unsigned char*>(gd[q].slots) - base);
        const size_t v0 = (size_t)(static_cast<unsigned char*>(gd[q].vg) - base);
        if (gd[q].cta0 != cta0 || gd[q].ctas != G) fail("grid CTA ranges", gd[q].cta0, cta0);
        if (t0 != off || t0 % 256 || s0 % 256 || v0 % 256) fail("grid area alignment");
        if (t0 + 33 * sizeof(int) > s0) fail("counters overlap the slots");
        if (s0 + (size_t)2 * G * sizeof(QrcpSlot) > v0) fail("slots overlap the reflectors");
        if (v0 + (size_t)2 * G * ((g.m_max + 3) & ~1) * elem > off + area) fail("reflectors past the area");
        off += area;
        cta0 += G;
      }
    } else if (g.cs == 0) {
      for (int i : g.idx) {
        if (ms[(size_t)i] > 64) fail("warp QRCP with more than 64 rows", ms[(size_t)i]);
        if (qrcp_warp_bytes(ms[(size_t)i], ns[(size_t)i], elem) > g.nl_max) fail("warp region", i);
        if (work[(size_t)i]) fail("warp work flag");
      }
      if ((long long)g.nl_max * 8 > kLimit) fail("warp CTA shared memory", g.nl_max);
    } else {
      if (!(g.cs == 1 || g.cs == 2 || g.cs == 4 || g.cs == 8 || g.cs == 16)) fail("cluster size", g.cs);
      for (int i : g.idx) {
        const int nl = (ns[(size_t)i] + g.cs - 1) / g.cs;
        if (nl > g.nl_max || ms[(size_t)i] > g.m_max) fail("cluster footprint", nl, g.nl_max);
        if (work[(size_t)i] != (g.slab ? 0 : 1)) fail("cluster work flag", i, g.slab);
      }
      if (g.slab) {
        if (qrcp_smem_bytes(g.m_max, g.nl_max, elem, true) > kLimit) fail("cluster slab shared memory");
      } else {
        if (g.cs != 16) fail("delayed form not on 16 CTAs", g.cs);
        if (g.nb < 1 || qrcp_smem_bytes(g.m_max, g.nl_max, elem, false, g.nb) > kLimit) fail("delayed panel", g.nb);
      }
    }
  }
  if (big_fp64 > 4) fail("more than four FP64 matrices in CTA groups", big_fp64);
  for (size_t i = 0; i < seen.size(); ++i)
    if (seen[i] != 1) fail("matrix planned other than once", (int)i, seen[i]);
}

void check_fronts(const std::vector<int>& ms, const std::vector<int>& ns, const std::vector<int>& cs, int elem) {
  const auto groups = plan_fronts(ms, ns, cs, elem, kLimit);
  std::vector<int> seen(ms.size(), 0);
  for (const auto& g : groups)
    for (int i : g.idx) {
      seen[(size_t)i]++;
      const int m = ms[(size_t)i], n = ns[(size_t)i], c = cs[(size_t)i];
      if (g.kind == 0) {
        if (c > 128 || m > 256) fail("warp front shape", m, c);
        if ((long long)(m | 1) * n > g.param) fail("warp front region", m, n);
        if ((long long)g.param * elem * 8 > kLimit) fail("warp front shared memory", g.param);
      } else if (g.kind == 1) {
        if (front_smem_bytes(m, n, c, elem) > g.param || g.param > kLimit) fail("smem front", m, n);
      } else if (g.param < std::min(c, m)) {
        fail("blocked front steps", g.param, c);
      }
    }
  for (size_t i = 0; i < seen.size(); ++i) {
    const bool work = cs[i] > 0 && ms[i] > 0 && ns[i] > 0;
    if (seen[i] != (work ? 1 : 0)) fail("front planned other than once", (int)i, seen[i]);
  }
}

}  // namespace

int main() {
  long long ngroups = 0, ngrid = 0;
  for (int trial = 0; trial < 6000; ++trial) {
    const int cnt = draw(1, trial % 5 ? 40 : 4);
    const int mmax = trial % 2 ? 4000 : 12000, nmax = trial % 3 ? 6000 : 12000;
    std::vector<int> ms, ns;
    for (int i = 0; i < cnt; ++i) {
      ms.push_back(draw(0, mmax));
      ns.push_back(draw(0, nmax));
    }
    for (int elem : {4, 8})
      for (int grid : {0, kGrid})
        for (bool force : {false, true}) check_qrcp(ms, ns, elem, grid, force, ngroups, ngrid);
  }
  for (int trial = 0; trial < 3000; ++trial) {
    const int cnt = draw(1, 60);
    std::vector<int> ms, ns, cs;
    for (int i = 0; i < cnt; ++i) {
      const int m = draw(0, trial % 2 ? 300 : 5000), n = draw(0, trial % 3 ? 200 : 3000);
      ms.push_back(m);
      ns.push_back(n);
      cs.push_back(draw(0, n));
    }
    for (int elem : {4, 8}) check_fronts(ms, ns, cs, elem);
  }
  if (g_bad) {
    std::printf("%d violations\n", g_bad);
    return 1;
  }
  std::printf("OK qrcp groups %lld (CTA groups %lld)\n", ngroups, ngrid);
  return 0;
}
