// Launchers for the device kernels of the factorization and the solve.
// All matrices are column-major.  Every launcher enqueues on `st` and returns
// the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <vector>

namespace spaqr {

// One 2D block copy dst[r + c*dld] = src[row(r) + c*sld], row(r) = r or
// rowidx[r]; src == nullptr writes zeros.  Optionally transposed:
// dst[c + r*dld] = src[row(r) + c*sld].
// steps per panel of the delayed-update QRCP (slabs in global memory); wide
// matrices whose coefficients would not fit use shallower panels (8, 4, 2, 1)
constexpr int kQrcpNB = 16;

template <typename T>
struct CopyDesc {
  const T* src;
  T* dst;
  const int32_t* rowidx;
  int sld, dld;
  int rows, cols;
  int transpose;
  int pad;
};

// Front for the Householder QR: factorize the first c columns of the m x n
// matrix at ptr (ld), apply the reflectors to the rest, zero below the diagonal
// of the first c columns and flip rows < c so that diag(R) >= 0.
template <typename T>
struct FrontDesc {
  T* ptr;
  int m, n, c, ld;
};

// Column-pivoted QR of the m x n matrix src (ld), stopped at the rank
// (|R_ii| >= eps |R_11|, R_ii != 0); src is only read.  The factorization runs
// in shared memory or, for large matrices, in `work` (m x n, ld m).  Writes
// rank[0]; if out != nullptr and k < m, the first k rows of Q^T A in the
// original column order are written to rows 0..k-1 of out (ldo); if V != nullptr
// the reflectors go to V (m x k, ld m, unit diagonal) and tau.  flags:
// kQrcpSignFix negates every written row i whose R_ii is negative (the rows
// then no longer depend on the reflector signs); kQrcpAlwaysOut writes out also
// when k == m (src is the triangular factor of a taller matrix).
constexpr int kQrcpSignFix = 1;
constexpr int kQrcpAlwaysOut = 2;
template <typename T>
struct QrcpDesc {
  const T* src;
  T* work;
  T* out;
  T* V;
  T* tau;
  int* rank;
  int m, n, ld, ldo;
  int flags = 0;
};

// Reflector application on a block X: mode 0: each row x^T <- x^T H_1..H_k
// (X is rows x len at ptr, ld) then columns k..len-1 zeroed; mode 1: each
// column y <- H_k..H_1 y (X is len x cols), rows k..len-1 zeroed.
template <typename T>
struct ReflDesc {
  T* ptr;
  const T* V;   // len x (>= k), ld = len
  const T* tau;
  const int* k; // device rank
  int ld, len, nvec, mode;
};

// X <- X R^{-1} for X (rows x c at ptr, ld) and upper-triangular R (c x c, ld rld).
template <typename T>
struct TrsmDesc {
  T* ptr;
  const T* R;
  int ld, rows, c, rld;
};

// Extra-row destination: for rows [r0, r1) of the front F (ld), score each of
// ncl column clusters (columns [coff[t], coff[t+1])) by the sum of squares and
// write the argmax cluster index (ties: larger lvl, then smaller id) to
// out[r - r0]; clusters with lvl < 0 are not candidates.
template <typename T>
struct ArgmaxDesc {
  const T* F;
  int ld, r0, r1, ncl;
  const int* coff;  // ncl + 1
  const int* lvl;   // ncl
  const int* cid;   // ncl
  int* out;
};

// chunk_start: count + 1 prefix sums of copy_chunks(rows * cols) over the descriptors
template <typename T>
cudaError_t launch_copy(const CopyDesc<T>* d_desc, const int* chunk_start, int count, int total_chunks, cudaStream_t st);
inline int copy_chunks(long long elems) { return (int)((elems + 2047) / 2048); }
// CTAs of one copy descriptor: 2048-entry chunks, or for a transposed copy
// 32 x 64 tiles (staged in shared memory so that reads and writes coalesce)
inline int copy_ctas(int rows, int cols, int transpose) {
  if (transpose) return ((rows + 31) / 32) * ((cols + 63) / 64);
  return copy_chunks((long long)rows * cols);
}
// Small fronts: whole front in shared memory (smem_bytes >= m*n*sizeof(T) for every front).
template <typename T> cudaError_t launch_front_qr_smem(const FrontDesc<T>* d, int count, int smem_bytes, cudaStream_t st);
// Tiny fronts (c <= 128, (m|1) * n * sizeof(T) * 8 <= shared memory): one warp per
// front, per_warp_elems >= (m|1) * n for every front of the launch.
template <typename T> cudaError_t launch_front_qr_warp(const FrontDesc<T>* d, int count, int per_warp_elems, cudaStream_t st);

// Large fronts, blocked: panel j0..j0+nb of each front then the trailing update.
template <typename T>
cudaError_t launch_front_panel(const FrontDesc<T>* d, int count, int j0, int nb, T* Tbuf, cudaStream_t st,
                               int rows_max);
template <typename T>
cudaError_t launch_front_trailing(const FrontDesc<T>* d, int count, int j0, int nb, const T* Tbuf, int max_tiles,
                                  cudaStream_t st);
template <typename T>
cudaError_t launch_front_finish(const FrontDesc<T>* d, int count, int max_c, int max_n, unsigned* masks, cudaStream_t st);
// One cluster of cs CTAs per matrix (cs in 1, 2, 4, 8, 16); every matrix of a
// launch shares cs, nl_max >= ceil(n / cs) and m_max >= m.  smem_slab: the
// column slabs live in shared memory, else in each descriptor's work buffer
// (m x n, ld m).
template <typename T>
cudaError_t launch_qrcp(const QrcpDesc<T>* d, int count, double eps, int cs, int nl_max, int m_max, bool smem_slab,
                        cudaStream_t st, int nb = kQrcpNB);
// dynamic shared memory of one QRCP CTA (nl columns of m rows): with the slab
// in shared memory (slab: two reflector buffers, taus, the slab), or the
// delayed-update form (reflector, taus, nb coefficients per column)
// Slab layout of the shared-memory QRCP: columns of ldx = m rounded up to four
// rows (16-byte vector rows for FP32 and FP64), reflector buffers of vstride
// elements (row-aligned, a multiple of four).
#ifdef __CUDACC__
#define SPAQR_HD __host__ __device__
#else
#define SPAQR_HD
#endif
SPAQR_HD inline int qrcp_ldx(int m) { return (m + 3) & ~3; }
SPAQR_HD inline int qrcp_vstride(int m) { return qrcp_ldx(m) + 4; }
inline int qrcp_smem_bytes(int m, int nl, int elem, bool slab, int nb = kQrcpNB) {
  long long b = ((long long)nl * 28 + 15) / 16 * 16;  // nu, nuref, step_of, act, pos
  const long long vs = (long long)qrcp_vstride(m) * elem;
  if (slab)
    b += 3 * vs + (long long)qrcp_ldx(m) * nl * elem;
  else
    b += 2 * vs + (long long)nl * nb * elem;
  return (int)(b + 64);
}
// dynamic shared memory of one grid-mode QRCP CTA: the slab layout, without
// the slab itself when the columns stay in the work copy
inline int qrcp_grid_smem_bytes(int m, int nl, int elem, bool slab) {
  return qrcp_smem_bytes(m, nl, elem, true) - (slab ? 0 : qrcp_ldx(m) * nl * elem);
}
// deepest panel (16, 8, 4, 2, 1) of the delayed-update QRCP that fits, 0 if none
inline int qrcp_panel_depth(int m, int nl, int elem, int limit) {
  for (int nb = kQrcpNB; nb >= 1; nb /= 2)
    if (qrcp_smem_bytes(m, nl, elem, false, nb) <= limit) return nb;
  return 0;
}
// Launch groups for a batch of QRCPs of shapes (m_i, n_i): each matrix takes
// the smallest cluster size whose per-CTA column slab fits in shared memory,
// else 16 CTAs over a global work copy (needs_work); members of a group share
// (cs, slab) and a footprint (m_max, nl_max) that fits `limit` bytes.
struct QrcpGroup {
  int cs = 1;  // 0: one warp per matrix (nl_max then holds the per-warp bytes)
  bool slab = true;
  int nb = kQrcpNB;  // panel depth of the delayed-update form (slab == false)
  int m_max = 0, nl_max = 0;
  std::vector<int> idx;
  bool grid = false;      // CTA groups exchanging through global memory (qrcp_grid_kernel)
  std::vector<int> ctas;  // grid: CTAs of each member (parallel to idx); slab: shared-memory slabs
};
// bytes of one warp's region in the warp-per-matrix QRCP (cs == 0 groups)
inline int qrcp_warp_bytes(int m, int n, int elem) {
  const int kmax = m < n ? m : n;
  long long b = ((long long)n * 20 + 15) / 16 * 16 + (long long)((kmax + 3) & ~1) * elem +
                (long long)(m | 1) * n * elem;
  return (int)((b + 15) / 16 * 16);
}
constexpr int kQrcpWarpCap = 24 << 10;  // per-warp region limit for the warp QRCP

// Grid-mode QRCP (slabs in shared memory, more CTAs per matrix than a cluster
// holds): matrix f of a launch runs on CTAs [cta0, cta0 + ctas) and exchanges
// proposals and reflectors through tags / slots / vg (device memory; tags holds
// the two arrival counters at ints 0 and 32, zeroed before the launch; vg
// holds 2 x ctas x ((m_max + 3) & ~1) elements).
struct QrcpSlot {
  double v, beta, tau;
  int j, stop;
};
struct QrcpGridDesc {
  int cta0, ctas;
  int* tags;        // two arrival counters (ints 0 and 32)
  QrcpSlot* slots;  // 2 x ctas
  void* vg;
};
// Exchange area of one grid-mode matrix: the counters (at least 64 ints, so
// that ints 0 and 32 exist), the slots, the reflector buffers, each part
// starting on a 256-byte boundary.
inline size_t qrcp_grid_tag_bytes(int ctas) {
  return (std::max<size_t>((size_t)2 * ctas, 64) * sizeof(int) + 255) & ~size_t(255);
}
inline size_t qrcp_grid_slot_bytes(int ctas) { return ((size_t)2 * ctas * sizeof(QrcpSlot) + 255) & ~size_t(255); }
inline size_t qrcp_grid_xchg_bytes(int ctas, int m_max, int elem) {
  return qrcp_grid_tag_bytes(ctas) + qrcp_grid_slot_bytes(ctas) +
         (((size_t)2 * ctas * ((m_max + 3) & ~1) * elem + 255) & ~size_t(255));
}
// descriptors of one grid-mode group whose exchange areas are laid out back to
// back from x (qrcp_grid_xchg_bytes each); returns the total CTA count
inline int qrcp_grid_descs(const std::vector<int>& ctas, int m_max, int elem, unsigned char* x,
                           std::vector<QrcpGridDesc>& out) {
  out.clear();
  int cta0 = 0;
  for (int c : ctas) {
    const size_t tb = qrcp_grid_tag_bytes(c), sb = qrcp_grid_slot_bytes(c);
    out.push_back(QrcpGridDesc{cta0, c, reinterpret_cast<int*>(x), reinterpret_cast<QrcpSlot*>(x + tb), x + tb + sb});
    x += qrcp_grid_xchg_bytes(c, m_max, elem);
    cta0 += c;
  }
  return cta0;
}
// Cooperative launch of one grid-mode group: gd[f].cta0 ascending, total_ctas
// = sum of ctas (all resident at once or the launch fails).  smem_slab: the
// column slabs live in shared memory, else in each descriptor's work buffer
// (m x n, ld m; the kernel copies src there first).
template <typename T>
cudaError_t launch_qrcp_grid(const QrcpDesc<T>* d, const QrcpGridDesc* gd, int count, int total_ctas, double eps,
                             int nl_max, int m_max, bool smem_slab, cudaStream_t st);
// CTAs of the grid-mode QRCP that fit on the device at once (SM count x
// resident CTAs per SM at the given dynamic shared memory, element size elem),
// at most one per thread of a CTA
int qrcp_grid_capacity(int smem_bytes, int elem);
// Wait limit of the grid-mode exchange in SM clock cycles (default about 2 s at
// the maximum SM clock) and a number of arrivals every wait expects beyond the
// CTAs that exist (0 in normal use; failure-path tests set it so that every
// wait expires).  An expired wait writes rank -1 for its matrix.
constexpr long long kQrcpGridWaitCyclesDefault = 4000000000LL;
void qrcp_grid_set_wait(long long cycles, int missing);

// Launch shape measured by the autotuner for matrices of this size class
// (autotune.cu): 0 = not tuned, 1..16 = CTAs with shared-memory slabs, 32 = 16
// CTAs over a global work copy.
int qrcp_tuned_choice(int elem, int m, int n);

inline bool plan_qrcp(const std::vector<int>& ms, const std::vector<int>& ns, int elem, int limit,
                      std::vector<QrcpGroup>& out, std::vector<char>& needs_work, int grid_ctas = 0,
                      bool force_grid = false) {
  const int nmat = (int)ms.size();
  needs_work.assign((size_t)nmat, 0);
  std::vector<int> cs((size_t)nmat), order;
  std::vector<char> slab((size_t)nmat);
  // warp groups first: small matrices, one warp each, packed 8 per CTA
  std::vector<int> rest, gridm, gridg;
  {
    QrcpGroup wg;
    wg.cs = 0;
    wg.slab = true;
    for (int i = 0; i < nmat; ++i) {
      const int wb = qrcp_warp_bytes(ms[(size_t)i], ns[(size_t)i], elem);
      if (ms[(size_t)i] <= 64 && wb <= kQrcpWarpCap && (long long)wb * 8 <= limit) {
        wg.idx.push_back(i);
        wg.nl_max = std::max(wg.nl_max, wb);  // per-warp bytes
        wg.m_max = std::max(wg.m_max, ms[(size_t)i]);
      } else {
        rest.push_back(i);
      }
    }
    out.clear();
    if (!wg.idx.empty()) out.push_back(wg);
  }
  for (int i : rest) {
    if (force_grid && grid_ctas > 16 &&
        qrcp_smem_bytes(ms[(size_t)i], (ns[(size_t)i] + grid_ctas - 1) / grid_ctas, elem, true) <= limit) {
      gridm.push_back(i);
      continue;
    }
    int c = 1;
    while (c < 16 && qrcp_smem_bytes(ms[(size_t)i], (ns[(size_t)i] + c - 1) / c, elem, true) > limit) c *= 2;
    const int tuned = qrcp_tuned_choice(elem, ms[(size_t)i], ns[(size_t)i]);
    if (tuned > c && tuned <= 16) c = tuned;  // a larger cluster always still fits
    const int nl = (ns[(size_t)i] + c - 1) / c;
    if (tuned != 32 && qrcp_smem_bytes(ms[(size_t)i], nl, elem, true) <= limit) {
      cs[(size_t)i] = c;
      slab[(size_t)i] = 1;
    } else if (tuned != 32 && grid_ctas > 16 &&
               qrcp_smem_bytes(ms[(size_t)i], (ns[(size_t)i] + grid_ctas - 1) / grid_ctas, elem, true) <= limit) {
      gridm.push_back(i);  // slabs in shared memory over more CTAs than a cluster holds
      continue;
    } else if (force_grid && grid_ctas > 16 && qrcp_grid_smem_bytes(ms[(size_t)i], 1, elem, false) <= limit) {
      gridg.push_back(i);  // too large for the slabs of every SM: CTA groups over a work copy
      continue;
    } else {
      cs[(size_t)i] = 16;
      slab[(size_t)i] = 0;
      needs_work[(size_t)i] = 1;
      if (!qrcp_panel_depth(ms[(size_t)i], (ns[(size_t)i] + 15) / 16, elem, limit)) return false;
    }
    order.push_back(i);
  }
  // FP64 pivoted QR is bound by the FP64 pipe: the delayed-update form on 16
  // SMs per matrix runs at about twice the FP64 efficiency of the CTA groups,
  // so once more than four such matrices fill the GPU it is the faster choice
  // (measured on 1 to 12 matrices of 1650 x 879); FP32 takes the groups always
  // Matrices too large for shared memory even over every SM take CTA groups
  // over a work copy only when forced (measured slower than the delayed form
  // on the 3D separator blocks: three passes through L2 per step against
  // about one); at most four share a launch.
  auto to_delayed = [&](std::vector<int>& v) {
    for (int i : v) {
      cs[(size_t)i] = 16;
      slab[(size_t)i] = 0;
      needs_work[(size_t)i] = 1;
      if (!qrcp_panel_depth(ms[(size_t)i], (ns[(size_t)i] + 15) / 16, elem, limit)) return false;
      order.push_back(i);
    }
    v.clear();
    return true;
  };
  if (!force_grid && elem == 8 && gridm.size() > 4 && !to_delayed(gridm)) return false;
  if (!force_grid && gridg.size() > 4 && !to_delayed(gridg)) return false;
  // spread small batches over more SMs: while the batch holds fewer CTAs than
  // the GPU has SMs, double the cluster of the largest shared-memory problems
  // that keep at least 64 columns per CTA
  // A cluster must sit inside one GPC (about 19 SMs on this GPU), so clusters
  // of 4 to 16 CTAs can hold only about 128 SMs at once (144 for pairs); a
  // size class is not grown past that (a second wave would double the time).
  {
    constexpr long long kSms = 152;
    auto cap = [](int c) -> long long { return c <= 1 ? 152 : (c == 2 ? 144 : 128); };
    long long ctas = 0;
    long long at[17] = {0};
    for (int i : order) {
      ctas += cs[(size_t)i];
      if (slab[(size_t)i]) at[cs[(size_t)i]] += cs[(size_t)i];
    }
    std::vector<int> bywork(order);
    std::sort(bywork.begin(), bywork.end(), [&](int a, int b) {
      const long long wa = (long long)ms[(size_t)a] * ns[(size_t)a], wb = (long long)ms[(size_t)b] * ns[(size_t)b];
      return wa != wb ? wa > wb : a < b;
    });
    bool grew = true;
    while (ctas < kSms && grew) {
      grew = false;
      for (int i : bywork) {
        if (ctas >= kSms) break;
        const int c2 = cs[(size_t)i] * 2;
        if (!slab[(size_t)i] || c2 > 16 || ns[(size_t)i] / c2 < 64) continue;
        if (at[c2] + c2 > cap(c2)) continue;
        at[cs[(size_t)i]] -= cs[(size_t)i];
        at[c2] += c2;
        ctas += cs[(size_t)i];
        cs[(size_t)i] = c2;
        grew = true;
      }
    }
  }
  // group by (cs, slab), larger footprints first, greedy packing under the limit
  const size_t first_cta_group = out.size();
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (cs[(size_t)a] != cs[(size_t)b]) return cs[(size_t)a] < cs[(size_t)b];
    if (slab[(size_t)a] != slab[(size_t)b]) return slab[(size_t)a] > slab[(size_t)b];
    const long long fa = (long long)ms[(size_t)a] * ((ns[(size_t)a] + cs[(size_t)a] - 1) / cs[(size_t)a]);
    const long long fb = (long long)ms[(size_t)b] * ((ns[(size_t)b] + cs[(size_t)b] - 1) / cs[(size_t)b]);
    return fa != fb ? fa > fb : a < b;
  });
  for (int i : order) {
    const int nl = (ns[(size_t)i] + cs[(size_t)i] - 1) / cs[(size_t)i];
    QrcpGroup* g = out.size() > first_cta_group ? &out.back() : nullptr;
    bool fits = g && g->cs == cs[(size_t)i] && g->slab == (bool)slab[(size_t)i] &&
                (g->slab ? qrcp_smem_bytes(std::max(g->m_max, ms[(size_t)i]), std::max(g->nl_max, nl), elem, true) <= limit
                         : (qrcp_panel_depth(std::max(g->m_max, ms[(size_t)i]), std::max(g->nl_max, nl), elem, limit) ==
                                qrcp_panel_depth(g->m_max, g->nl_max, elem, limit) &&
                            qrcp_panel_depth(ms[(size_t)i], nl, elem, limit) == qrcp_panel_depth(g->m_max, g->nl_max, elem, limit)));
    // keep small problems away from large footprints (occupancy)
    if (fits && g->slab) {
      const int cur = qrcp_smem_bytes(g->m_max, g->nl_max, elem, true);
      const int mine = qrcp_smem_bytes(ms[(size_t)i], nl, elem, true);
      if (cur > 4 * mine && cur > (24 << 10)) fits = false;
    }
    if (!fits) {
      out.emplace_back();
      g = &out.back();
      g->cs = cs[(size_t)i];
      g->slab = slab[(size_t)i];
    }
    g->m_max = std::max(g->m_max, ms[(size_t)i]);
    g->nl_max = std::max(g->nl_max, nl);
    g->idx.push_back(i);
  }
  for (auto& g : out)
    if (!g.slab && g.cs > 0) g.nb = qrcp_panel_depth(g.m_max, g.nl_max, elem, limit);
  // grid mode: each matrix takes the fewest CTAs whose slabs fit, matrices are
  // packed (taller first) into launches of at most grid_ctas CTAs whose common
  // footprint fits, then each launch spreads its spare CTAs over its widest
  // members (one CTA at a time, until a member has at most 8 columns per CTA:
  // one per warp)
  if (!gridm.empty()) {
    std::sort(gridm.begin(), gridm.end(), [&](int a, int b) {
      return ms[(size_t)a] != ms[(size_t)b] ? ms[(size_t)a] > ms[(size_t)b] : a < b;
    });
    auto min_ctas = [&](int i) {
      int g = 17;
      while (g < grid_ctas && qrcp_smem_bytes(ms[(size_t)i], (ns[(size_t)i] + g - 1) / g, elem, true) > limit) ++g;
      return g;
    };
    QrcpGroup* cur = nullptr;
    int used = 0;
    for (int i : gridm) {
      const int g = min_ctas(i);
      const int nl = (ns[(size_t)i] + g - 1) / g;
      const bool fits = cur && used + g <= grid_ctas &&
                        qrcp_smem_bytes(std::max(cur->m_max, ms[(size_t)i]), std::max(cur->nl_max, nl), elem, true) <= limit;
      if (!fits) {
        out.emplace_back();
        cur = &out.back();
        cur->grid = true;
        cur->slab = true;
        cur->cs = 0;
        used = 0;
      }
      cur->idx.push_back(i);
      cur->ctas.push_back(g);
      cur->m_max = std::max(cur->m_max, ms[(size_t)i]);
      cur->nl_max = std::max(cur->nl_max, nl);
      used += g;
    }
    for (auto& g : out) {
      if (!g.grid) continue;
      int tot = 0;
      for (int c : g.ctas) tot += c;
      bool grew = true;
      while (tot < grid_ctas && grew) {
        grew = false;
        for (size_t q = 0; q < g.idx.size() && tot < grid_ctas; ++q) {
          const int n = ns[(size_t)g.idx[q]];
          if ((n + g.ctas[q] - 1) / g.ctas[q] <= 8) continue;
          ++g.ctas[q];
          ++tot;
          grew = true;
        }
      }
      g.nl_max = 0;
      for (size_t q = 0; q < g.idx.size(); ++q)
        g.nl_max = std::max(g.nl_max, (ns[(size_t)g.idx[q]] + g.ctas[q] - 1) / g.ctas[q]);
    }
  }
  // work-copy groups (at most four matrices): one launch, the CTAs shared in
  // proportion to the column counts (at least 17 each)
  if (!gridg.empty()) {
    QrcpGroup g;
    g.grid = true;
    g.slab = false;
    g.cs = 0;
    long long ntot = 0;
    for (int i : gridg) ntot += ns[(size_t)i];
    int used = 0;
    for (int i : gridg) {
      int c = (int)std::max<long long>(17, (long long)grid_ctas * ns[(size_t)i] / std::max<long long>(ntot, 1));
      c = std::min(c, std::max(1, ns[(size_t)i]));
      c = std::max(c, 1);
      g.idx.push_back(i);
      g.ctas.push_back(c);
      used += c;
      needs_work[(size_t)i] = 1;
    }
    while (used > grid_ctas) {  // trim the largest share
      size_t q = 0;
      for (size_t t = 1; t < g.ctas.size(); ++t)
        if (g.ctas[t] > g.ctas[q]) q = t;
      --g.ctas[q];
      --used;
    }
    for (size_t q = 0; q < g.idx.size(); ++q) {
      g.m_max = std::max(g.m_max, ms[(size_t)g.idx[q]]);
      g.nl_max = std::max(g.nl_max, (ns[(size_t)g.idx[q]] + g.ctas[q] - 1) / g.ctas[q]);
    }
    if (qrcp_grid_smem_bytes(g.m_max, g.nl_max, elem, false) > limit) return false;
    out.push_back(std::move(g));
  }
  return true;
}

// Routing of a batch of fronts: kind 0 = one warp per front (param = elements
// per warp region), kind 1 = one CTA per front in shared memory (param =
// dynamic bytes), kind 2 = blocked multi-CTA path (param = max eliminated
// columns).  Fronts with c == 0 or an empty shape need no work and are skipped.
struct FrontGroup {
  int kind = 0;
  int param = 0;
  std::vector<int> idx;
};
int front_smem_bytes(int m, int n, int c, int elem);
inline std::vector<FrontGroup> plan_fronts(const std::vector<int>& ms, const std::vector<int>& ns,
                                           const std::vector<int>& cs, int elem, int limit) {
  const int tiny_cap[3] = {8 << 10, 16 << 10, 28 << 10};
  const int cta_cap[4] = {24 << 10, 48 << 10, 100 << 10, limit};
  std::vector<FrontGroup> g(8);
  for (int q = 0; q < 3; ++q) g[(size_t)q].kind = 0;
  for (int q = 0; q < 4; ++q) g[(size_t)q + 3].kind = 1;
  g[7].kind = 2;
  for (size_t i = 0; i < ms.size(); ++i) {
    const int m = ms[i], n = ns[i], c = cs[i];
    if (c == 0 || m == 0 || n == 0) continue;
    const long long wb = (long long)(m | 1) * n * elem;
    if (c <= 128 && m <= 256 && wb <= tiny_cap[2]) {
      int q = 0;
      while (wb > tiny_cap[q]) ++q;
      g[(size_t)q].idx.push_back((int)i);
      g[(size_t)q].param = std::max(g[(size_t)q].param, (m | 1) * n);
      continue;
    }
    if ((long long)m * n * elem + 64 <= limit) {
      const int need = front_smem_bytes(m, n, c, elem);
      int q = 0;
      while (q < 3 && need > cta_cap[q]) ++q;
      g[(size_t)q + 3].idx.push_back((int)i);
      g[(size_t)q + 3].param = std::max(g[(size_t)q + 3].param, need);
      continue;
    }
    g[7].idx.push_back((int)i);
    g[7].param = std::max(g[7].param, std::min(c, m));
  }
  std::vector<FrontGroup> out;
  for (auto& x : g)
    if (!x.idx.empty()) out.push_back(std::move(x));
  return out;
}

// Run every group of plan_fronts: d[g] are the device descriptor arrays of the
// groups (in order), Tbuf holds 32*32 elements per front of the blocked group.
// tc_scratch (FP32 only; may be null = SIMT trailing updates) holds
// front_groups_tc_bytes() bytes for the tensor-core trailing updates.
template <typename T>
cudaError_t launch_front_groups(const std::vector<FrontGroup>& groups, const std::vector<const FrontDesc<T>*>& d,
                                const std::vector<std::vector<FrontDesc<T>>>& host, T* Tbuf, cudaStream_t st,
                                int64_t* launches, void* tc_scratch = nullptr, int* tc_flag = nullptr);
template <typename T>
size_t front_groups_tc_bytes(const std::vector<FrontGroup>& groups, const std::vector<std::vector<FrontDesc<T>>>& host);

inline int front_smem_bytes(int m, int n, int c, int elem) {
  return (int)((long long)m * n * elem + ((c + 31) / 32) * 4 + 16);
}
// The next three take work items (descriptor index, first vector/row): one CTA
// per item; refl covers 8 vectors per item, trsm and argmax 256 rows.
template <typename T> cudaError_t launch_refl(const ReflDesc<T>* d, const int2* items, int nitems, cudaStream_t st);
template <typename T> cudaError_t launch_trsm(const TrsmDesc<T>* d, const int2* items, int nitems, cudaStream_t st);
template <typename T> cudaError_t launch_argmax(const ArgmaxDesc<T>* d, const int2* items, int nitems, cudaStream_t st);
constexpr int kReflPerItem = 8;        // column vectors: one per warp
constexpr int kReflRowsPerItem = 256;  // row vectors: one per thread
constexpr int kRowsPerItem = 256;
// Write an identity c x c block at ptr (ld) for each desc (src/transposed unused).
template <typename T> cudaError_t launch_identity(const CopyDesc<T>* d, int count, cudaStream_t st);

// base[dest[e]] = vals[e] for e < n (initial matrix into the group blocks)
template <typename T> cudaError_t launch_scatter_values(T* base, const int64_t* dest, const T* vals, int64_t n, cudaStream_t st);

int max_smem_optin();

// ---------------------------------------------- tensor-core trailing update
// One panel step of the FP32 blocked front QR on tcgen05 in 3xTF32
// (tc_kernels.cu): with V = the b (<= 32) reflectors of columns j0..j0+b-1 of
// X (rows j0..m-1) and T (32 x 32, ld 32) from the panel kernel,
// C = X[j0:m, j0+b : j0+b+ncols] <- C - V T^T V^T C.  P and Wp are scratch
// (tc_panel_scratch floats from P, Wp right after).
struct TcPanel {
  float* X;
  const float* Tm;
  float* P;
  float* Wp;
  int mr, ld, j0, b, ncols;  // mr = m - j0 rows
  int nsl, rps;              // row slices of the projection and rows per slice (tc_plan_panel)
  int* flag;                 // device int set to 1 when an MMA completion wait gives up (may be null)
};
void tc_plan_panel(TcPanel& f);
size_t tc_panel_scratch(const TcPanel& f);
cudaError_t launch_tc_panels(const TcPanel* d_panels, const std::vector<TcPanel>& host, cudaStream_t st);
// C[0:m, 0:n] -= A[0:m, 0:k] B[0:k, 0:n] (FP32, column-major) on tcgen05, 3xTF32
// (flag: device int set to 1 if an MMA completion wait gives up; may be null)
cudaError_t launch_tc_gemm(int m, int n, int k, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                           int* flag, cudaStream_t st);

}  // namespace spaqr
