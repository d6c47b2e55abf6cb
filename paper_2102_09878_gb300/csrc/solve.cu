// Apply of the stored factor W and the W-preconditioned CGLS (Section 2.7,
// Section 4).
//
// W = W_1 ... W_L with W_l = (prod Q_p^T)(prod R_p)(prod R_s) for the
// operations of stage l.  W^{-1} z replays the operations in reverse
// factorization order, W^{-T} z in factorization order.  Operations of one
// elimination round, of one scaling phase and of one step-2 phase act on
// disjoint slots and form one "segment".
//
// Each op takes one of two forms:
//  * small (c <= 32, and at most kWideW R_sn columns): one warp per op, the
//    triangular solves by shuffles, Q_pp as its Householder product;
//  * dense (all others): the op is replaced, once after the factorization, by
//    the dense operator it applies, G = R^{-1} [I  -R_sn] (c x (c + w)) for
//    R_s and R_p, G = Q_pp for Q_p.  With G = [X Y]:
//      W^{-1}:  z_s <- G [z_s; z_n]
//      W^{-T}:  z_s <- X^T z_s,  z_n <- z_n + Y^T z_s
//    Both run as tiled GEMVs over many CTAs (one partial sum per tile),
//    followed by a pass that reduces the partials in a fixed order and
//    scatters them to the slot vector.
// Q_p ops of rank 0 are the identity and are skipped.
//
// Slot vectors are FP64 in memory.  The arithmetic type TA is FP64 with the
// FP64 factor and FP32 with the mixed-precision (FP32) factor: the apply is
// the preconditioner, while the CGLS recurrences, residuals and norms stay
// FP64 (and x, r are updated from the same computed W^{-1} p, so they stay
// consistent).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "internal.h"

namespace spaqr {

namespace {
constexpr int kT = 256;
constexpr int kW = kT / 32;
constexpr int kWideW = 128;  // R_s ops with more R_sn columns take the dense form
constexpr int kTile = 8192;  // entries of one GEMV tile: 32 x 256 (c <= 32) or 128 x 64
constexpr int kStage = 256 * 33;  // staged tile of the transposed GEMV, padded

template <typename TW>
constexpr size_t kWarpSmem = (size_t)kW * 32 * 33 * sizeof(TW);  // staged R_ss per warp

template <typename TW>
struct SmallOp {
  const TW* R;     // kind 0: c x (c + w) = [R_ss R_sn]; kind 1: c x c; ld c
  const TW* V;     // kind 2: reflectors, c x k, ld c
  const TW* tau;
  const int32_t* slots;
  const int32_t* nslots;
  const double* rdiag;  // kinds 0, 1: 1 / R_ii
  int c, w, k;
};

template <typename TW>
struct DenseOp {
  TW* G;  // c x (c + w), ld c
  const TW* R;
  const TW* V;
  const TW* tau;
  const int32_t* slots;
  const int32_t* nslots;
  int64_t poff_f, poff_t;  // this op's partial sums in the segment scratch (W^{-1}, W^{-T})
  int c, w, k, kind;
  int tr, nrt, nct;  // tile rows (32 or 128), row tiles, column tiles
  int tri;           // X = G[:, :c] upper triangular: tiles strictly below the diagonal are skipped
};

__host__ __device__ inline int tile_cols(int tr) { return kTile / tr; }

template <typename TA>
__device__ __forceinline__ TA wsum(TA v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------- small ops: one warp per op
// W^{-1}: z_s <- R_ss^{-1} (z_s - R_sn z_n) (kind 0), z_p <- R_pp^{-1} z_p (kind 1).
// Lane i holds row i; R_ss is staged in the warp's shared region B (32 x 33).
template <typename TW, typename TA>
__device__ __forceinline__ void r_inv_warp_op(const SmallOp<TW>& op, double* z, TW* B) {
  const int lane = threadIdx.x & 31, c = op.c, w = op.w;
  TA x = lane < c ? (TA)z[op.slots[lane]] : TA(0);
  if (w > 0) {
    const TW* Rn = op.R + (int64_t)c * c;
    TA acc = TA(0);
    for (int j0 = 0; j0 < w; j0 += 32) {
      const TA zl = (j0 + lane < w) ? (TA)z[op.nslots[j0 + lane]] : TA(0);
      const int jn = min(32, w - j0);
      for (int t = 0; t < jn; ++t) {
        const TA zj = __shfl_sync(0xffffffffu, zl, t);
        if (lane < c) acc += (TA)Rn[lane + (int64_t)(j0 + t) * c] * zj;
      }
    }
    x -= acc;
  }
  for (int q = 0; q < c; ++q)
    if (lane < c) B[lane * 33 + q] = op.R[lane + (int64_t)q * c];
  const TA rd = lane < c ? (TA)op.rdiag[lane] : TA(0);
  __syncwarp();
  for (int j = c - 1; j >= 0; --j) {
    const TA yj = __shfl_sync(0xffffffffu, x, j) * __shfl_sync(0xffffffffu, rd, j);
    if (lane == j) x = yj;
    if (lane < j) x -= (TA)B[lane * 33 + j] * yj;
  }
  if (lane < c) z[op.slots[lane]] = (double)x;
  __syncwarp();
}

// W^{-T}: y = R_ss^{-T} z_s, z_s <- y, z_n -= R_sn^T y (kind 0); z_p <- R_pp^{-T} z_p (kind 1).
// The R_sn^T y products run lane-per-column (y broadcast by shuffles).
template <typename TW, typename TA>
__device__ __forceinline__ void r_invT_warp_op(const SmallOp<TW>& op, double* z, TW* B) {
  const int lane = threadIdx.x & 31, c = op.c, w = op.w;
  TA x = lane < c ? (TA)z[op.slots[lane]] : TA(0);
  for (int q = 0; q < c; ++q)
    if (lane < c) B[lane * 33 + q] = op.R[lane + (int64_t)q * c];
  const TA rd = lane < c ? (TA)op.rdiag[lane] : TA(0);
  __syncwarp();
  for (int i = 0; i < c; ++i) {
    const TA yi = __shfl_sync(0xffffffffu, x, i) * __shfl_sync(0xffffffffu, rd, i);
    if (lane == i) x = yi;
    if (lane > i && lane < c) x -= (TA)B[i * 33 + lane] * yi;
  }
  if (lane < c) z[op.slots[lane]] = (double)x;
  if (w > 0) {
    const TW* Rn = op.R + (int64_t)c * c;
    for (int j0 = 0; j0 < w; j0 += 32) {
      const int j = j0 + lane;
      const TW* col = Rn + (int64_t)(j < w ? j : 0) * c;
      TA acc = TA(0);
      for (int i = 0; i < c; ++i) acc += (TA)col[i] * __shfl_sync(0xffffffffu, x, i);
      if (j < w) atomicAdd(&z[op.nslots[j]], -(double)acc);
    }
  }
  __syncwarp();
}

// W^{-1}: z_p <- Q_pp z_p = H_1 ... H_k z_p;  W^{-T}: z_p <- Q_pp^T z_p.
template <typename TW, typename TA>
__device__ __forceinline__ void q_warp_op(const SmallOp<TW>& op, double* z, int transpose) {
  const int lane = threadIdx.x & 31, c = op.c, k = op.k;
  TA x = lane < c ? (TA)z[op.slots[lane]] : TA(0);
  for (int t = 0; t < k; ++t) {
    const int i = transpose ? t : k - 1 - t;
    const TA v = lane == i ? TA(1) : ((lane > i && lane < c) ? (TA)op.V[lane + (int64_t)i * c] : TA(0));
    const TA d = wsum(v * x) * (TA)op.tau[i];
    x -= d * v;
  }
  if (lane < c) z[op.slots[lane]] = (double)x;
}

template <typename TW, typename TA>
__global__ void __launch_bounds__(kT) r_inv_warp_kernel(const SmallOp<TW>* ops, int count, double* z) {
  const int gw = (int)((blockIdx.x * (unsigned)kT + threadIdx.x) >> 5);
  if (gw >= count) return;
  extern __shared__ __align__(16) unsigned char wsm[];
  r_inv_warp_op<TW, TA>(ops[gw], z, reinterpret_cast<TW*>(wsm) + (size_t)(threadIdx.x >> 5) * (32 * 33));
}

template <typename TW, typename TA>
__global__ void __launch_bounds__(kT) r_invT_warp_kernel(const SmallOp<TW>* ops, int count, double* z) {
  const int gw = (int)((blockIdx.x * (unsigned)kT + threadIdx.x) >> 5);
  if (gw >= count) return;
  extern __shared__ __align__(16) unsigned char wsm[];
  r_invT_warp_op<TW, TA>(ops[gw], z, reinterpret_cast<TW*>(wsm) + (size_t)(threadIdx.x >> 5) * (32 * 33));
}

template <typename TW, typename TA>
__global__ void __launch_bounds__(kT) q_warp_kernel(const SmallOp<TW>* ops, int count, double* z, int transpose) {
  const int gw = (int)((blockIdx.x * (unsigned)kT + threadIdx.x) >> 5);
  if (gw >= count) return;
  q_warp_op<TW, TA>(ops[gw], z, transpose);
}

// ------------------------------------------- dense ops: tiled GEMVs
// W^{-1} partials of one tile: part[poff_f + ct c + i] = sum over the tile's
// columns j of G[i, j] u_j, u = [z_s; z_n].  Thread (row, column group); a warp
// reads 32 consecutive rows of a column.  u (256) and red (kT) in shared memory.
template <typename TW, typename TA>
__device__ void dense_fwd_tile(const DenseOp<TW>* dops, int4 tl, const double* z, TA* part, TA* u, TA* red) {
  const DenseOp<TW>* op = dops + tl.x;
  const int c = op->c, ncol = c + op->w, TR = op->tr, TC = tile_cols(TR);
  const int r0 = tl.y * TR, c0 = tl.z * TC;
  const int nr = min(TR, c - r0), nc = min(TC, ncol - c0);
  const int32_t* slots = op->slots;
  const int32_t* nslots = op->nslots;
  for (int j = threadIdx.x; j < nc; j += kT) {
    const int jj = c0 + j;
    u[j] = (TA)z[jj < c ? slots[jj] : nslots[jj - c]];
  }
  __syncthreads();
  const int groups = kT / TR, ri = threadIdx.x % TR, g = threadIdx.x / TR;
  TA acc = TA(0);
  if (ri < nr) {
    const TW* base = op->G + (r0 + ri) + (int64_t)c0 * c;
#pragma unroll 8
    for (int j = g; j < nc; j += groups) acc += (TA)base[(int64_t)j * c] * u[j];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < nr) {
    TA s = TA(0);
    for (int q = 0; q < groups; ++q) s += red[q * TR + threadIdx.x];
    part[op->poff_f + (int64_t)tl.z * c + r0 + threadIdx.x] = s;
  }
}

// W^{-T} partials of one tile: part[poff_t + rt (c + w) + j] = sum over the
// tile's rows i of G[i, j] v_i, v = z_s.  The tile is staged in shared memory
// (s, TC x (TR + 1)), then thread (column, row group).
template <typename TW, typename TA>
__device__ void dense_T_tile(const DenseOp<TW>* dops, int4 tl, const double* z, TA* part, TW* s, TA* v, TA* red) {
  const DenseOp<TW>* op = dops + tl.x;
  const int c = op->c, ncol = c + op->w, TR = op->tr, TC = tile_cols(TR);
  const int r0 = tl.y * TR, c0 = tl.z * TC;
  const int nr = min(TR, c - r0), nc = min(TC, ncol - c0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < nr; i += kT) v[i] = (TA)z[op->slots[r0 + i]];
  const TW* G = op->G + r0 + (int64_t)c0 * c;
  for (int q = warp; q < nc; q += kW)
    for (int r = lane; r < nr; r += 32) s[q * (TR + 1) + r] = G[r + (int64_t)q * c];
  __syncthreads();
  const int groups = kT / TC, cj = threadIdx.x % TC, g = threadIdx.x / TC;
  TA acc = TA(0);
  if (cj < nc) {
    const int i1 = min(nr, g * 32 + 32);
    const TW* col = s + cj * (TR + 1);
    for (int i = g * 32; i < i1; ++i) acc += (TA)col[i] * v[i];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < nc) {
    TA t = TA(0);
    for (int q = 0; q < groups; ++q) t += red[q * TC + threadIdx.x];
    part[op->poff_t + (int64_t)tl.y * ncol + c0 + threadIdx.x] = t;
  }
}

// z_s[i] <- sum over the column tiles of the partials (fixed order)
template <typename TW, typename TA>
__device__ __forceinline__ void dense_fwd_reduce(const DenseOp<TW>* dops, int2 it, const TA* part, double* z) {
  const DenseOp<TW>* op = dops + it.x;
  const int i = it.y + threadIdx.x, c = op->c;
  if (i >= c) return;
  const int TR = op->tr, TC = tile_cols(TR);
  const int ct0 = op->tri ? ((i / TR) * TR) / TC : 0;
  TA s = TA(0);
  for (int ct = ct0; ct < op->nct; ++ct) s += part[op->poff_f + (int64_t)ct * c + i];
  z[op->slots[i]] = (double)s;
}

// z_s[j] <- sum over the row tiles (j < c);  z_n[j - c] += sum (j >= c)
template <typename TW, typename TA>
__device__ __forceinline__ void dense_T_reduce(const DenseOp<TW>* dops, int2 it, const TA* part, double* z) {
  const DenseOp<TW>* op = dops + it.x;
  const int c = op->c, ncol = c + op->w, j = it.y + threadIdx.x;
  if (j >= ncol) return;
  const int TR = op->tr, TC = tile_cols(TR);
  int rt1 = op->nrt - 1;
  if (op->tri) rt1 = min(rt1, ((j / TC + 1) * TC - 1) / TR);
  TA s = TA(0);
  for (int rt = 0; rt <= rt1; ++rt) s += part[op->poff_t + (int64_t)rt * ncol + j];
  if (j < c)
    z[op->slots[j]] = (double)s;
  else
    atomicAdd(&z[op->nslots[j - c]], (double)s);
}

template <typename TW, typename TA>
__global__ void __launch_bounds__(kT) dense_fwd_kernel(const DenseOp<TW>* dops, const int4* tiles, const double* z,
                                                       TA* part) {
  __shared__ TA u[256];
  __shared__ TA red[kT];
  dense_fwd_tile<TW, TA>(dops, tiles[blockIdx.x], z, part, u, red);
}

template <typename TW, typename TA>
__global__ void __launch_bounds__(kT) dense_T_kernel(const DenseOp<TW>* dops, const int4* tiles, const double* z,
                                                     TA* part) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ TA v[128];
  __shared__ TA red[kT];
  dense_T_tile<TW, TA>(dops, tiles[blockIdx.x], z, part, reinterpret_cast<TW*>(dsm), v, red);
}

template <typename TW, typename TA>
__global__ void __launch_bounds__(kT) dense_fwd_reduce_kernel(const DenseOp<TW>* dops, const int2* items,
                                                              const TA* part, double* z) {
  dense_fwd_reduce<TW, TA>(dops, items[blockIdx.x], part, z);
}

template <typename TW, typename TA>
__global__ void __launch_bounds__(kT) dense_T_reduce_kernel(const DenseOp<TW>* dops, const int2* items,
                                                            const TA* part, double* z) {
  dense_T_reduce<TW, TA>(dops, items[blockIdx.x], part, z);
}

// ------------------------------------------- the whole apply in one launch
// Segments on the device; the persistent kernel below walks them in order.
struct SegDev {
  int kind, small0, nsmall, tile0, ntile, rf0, nrf, rt0, nrt;
};

constexpr long long kBarrierLimit = 1LL << 28;  // polls before a barrier gives up (seconds)

// Software barrier of all CTAs of a cooperative launch (all co-resident):
// bar[0] counts arrivals, bar[1] is the generation.  Bounded: a CTA that waits
// too long records the error and proceeds.
__device__ __forceinline__ void grid_sync(unsigned* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (++it > kBarrierLimit) {
          atomicExch(err, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// W^{-1} (transpose = 0) or W^{-T} in one cooperative launch: per segment the
// small ops (one warp each over all warps of the grid) and the dense tiles
// (one CTA each), a grid barrier, the ordered reductions, a grid barrier.
template <typename TW, typename TA>
__global__ void __launch_bounds__(kT) apply_persistent_kernel(const SegDev* segs, int nseg, const SmallOp<TW>* small,
                                                              const DenseOp<TW>* dense, const int4* tiles,
                                                              const int2* red, TA* part, double* z, int transpose,
                                                              unsigned* bar, int* err) {
  extern __shared__ __align__(16) unsigned char psm[];
  __shared__ TA s_u[256];
  __shared__ TA s_red[kT];
  __shared__ TA s_v[128];
  TW* B = reinterpret_cast<TW*>(psm) + (size_t)(threadIdx.x >> 5) * (32 * 33);
  TW* stage = reinterpret_cast<TW*>(psm);
  const int gw = (int)((blockIdx.x * (unsigned)kT + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * (unsigned)kT) >> 5);
  for (int t = 0; t < nseg; ++t) {
    const SegDev s = segs[transpose ? t : nseg - 1 - t];
    const SmallOp<TW>* ops = small + s.small0;
    for (int o = gw; o < s.nsmall; o += nw) {
      const SmallOp<TW> op = ops[o];
      if (s.kind == 2)
        q_warp_op<TW, TA>(op, z, transpose);
      else if (transpose)
        r_invT_warp_op<TW, TA>(op, z, B);
      else
        r_inv_warp_op<TW, TA>(op, z, B);
    }
    if (s.ntile) {
      __syncthreads();  // the warps' shared regions are free before a tile stages into them
      for (int q = blockIdx.x; q < s.ntile; q += gridDim.x) {
        const int4 tl = tiles[s.tile0 + q];
        if (transpose)
          dense_T_tile<TW, TA>(dense, tl, z, part, stage, s_v, s_red);
        else
          dense_fwd_tile<TW, TA>(dense, tl, z, part, s_u, s_red);
        __syncthreads();
      }
      grid_sync(bar, err);
      const int nred = transpose ? s.nrt : s.nrf, r0 = transpose ? s.rt0 : s.rf0;
      for (int q = blockIdx.x; q < nred; q += gridDim.x) {
        if (transpose)
          dense_T_reduce<TW, TA>(dense, red[r0 + q], part, z);
        else
          dense_fwd_reduce<TW, TA>(dense, red[r0 + q], part, z);
      }
    }
    grid_sync(bar, err);
  }
}

// Forms column j of every dense operator in FP64 (one warp per column, work
// vector y in global scratch):  Q_pp e_j = H_1 (... (H_k e_j)) for Q_p ops;
// for R ops the column-oriented back substitution R g = b with b = e_j
// (j < c) or b = -R_sn[:, j - c].
template <typename TW>
__global__ void __launch_bounds__(kT) form_dense_kernel(const DenseOp<TW>* dops, const int2* items, int64_t nitems,
                                                        double* scratch, int cmax) {
  // in the arithmetic of the stored factor (FP64, or FP32 for the mixed-precision
  // factor: the applies use G and G^T alike, so the operator stays consistent)
  using A = TW;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kT) >> 5;
  A* y = reinterpret_cast<A*>(scratch) + gw * cmax;
  for (int64_t t = gw; t < nitems; t += nw) {
    const int2 it = items[t];
    const DenseOp<TW>* op = dops + it.x;
    const int c = op->c, j = it.y;
    if (op->kind == 2) {
      for (int i = lane; i < c; i += 32) y[i] = i == j ? A(1) : A(0);
      __syncwarp();
      for (int q = op->k - 1; q >= 0; --q) {
        const TW* v = op->V + (int64_t)q * c;
        A d = A(0);
        for (int i = q + lane; i < c; i += 32) d += (i == q ? A(1) : (A)v[i]) * y[i];
        d = wsum(d) * (A)op->tau[q];
        for (int i = q + lane; i < c; i += 32) y[i] -= d * (i == q ? A(1) : (A)v[i]);
        __syncwarp();
      }
    } else {
      const TW* R = op->R;
      int top = c - 1;
      if (j < c) {
        for (int i = lane; i < c; i += 32) y[i] = i == j ? A(1) : A(0);
        top = j;
      } else {
        const TW* b = R + (int64_t)j * c;  // column j - c of R_sn
        for (int i = lane; i < c; i += 32) y[i] = -(A)b[i];
      }
      __syncwarp();
      for (int i = top; i >= 0; --i) {
        const A yi = y[i] / (A)R[i + (int64_t)i * c];
        __syncwarp();
        if (lane == 0) y[i] = yi;
        const TW* col = R + (int64_t)i * c;
        for (int r = lane; r < i; r += 32) y[r] -= yi * (A)col[r];
        __syncwarp();
      }
    }
    TW* out = op->G + (int64_t)j * c;
    for (int i = lane; i < c; i += 32) out[i] = (TW)y[i];
    __syncwarp();
  }
}

// 1 / R_ii of every small triangular op (one warp per op).
template <typename TW>
__global__ void __launch_bounds__(kT) recip_diag_kernel(const SmallOp<TW>* ops, int nops) {
  const int gw = (int)((blockIdx.x * (unsigned)kT + threadIdx.x) >> 5);
  if (gw >= nops) return;
  const SmallOp<TW> op = ops[gw];
  if (!op.rdiag) return;
  double* rd = const_cast<double*>(op.rdiag);
  for (int i = threadIdx.x & 31; i < op.c; i += 32) rd[i] = 1.0 / (double)op.R[i + (int64_t)i * op.c];
}

// ----------------------------------------------------------- CGLS kernels
// y = A x (CSR, one thread per row) with per-block partial sums of y_i^2 * wgt_i^2
__global__ void __launch_bounds__(kT) spmv_kernel(int64_t rows, const int64_t* rp, const int32_t* ci, const double* v,
                                                  const double* x, double* y, const double* wdiv, double* part) {
  __shared__ double red[kW];
  const int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x;
  double sq = 0.0;
  if (r < rows) {
    double s = 0.0;
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e) s += v[e] * x[ci[e]];
    y[r] = s;
    const double q = wdiv ? s / wdiv[r] : s;
    sq = q * q;
  }
  sq = wsum(sq);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kW; ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kT) sumsq_kernel(int64_t n, const double* x, double* part) {
  __shared__ double red[kW];
  double sq = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) sq += x[i] * x[i];
  sq = wsum(sq);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kW; ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

// out = sum of part[0..n) in a fixed order (one block)
__global__ void __launch_bounds__(kT) finish_sum_kernel(int n, const double* part, double* out) {
  __shared__ double red[kT];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kT) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// scal[0] = gamma, scal[1] = |q|^2, scal[2] = |D^-1 u|^2, scal[3] = |s|^2, scal[4] = beta
__global__ void __launch_bounds__(kT) update_xr_kernel(int64_t n, int64_t m, double* x, const double* t, double* r,
                                                       const double* q, const double* scal) {
  const double alpha = scal[0] / scal[1];
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i < n) x[i] += alpha * t[i];
  if (i < m) r[i] -= alpha * q[i];
}

__global__ void beta_kernel(double* scal) {
  scal[4] = scal[3] / scal[0];
  scal[0] = scal[3];
}

__global__ void __launch_bounds__(kT) update_p_kernel(int64_t n, double* p, const double* s, const double* scal) {
  const double beta = scal[4];
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i < n) p[i] = s[i] + beta * p[i];
}

// x <- x + s (n entries), r <- r - q (m entries): one refinement step of the
// corrected seminormal equations
__global__ void __launch_bounds__(kT) csne_update_kernel(int64_t n, int64_t m, double* x, const double* s, double* r,
                                                         const double* q) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i < n) x[i] += s[i];
  if (i < m) r[i] -= q[i];
}

__global__ void __launch_bounds__(kT) scale_kernel(int64_t n, const double* a, const double* d, double* out) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i < n) out[i] = a[i] * d[i];
}

// per-block partial sums of x_i y_i / wdiv_i^2 (wdiv may be null)
__global__ void __launch_bounds__(kT) dot_kernel(int64_t n, const double* x, const double* y, const double* wdiv,
                                                 double* part) {
  __shared__ double red[kW];
  double sq = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const double t = x[i] * y[i];
    sq += wdiv ? t / (wdiv[i] * wdiv[i]) : t;
  }
  sq = wsum(sq);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kW; ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

// Adjoint of x = argmin ||A x - b|| = (A^T A)^{-1} A^T b.  With lambda =
// (A^T A)^{-1} g_x and r = b - A x (one thread per row of A; A = A~ D^{-1}):
//   g_b = A lambda,   g_A[i, j] = r_i lambda_j - (A lambda)_i x_j  on the nonzeros.
__global__ void __launch_bounds__(kT) lstsq_grad_kernel(int64_t m, const int64_t* rp, const int32_t* ci,
                                                        const double* vs, const double* D, const double* b,
                                                        const double* x, const double* lam, double* gb,
                                                        double* gv) {
  const int64_t r = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (r >= m) return;
  double ax = 0.0, al = 0.0;
  for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
    const int32_t j = ci[e];
    const double a = vs[e] / D[j];
    ax += a * x[j];
    al += a * lam[j];
  }
  const double rr = b[r] - ax;
  if (gb) gb[r] = al;
  if (gv)
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int32_t j = ci[e];
      gv[e] = rr * lam[j] - al * x[j];
    }
}

// New values of A (same pattern): A~ = A D for the row-major and the transposed copies.
__global__ void __launch_bounds__(kT) set_values_kernel(int64_t nnz, const double* a, const int32_t* ci,
                                                        const double* D, double* vs) {
  const int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (e < nnz) vs[e] = a[e] * D[ci[e]];
}

__global__ void __launch_bounds__(kT) gather_values_kernel(int64_t nnz, const double* vs, const int64_t* perm,
                                                           double* tv) {
  const int64_t q = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (q < nnz) tv[q] = vs[perm[q]];
}

int blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + kT - 1) / kT); }

}  // namespace

// ------------------------------------------------------------------ plan
struct Segment {
  int kind;            // 0 R_s, 1 R_p, 2 Q_p
  int small0, nsmall;  // small ops (segment-contiguous in the small-op array)
  int tile0, ntile;    // GEMV tiles of the dense ops
  int rf0, nrf;        // W^{-1} reduce items
  int rt0, nrt;        // W^{-T} reduce items
};

struct ApplyPlan {
  cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool fp32 = false;
  double* d_rdiag = nullptr;
  void* d_small = nullptr;  // SmallOp<TW>[]
  void* d_dense = nullptr;  // DenseOp<TW>[]
  int32_t* d_idx = nullptr;
  int4* d_tiles = nullptr;
  int2* d_red = nullptr;    // reduce items (W^{-1} ones, then W^{-T} ones)
  void* d_dpart = nullptr;  // partial sums of the dense GEMVs (TA), sized for the largest segment
  std::vector<Segment> segs;  // factorization order
  int64_t launches = 0;       // kernel launches of one W^{-1} (equal for W^{-T})
  SegDev* d_segs = nullptr;      // the segments for the persistent apply
  unsigned* d_bar = nullptr;     // its grid barrier (count, generation)
  int* d_err = nullptr;          // set when a grid barrier gave up
  int pgrid = 0;                 // CTAs of the persistent launch (all co-resident); 0 = per-segment launches
  size_t psmem = 0;
  cudaGraphExec_t graph = nullptr;      // one CGLS iteration
  cudaGraphExec_t graph_pcg = nullptr;  // one PCG iteration
  cudaGraphExec_t graph_csne = nullptr;  // one CSNE refinement step
  double* h_res = nullptr;              // pinned host copy of the residual norm
  double* d_scal = nullptr;
  double* d_part = nullptr;
  int part_n = 0;
};

// Allow a kernel the opt-in shared memory minus its static footprint.
template <typename K>
static void set_dyn_smem(K kernel) {
  int dev = 0, mx = 0;
  SPAQR_CUDA(cudaGetDevice(&dev));
  SPAQR_CUDA(cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  SPAQR_CUDA(cudaFuncGetAttributes(&fa, kernel));
  SPAQR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes));
}

// one cooperative launch of the persistent apply (W^{-1}: transpose = 0)
template <typename TW, typename TA>
static cudaError_t launch_persistent(Handle& h, double* z, int transpose) {
  ApplyPlan& P = *h.plan;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)P.pgrid);
  cfg.blockDim = dim3(kT);
  cfg.dynamicSmemBytes = P.psmem;
  cfg.stream = h.st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, apply_persistent_kernel<TW, TA>, static_cast<const SegDev*>(P.d_segs),
                            (int)P.segs.size(), static_cast<const SmallOp<TW>*>(P.d_small),
                            static_cast<const DenseOp<TW>*>(P.d_dense), static_cast<const int4*>(P.d_tiles),
                            static_cast<const int2*>(P.d_red), static_cast<TA*>(P.d_dpart), z, transpose, P.d_bar,
                            P.d_err);
}

template <typename TW, typename TA>
static void build_plan_t(Handle& h, ApplyPlan& P) {
  const size_t nops = h.ops.size();
  // op form: 0 skipped (identity), 1 small, 2 dense
  std::vector<int> form(nops, 0);
  for (size_t i = 0; i < nops; ++i) {
    const WOp& op = h.ops[i];
    if (op.c <= 0 || (op.kind == 2 && op.k <= 0))
      form[i] = 0;
    else if (op.c <= 32 && (op.kind != 0 || op.w <= kWideW))
      form[i] = 1;
    else
      form[i] = 2;
  }
  std::vector<int32_t> idx;
  std::vector<size_t> soff(nops), noff(nops);
  for (size_t i = 0; i < nops; ++i) {
    const WOp& op = h.ops[i];
    soff[i] = idx.size();
    idx.insert(idx.end(), op.slots.begin(), op.slots.end());
    noff[i] = idx.size();
    idx.insert(idx.end(), op.nslots.begin(), op.nslots.end());
  }
  SPAQR_CUDA(dmalloc(&P.d_idx, std::max<size_t>(idx.size(), 1) * sizeof(int32_t)));
  SPAQR_CUDA(cudaMemcpy(P.d_idx, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  size_t nrd = 0;
  for (size_t i = 0; i < nops; ++i)
    if (form[i] == 1 && h.ops[i].kind != 2) nrd += (size_t)h.ops[i].c;
  SPAQR_CUDA(dmalloc(&P.d_rdiag, std::max<size_t>(nrd, 1) * sizeof(double)));

  std::vector<SmallOp<TW>> small;
  std::vector<DenseOp<TW>> dense;
  std::vector<int4> tiles;
  std::vector<int2> red_f, red_t;
  std::vector<int2> form_items;
  std::vector<Segment> segs;
  size_t rd_next = 0, part_max = 0;
  int cmax = 0;
  size_t i = 0;
  while (i < nops) {
    const WOp& a = h.ops[i];
    size_t j = i + 1;
    while (j < nops && h.ops[j].kind == a.kind && h.ops[j].stage == a.stage &&
           (a.kind != 0 || h.ops[j].round == a.round))
      ++j;
    Segment sg{a.kind, (int)small.size(), 0, (int)tiles.size(), 0, (int)red_f.size(), 0, (int)red_t.size(), 0};
    int64_t pf = 0, pt = 0;
    for (size_t q = i; q < j; ++q) {
      WOp& op = h.ops[q];
      const int32_t* sl = P.d_idx + soff[q];
      const int32_t* nl = P.d_idx + noff[q];
      if (form[q] == 1) {
        SmallOp<TW> s{};
        s.R = static_cast<const TW*>(op.R);
        s.V = static_cast<const TW*>(op.V);
        s.tau = static_cast<const TW*>(op.tau);
        s.slots = sl;
        s.nslots = nl;
        s.rdiag = nullptr;
        if (op.kind != 2) {
          s.rdiag = P.d_rdiag + rd_next;
          rd_next += (size_t)op.c;
        }
        s.c = op.c;
        s.w = op.kind == 0 ? op.w : 0;
        s.k = op.kind == 2 ? op.k : 0;
        small.push_back(s);
      } else if (form[q] == 2) {
        DenseOp<TW> d{};
        const int w = op.kind == 0 ? op.w : 0;
        const int ncol = op.c + w;
        op.G = h.wpool.alloc((size_t)op.c * ncol * sizeof(TW));
        d.G = static_cast<TW*>(op.G);
        d.R = static_cast<const TW*>(op.R);
        d.V = static_cast<const TW*>(op.V);
        d.tau = static_cast<const TW*>(op.tau);
        d.slots = sl;
        d.nslots = nl;
        d.c = op.c;
        d.w = w;
        d.k = op.kind == 2 ? op.k : 0;
        d.kind = op.kind;
        d.tr = op.c <= 32 ? 32 : 128;
        const int tc = tile_cols(d.tr);
        d.nrt = (op.c + d.tr - 1) / d.tr;
        d.nct = (ncol + tc - 1) / tc;
        d.tri = op.kind != 2;
        d.poff_f = pf;
        d.poff_t = pt;
        pf += (int64_t)d.nct * op.c;
        pt += (int64_t)d.nrt * ncol;
        const int di = (int)dense.size();
        for (int rt = 0; rt < d.nrt; ++rt)
          for (int ct = 0; ct < d.nct; ++ct)
            if (!d.tri || (int64_t)(ct + 1) * tc > (int64_t)rt * d.tr) tiles.push_back(make_int4(di, rt, ct, 0));
        for (int r = 0; r < op.c; r += kT) red_f.push_back(make_int2(di, r));
        for (int r = 0; r < ncol; r += kT) red_t.push_back(make_int2(di, r));
        for (int c2 = 0; c2 < ncol; ++c2) form_items.push_back(make_int2(di, c2));
        cmax = std::max(cmax, op.c);
        dense.push_back(d);
      }
    }
    sg.nsmall = (int)small.size() - sg.small0;
    sg.ntile = (int)tiles.size() - sg.tile0;
    sg.nrf = (int)red_f.size() - sg.rf0;
    sg.nrt = (int)red_t.size() - sg.rt0;
    part_max = std::max(part_max, (size_t)std::max(pf, pt));
    if (sg.nsmall || sg.ntile) segs.push_back(sg);
    i = j;
  }
  auto upload = [](auto& vec, auto** dst) {
    using E = typename std::remove_reference<decltype(vec)>::type::value_type;
    SPAQR_CUDA(dmalloc(reinterpret_cast<void**>(dst), std::max<size_t>(vec.size(), 1) * sizeof(E)));
    if (!vec.empty())
      SPAQR_CUDA(cudaMemcpy(*dst, vec.data(), vec.size() * sizeof(E), cudaMemcpyHostToDevice));
  };
  SmallOp<TW>* d_small = nullptr;
  DenseOp<TW>* d_dense = nullptr;
  upload(small, &d_small);
  upload(dense, &d_dense);
  P.d_small = d_small;
  P.d_dense = d_dense;
  upload(tiles, &P.d_tiles);
  std::vector<int2> red(red_f);
  const int rt_base = (int)red_f.size();
  red.insert(red.end(), red_t.begin(), red_t.end());
  for (auto& sg : segs) sg.rt0 += rt_base;
  upload(red, &P.d_red);
  SPAQR_CUDA(dmalloc(&P.d_dpart, std::max<size_t>(part_max, 1) * sizeof(TA)));
  if (!small.empty()) {
    recip_diag_kernel<TW><<<(unsigned)((small.size() + kW - 1) / kW), kT, 0, h.st>>>(d_small, (int)small.size());
    SPAQR_CUDA(cudaGetLastError());
  }
  if (!form_items.empty()) {
    // scratch: one FP64 column of length cmax per warp in flight
    const int64_t nit = (int64_t)form_items.size();
    const int grid = (int)std::min<int64_t>((nit + kW - 1) / kW, 1216);
    int2* d_items = nullptr;
    double* d_scr = nullptr;
    upload(form_items, &d_items);
    SPAQR_CUDA(dmalloc(&d_scr, (size_t)grid * kW * cmax * sizeof(double)));
    form_dense_kernel<TW><<<grid, kT, 0, h.st>>>(d_dense, d_items, nit, d_scr, cmax);
    SPAQR_CUDA(cudaGetLastError());
    SPAQR_CUDA(cudaStreamSynchronize(h.st));
    dfree(d_items);
    dfree(d_scr);
  }
  SPAQR_CUDA(cudaStreamSynchronize(h.st));
  P.segs = segs;
  P.launches = 0;
  for (auto& sg : segs) P.launches += (sg.nsmall > 0) + 2 * (sg.ntile > 0);
  set_dyn_smem(r_inv_warp_kernel<TW, TA>);
  set_dyn_smem(r_invT_warp_kernel<TW, TA>);
  set_dyn_smem(dense_T_kernel<TW, TA>);
  // persistent apply: segments on the device, a co-resident grid, and a probe
  // (one launch and one captured launch on a zero vector) before it is used
  P.pgrid = 0;
  if (h.opt.apply_persistent && !segs.empty()) {
    std::vector<SegDev> sd;
    for (auto& g : segs) sd.push_back(SegDev{g.kind, g.small0, g.nsmall, g.tile0, g.ntile, g.rf0, g.nrf, g.rt0, g.nrt});
    upload(sd, &P.d_segs);
    SPAQR_CUDA(dmalloc(&P.d_bar, 2 * sizeof(unsigned)));
    SPAQR_CUDA(cudaMemset(P.d_bar, 0, 2 * sizeof(unsigned)));
    SPAQR_CUDA(dmalloc(&P.d_err, sizeof(int)));
    SPAQR_CUDA(cudaMemset(P.d_err, 0, sizeof(int)));
    P.psmem = std::max(kWarpSmem<TW>, (size_t)kStage * sizeof(TW));
    set_dyn_smem(apply_persistent_kernel<TW, TA>);
    int dev = 0, sms = 0, per = 0;
    SPAQR_CUDA(cudaGetDevice(&dev));
    SPAQR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SPAQR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, apply_persistent_kernel<TW, TA>, kT, P.psmem));
    if (per > 0) {
      P.pgrid = sms * per;
      double* zt = nullptr;
      bool ok = dmalloc(&zt, (size_t)std::max<int64_t>(h.n, 1) * sizeof(double)) == cudaSuccess;
      if (ok) ok = cudaMemsetAsync(zt, 0, (size_t)std::max<int64_t>(h.n, 1) * sizeof(double), h.st) == cudaSuccess;
      if (ok) {
        const cudaError_t e0 = launch_persistent<TW, TA>(h, zt, 0);
        ok = e0 == cudaSuccess && cudaStreamSynchronize(h.st) == cudaSuccess;
      }
      if (ok) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        ok = cudaStreamBeginCapture(h.st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          const cudaError_t e1 = launch_persistent<TW, TA>(h, zt, 1);
          const bool launched = e1 == cudaSuccess;
          ok = cudaStreamEndCapture(h.st, &g) == cudaSuccess && launched;
        }
        if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (ok) ok = cudaGraphLaunch(ge, h.st) == cudaSuccess && cudaStreamSynchronize(h.st) == cudaSuccess;
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
      }
      int err = 0;
      if (ok) ok = cudaMemcpy(&err, P.d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && err == 0;
      if (zt) dfree(zt);
      if (!ok) {
        cudaGetLastError();
        P.pgrid = 0;  // per-segment launches
      }
    }
  }
  if (P.pgrid > 0) P.launches = 1;
}

void build_apply_plan(Handle& h) {
  free_apply_plan(h);
  h.plan = new ApplyPlan();
  h.plan->fp32 = h.precision == SPAQR_PREC_MIXED;
  if (h.plan->fp32)
    build_plan_t<float, float>(h, *h.plan);
  else
    build_plan_t<double, double>(h, *h.plan);
  for (auto& e : h.plan->ev) SPAQR_CUDA(cudaEventCreate(&e));
  // algorithmic bytes of one W^{-1} plus one W^{-T} apply: every stored entry
  // once per direction, the slot indices, and the slot-vector reads/writes
  {
    const double es = h.plan->fp32 ? 4.0 : 8.0;
    double b = 0.0;
    for (auto& op : h.ops) {
      if (op.kind == 2 && op.k <= 0) continue;
      const double c = op.c, w = op.kind == 0 ? op.w : 0, k = op.k;
      double stored = 0.0;
      if (op.kind == 0)
        stored = c * (c + 1) / 2 + c * w;
      else if (op.kind == 1)
        stored = c * (c + 1) / 2;
      else
        stored = c * k - k * (k - 1) / 2 + k;
      b += 2 * es * stored + 2 * 4.0 * (c + w);
      b += 8.0 * (c + w + c);      // W^{-1}: read z_s, z_n; write z_s
      b += 8.0 * (2 * c + 2 * w);  // W^{-T}: read/write z_s, read/write z_n
    }
    h.stats.bytes_apply = b;
  }
  const int64_t big = std::max(h.m, h.n);
  h.plan->part_n = blocks(big);
  SPAQR_CUDA(dmalloc(&h.plan->d_scal, 8 * sizeof(double)));
  SPAQR_CUDA(cudaMallocHost(&h.plan->h_res, sizeof(double)));
  SPAQR_CUDA(dmalloc(&h.plan->d_part, (size_t)h.plan->part_n * sizeof(double)));
}

void free_apply_plan(Handle& h) {
  if (!h.plan) return;
  for (auto& e : h.plan->ev)
    if (e) cudaEventDestroy(e);
  if (h.plan->graph) cudaGraphExecDestroy(h.plan->graph);
  if (h.plan->graph_pcg) cudaGraphExecDestroy(h.plan->graph_pcg);
  if (h.plan->graph_csne) cudaGraphExecDestroy(h.plan->graph_csne);
  if (h.plan->h_res) cudaFreeHost(h.plan->h_res);
  dfree(h.plan->d_segs);
  dfree(h.plan->d_bar);
  dfree(h.plan->d_err);
  dfree(h.plan->d_small);
  dfree(h.plan->d_dense);
  dfree(h.plan->d_idx);
  dfree(h.plan->d_tiles);
  dfree(h.plan->d_red);
  dfree(h.plan->d_dpart);
  dfree(h.plan->d_rdiag);
  dfree(h.plan->d_scal);
  dfree(h.plan->d_part);
  delete h.plan;
  h.plan = nullptr;
}

// The launches of one segment of W^{-1} (transpose = 0) or W^{-T}.
template <typename TW, typename TA>
static void run_segment(Handle& h, const Segment& s, double* z, int transpose) {
  ApplyPlan& P = *h.plan;
  if (s.nsmall) {
    const SmallOp<TW>* ops = static_cast<const SmallOp<TW>*>(P.d_small) + s.small0;
    const int grid = (s.nsmall + kW - 1) / kW;
    if (s.kind == 2)
      q_warp_kernel<TW, TA><<<grid, kT, 0, h.st>>>(ops, s.nsmall, z, transpose);
    else if (transpose)
      r_invT_warp_kernel<TW, TA><<<grid, kT, kWarpSmem<TW>, h.st>>>(ops, s.nsmall, z);
    else
      r_inv_warp_kernel<TW, TA><<<grid, kT, kWarpSmem<TW>, h.st>>>(ops, s.nsmall, z);
  }
  if (s.ntile) {
    const DenseOp<TW>* d = static_cast<const DenseOp<TW>*>(P.d_dense);
    TA* part = static_cast<TA*>(P.d_dpart);
    if (transpose) {
      dense_T_kernel<TW, TA><<<s.ntile, kT, kStage * sizeof(TW), h.st>>>(d, P.d_tiles + s.tile0, z, part);
      dense_T_reduce_kernel<TW, TA><<<s.nrt, kT, 0, h.st>>>(d, P.d_red + s.rt0, part, z);
    } else {
      dense_fwd_kernel<TW, TA><<<s.ntile, kT, 0, h.st>>>(d, P.d_tiles + s.tile0, z, part);
      dense_fwd_reduce_kernel<TW, TA><<<s.nrf, kT, 0, h.st>>>(d, P.d_red + s.rf0, part, z);
    }
  }
}

template <typename TW, typename TA>
static void apply_t(Handle& h, double* z, int transpose) {
  ApplyPlan& P = *h.plan;
  if (P.pgrid > 0) {
    const cudaError_t e = launch_persistent<TW, TA>(h, z, transpose);
    SPAQR_CUDA(e);
    return;
  }
  const int nseg = (int)P.segs.size();
  for (int t = 0; t < nseg; ++t) run_segment<TW, TA>(h, P.segs[(size_t)(transpose ? t : nseg - 1 - t)], z, transpose);
  SPAQR_CUDA(cudaGetLastError());
}

// Diagnostic (SPAQR_PROFILE_APPLY=1): one W^{-1} and one W^{-T} with CUDA events
// around every segment, printed to stderr as stage/kind/ops/microseconds.
template <typename TW, typename TA>
static void profile_apply_t(Handle& h, double* z) {
  ApplyPlan& P = *h.plan;
  const int nseg = (int)P.segs.size();
  std::vector<cudaEvent_t> ev(2 * (size_t)nseg + 2);
  for (auto& e : ev) SPAQR_CUDA(cudaEventCreate(&e));
  for (int transpose = 0; transpose < 2; ++transpose) {
    for (int t = 0; t < nseg; ++t) {
      const int si = transpose ? t : nseg - 1 - t;
      SPAQR_CUDA(cudaEventRecord(ev[2 * (size_t)t], h.st));
      run_segment<TW, TA>(h, P.segs[(size_t)si], z, transpose);
      SPAQR_CUDA(cudaEventRecord(ev[2 * (size_t)t + 1], h.st));
    }
    SPAQR_CUDA(cudaStreamSynchronize(h.st));
    double tot = 0.0;
    for (int t = 0; t < nseg; ++t) {
      const int si = transpose ? t : nseg - 1 - t;
      const Segment& s = P.segs[(size_t)si];
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * (size_t)t], ev[2 * (size_t)t + 1]);
      tot += ms;
      if (ms > 0.05f)
        std::fprintf(stderr, "[spaqr] apply %s seg %3d kind %d small %6d tiles %6d: %8.1f us\n",
                     transpose ? "W^-T" : "W^-1", si, s.kind, s.nsmall, s.ntile, ms * 1e3);
    }
    std::fprintf(stderr, "[spaqr] apply %s total %.3f ms over %d segments\n", transpose ? "W^-T" : "W^-1", tot, nseg);
  }
  for (auto& e : ev) cudaEventDestroy(e);
}

void profile_apply(Handle& h, double* z) {
  if (h.plan->fp32)
    profile_apply_t<float, float>(h, z);
  else
    profile_apply_t<double, double>(h, z);
}

void apply_Winv(Handle& h, double* z, int transpose) {
  if (!h.plan) throw Error(SPAQR_ERR_INVALID_ARG, "no factorization");
  if (h.plan->fp32)
    apply_t<float, float>(h, z, transpose);
  else
    apply_t<double, double>(h, z, transpose);
}

void apply_A(Handle& h, const double* x, double* y, int forward) {
  ApplyPlan& P = *h.plan;
  if (forward)
    spmv_kernel<<<blocks(h.m), kT, 0, h.st>>>(h.m, h.d_rowptr, h.d_colidx, h.d_vals, x, y, nullptr, P.d_part);
  else
    spmv_kernel<<<blocks(h.n), kT, 0, h.st>>>(h.n, h.d_trowptr, h.d_tcolidx, h.d_tvals, x, y, nullptr, P.d_part);
  SPAQR_CUDA(cudaGetLastError());
}

// One CGLS iteration (everything on the stream, no host wait).  Events
// ev[0..3] bracket the two W applies, ev[4..7] the two SpMVs.
static void cgls_body(Handle& h, double* x, double* r, double* p, double* t, double* q, double* u, double* s,
                      const double* Dv, bool capturing) {
  ApplyPlan& P = *h.plan;
  // inside a stream capture an event record must be an external record node
  auto rec = [&](cudaEvent_t e) {
    SPAQR_CUDA(capturing ? cudaEventRecordWithFlags(e, h.st, cudaEventRecordExternal) : cudaEventRecord(e, h.st));
  };
  const int64_t m = h.m, n = h.n;
  SPAQR_CUDA(cudaMemcpyAsync(t, p, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h.st));
  rec(P.ev[0]);
  apply_Winv(h, t, 0);
  rec(P.ev[1]);
  rec(P.ev[4]);
  spmv_kernel<<<blocks(m), kT, 0, h.st>>>(m, h.d_rowptr, h.d_colidx, h.d_vals, t, q, nullptr, P.d_part);
  rec(P.ev[5]);
  finish_sum_kernel<<<1, kT, 0, h.st>>>(blocks(m), P.d_part, P.d_scal + 1);
  update_xr_kernel<<<blocks(std::max(m, n)), kT, 0, h.st>>>(n, m, x, t, r, q, P.d_scal);
  rec(P.ev[6]);
  spmv_kernel<<<blocks(n), kT, 0, h.st>>>(n, h.d_trowptr, h.d_tcolidx, h.d_tvals, r, u, Dv, P.d_part);
  rec(P.ev[7]);
  finish_sum_kernel<<<1, kT, 0, h.st>>>(blocks(n), P.d_part, P.d_scal + 2);
  SPAQR_CUDA(cudaMemcpyAsync(s, u, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h.st));
  rec(P.ev[2]);
  apply_Winv(h, s, 1);
  rec(P.ev[3]);
  sumsq_kernel<<<std::min(blocks(n), P.part_n), kT, 0, h.st>>>(n, s, P.d_part);
  finish_sum_kernel<<<1, kT, 0, h.st>>>(std::min(blocks(n), P.part_n), P.d_part, P.d_scal + 3);
  beta_kernel<<<1, 1, 0, h.st>>>(P.d_scal);
  update_p_kernel<<<blocks(n), kT, 0, h.st>>>(n, p, s, P.d_scal);
  SPAQR_CUDA(cudaGetLastError());
}

static void accumulate_solve_timers(Handle& h) {
  ApplyPlan& P = *h.plan;
  float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
  if (cudaEventElapsedTime(&a, P.ev[0], P.ev[1]) == cudaSuccess &&
      cudaEventElapsedTime(&b, P.ev[2], P.ev[3]) == cudaSuccess &&
      cudaEventElapsedTime(&c, P.ev[4], P.ev[5]) == cudaSuccess &&
      cudaEventElapsedTime(&d, P.ev[6], P.ev[7]) == cudaSuccess) {
    h.stats.t_kernel[4] += (a + b) * 1e-3;
    h.stats.n_kernel[4] += 2 * P.launches;
    h.stats.t_kernel[5] += (c + d) * 1e-3;
    h.stats.n_kernel[5] += 2;
  } else {
    cudaGetLastError();
  }
}

// One PCG iteration on A~^T A~ nu = D g with the preconditioner W^{-1} W^{-T}
// (everything on the stream, no host wait).  scal[0] = rho = r.z, scal[1] = p.q,
// scal[2] = |D^{-1} r|^2 (the residual of (A^T A) lambda = g), scal[3] = new rho.
static void pcg_body(Handle& h, double* nu, double* r, double* z, double* p, double* q, double* t) {
  ApplyPlan& P = *h.plan;
  const int64_t m = h.m, n = h.n;
  const int nb = std::min(blocks(n), P.part_n);
  spmv_kernel<<<blocks(m), kT, 0, h.st>>>(m, h.d_rowptr, h.d_colidx, h.d_vals, p, t, nullptr, P.d_part);
  spmv_kernel<<<blocks(n), kT, 0, h.st>>>(n, h.d_trowptr, h.d_tcolidx, h.d_tvals, t, q, nullptr, P.d_part);
  dot_kernel<<<nb, kT, 0, h.st>>>(n, p, q, nullptr, P.d_part);
  finish_sum_kernel<<<1, kT, 0, h.st>>>(nb, P.d_part, P.d_scal + 1);
  update_xr_kernel<<<blocks(n), kT, 0, h.st>>>(n, n, nu, p, r, q, P.d_scal);
  dot_kernel<<<nb, kT, 0, h.st>>>(n, r, r, h.d_D, P.d_part);
  finish_sum_kernel<<<1, kT, 0, h.st>>>(nb, P.d_part, P.d_scal + 2);
  SPAQR_CUDA(cudaMemcpyAsync(z, r, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h.st));
  apply_Winv(h, z, 1);
  apply_Winv(h, z, 0);
  dot_kernel<<<nb, kT, 0, h.st>>>(n, r, z, nullptr, P.d_part);
  finish_sum_kernel<<<1, kT, 0, h.st>>>(nb, P.d_part, P.d_scal + 3);
  beta_kernel<<<1, 1, 0, h.st>>>(P.d_scal);
  update_p_kernel<<<blocks(n), kT, 0, h.st>>>(n, p, z, P.d_scal);
  SPAQR_CUDA(cudaGetLastError());
}

// One refinement step of the corrected seminormal equations (Section 1: the
// factor gives W^T W ~= A~^T A~): s = W^{-1} W^{-T} u with u = A~^T r,
// x <- x + s, r <- r - A~ s, u <- A~^T r and scal[2] = |D^{-1} u|^2, the
// unscaled normal-equation residual of the stopping test.  No host wait.
static void csne_body(Handle& h, double* x, double* r, double* q, double* u, double* s, const double* Dv) {
  ApplyPlan& P = *h.plan;
  const int64_t m = h.m, n = h.n;
  SPAQR_CUDA(cudaMemcpyAsync(s, u, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h.st));
  apply_Winv(h, s, 1);
  apply_Winv(h, s, 0);
  spmv_kernel<<<blocks(m), kT, 0, h.st>>>(m, h.d_rowptr, h.d_colidx, h.d_vals, s, q, nullptr, P.d_part);
  csne_update_kernel<<<blocks(std::max(m, n)), kT, 0, h.st>>>(n, m, x, s, r, q);
  spmv_kernel<<<blocks(n), kT, 0, h.st>>>(n, h.d_trowptr, h.d_tcolidx, h.d_tvals, r, u, Dv, P.d_part);
  finish_sum_kernel<<<1, kT, 0, h.st>>>(blocks(n), P.d_part, P.d_scal + 2);
  SPAQR_CUDA(cudaGetLastError());
}

// Workspace of the iterative solvers: CGLS r, q (m) and x, p, t, u, s (n);
// PCG nu, r, z, p, q (n) and t (m).
static void ensure_work(Handle& h) {
  ApplyPlan& P = *h.plan;
  const size_t need = (size_t)3 * h.m + (size_t)5 * h.n;
  if (h.work_elems >= need) return;
  if (h.d_work) cudaFree(h.d_work);
  h.d_work = nullptr;
  SPAQR_CUDA(cudaMalloc(&h.d_work, need * sizeof(double)));
  h.work_elems = need;
  if (P.graph) cudaGraphExecDestroy(P.graph);
  if (P.graph_pcg) cudaGraphExecDestroy(P.graph_pcg);
  if (P.graph_csne) cudaGraphExecDestroy(P.graph_csne);
  P.graph = P.graph_pcg = P.graph_csne = nullptr;
}

void IterSolve::begin() {
  Handle& hh = *h;
  ApplyPlan& P = *hh.plan;
  t0 = std::chrono::steady_clock::now();
  ensure_work(hh);
  const int64_t m = hh.m, n = hh.n;
  double* w = hh.d_work;
  it = 0;
  done = false;
  if (kind == 2) {
    // CSNE: x = 0, r = b, u = A~^T r, res0 = |D^{-1} A~^T b|
    double* r = w;
    double* xt = w + 2 * m;
    double* u = xt + 3 * n;
    SPAQR_CUDA(cudaMemsetAsync(xt, 0, (size_t)n * sizeof(double), hh.st));
    SPAQR_CUDA(cudaMemcpyAsync(r, rhs, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, hh.st));
    spmv_kernel<<<blocks(n), kT, 0, hh.st>>>(n, hh.d_trowptr, hh.d_tcolidx, hh.d_tvals, r, u, hh.d_D, P.d_part);
    finish_sum_kernel<<<1, kT, 0, hh.st>>>(blocks(n), P.d_part, P.d_scal + 2);
  } else if (kind == 0) {
    // CGLS: x = 0, r = b, s = W^{-T} (A~^T r), p = s, gamma = |s|^2, res0 = |D^{-1} A~^T b|
    double* r = w;
    double* xt = w + 2 * m;
    double* p = xt + n;
    double* u = p + 2 * n;
    double* sv = u + n;
    const char* e = std::getenv("SPAQR_PROFILE_APPLY");
    if (e && e[0] == '1') {
      SPAQR_CUDA(cudaMemsetAsync(p + n, 0, (size_t)n * sizeof(double), hh.st));
      profile_apply(hh, p + n);
    }
    SPAQR_CUDA(cudaMemsetAsync(xt, 0, (size_t)n * sizeof(double), hh.st));
    SPAQR_CUDA(cudaMemcpyAsync(r, rhs, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, hh.st));
    spmv_kernel<<<blocks(n), kT, 0, hh.st>>>(n, hh.d_trowptr, hh.d_tcolidx, hh.d_tvals, r, u, hh.d_D, P.d_part);
    finish_sum_kernel<<<1, kT, 0, hh.st>>>(blocks(n), P.d_part, P.d_scal + 2);
    SPAQR_CUDA(cudaMemcpyAsync(sv, u, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, hh.st));
    apply_Winv(hh, sv, 1);
    SPAQR_CUDA(cudaMemcpyAsync(p, sv, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, hh.st));
    sumsq_kernel<<<std::min(blocks(n), P.part_n), kT, 0, hh.st>>>(n, sv, P.d_part);
    finish_sum_kernel<<<1, kT, 0, hh.st>>>(std::min(blocks(n), P.part_n), P.d_part, P.d_scal + 0);
  } else {
    // PCG: nu = 0, r = D g, z = W^{-1} W^{-T} r, p = z, rho = r.z, res0 = |g|
    double* nu = w;
    double* r = nu + n;
    double* z = r + n;
    double* p = z + n;
    const int nb = std::min(blocks(n), P.part_n);
    SPAQR_CUDA(cudaMemsetAsync(nu, 0, (size_t)n * sizeof(double), hh.st));
    scale_kernel<<<blocks(n), kT, 0, hh.st>>>(n, rhs, hh.d_D, r);
    dot_kernel<<<nb, kT, 0, hh.st>>>(n, r, r, hh.d_D, P.d_part);
    finish_sum_kernel<<<1, kT, 0, hh.st>>>(nb, P.d_part, P.d_scal + 2);
    SPAQR_CUDA(cudaMemcpyAsync(z, r, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, hh.st));
    apply_Winv(hh, z, 1);
    apply_Winv(hh, z, 0);
    SPAQR_CUDA(cudaMemcpyAsync(p, z, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, hh.st));
    dot_kernel<<<nb, kT, 0, hh.st>>>(n, r, z, nullptr, P.d_part);
    finish_sum_kernel<<<1, kT, 0, hh.st>>>(nb, P.d_part, P.d_scal + 0);
  }
  SPAQR_CUDA(cudaMemcpyAsync(P.h_res, P.d_scal + 2, sizeof(double), cudaMemcpyDeviceToHost, hh.st));
}

void IterSolve::begun() {
  norm0 = std::sqrt(*h->plan->h_res);
  if (!std::isfinite(norm0))
    throw Error(SPAQR_ERR_INVALID_ARG, kind == 0 ? "right-hand side b has non-finite entries (||A^T b|| is not finite)"
                                                 : "right-hand side g has non-finite entries");
  rel = norm0 > 0.0 ? 1.0 : 0.0;
  done = !(norm0 > 0.0);
  if (kind != 1) {
    h->stats.t_kernel[4] = h->stats.t_kernel[5] = 0.0;
    h->stats.n_kernel[4] = h->stats.n_kernel[5] = 0;
  }
}

void IterSolve::step() {
  Handle& hh = *h;
  ApplyPlan& P = *hh.plan;
  const int64_t m = hh.m, n = hh.n;
  double* w = hh.d_work;
  const bool graphs = hh.opt.use_graphs != 0;
  cudaGraphExec_t* g = kind == 0 ? &P.graph : (kind == 1 ? &P.graph_pcg : &P.graph_csne);
  auto body = [&](bool capturing) {
    if (kind == 2) {
      double* r = w;
      double* q = r + m;
      double* xt = q + m;
      double* u = xt + 3 * n;
      double* sv = u + n;
      csne_body(hh, xt, r, q, u, sv, hh.d_D);
    } else if (kind == 0) {
      double* r = w;
      double* q = r + m;
      double* xt = q + m;
      double* p = xt + n;
      double* t = p + n;
      double* u = t + n;
      double* sv = u + n;
      cgls_body(hh, xt, r, p, t, q, u, sv, hh.d_D, capturing);
    } else {
      double* nu = w;
      double* r = nu + n;
      double* z = r + n;
      double* p = z + n;
      double* q = p + n;
      double* t = q + n;
      pcg_body(hh, nu, r, z, p, q, t);
    }
  };
  if (graphs && !*g) {
    cudaGraph_t gr;
    SPAQR_CUDA(cudaStreamBeginCapture(hh.st, cudaStreamCaptureModeThreadLocal));
    body(true);
    SPAQR_CUDA(cudaStreamEndCapture(hh.st, &gr));
    SPAQR_CUDA(cudaGraphInstantiate(g, gr, 0));
    cudaGraphDestroy(gr);
  }
  if (graphs)
    SPAQR_CUDA(cudaGraphLaunch(*g, hh.st));
  else
    body(false);
  SPAQR_CUDA(cudaMemcpyAsync(P.h_res, P.d_scal + 2, sizeof(double), cudaMemcpyDeviceToHost, hh.st));
}

void IterSolve::stepped() {
  ++it;
  if (kind == 0) accumulate_solve_timers(*h);
  rel = std::sqrt(*h->plan->h_res) / norm0;
  if (!(rel >= tol) || it >= maxit) done = true;
}

void IterSolve::finish() {
  Handle& hh = *h;
  const int64_t m = hh.m, n = hh.n;
  const double* sol = kind != 1 ? hh.d_work + 2 * m : hh.d_work;  // x~ (CGLS, CSNE) or nu (PCG)
  scale_kernel<<<blocks(n), kT, 0, hh.st>>>(n, sol, hh.d_D, out);
  SPAQR_CUDA(cudaGetLastError());
}

void IterSolve::report(spaqr_solve_info* info) {
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (kind != 1) {
    h->stats.t_solve = secs;
    h->stats.iters = it;
  }
  if (info) {
    info->iters = it;
    info->rel_resid = rel;
    info->converged = rel < tol;
    info->seconds = secs;
  }
}

// Runs the solvers of several handles side by side: every round launches one
// iteration on each unfinished handle's stream, then reads their residuals.
void run_iterative(std::vector<IterSolve>& S) {
  for (auto& s : S) s.begin();
  for (auto& s : S) {
    SPAQR_CUDA(cudaStreamSynchronize(s.h->st));
    s.begun();
  }
  for (;;) {
    bool any = false;
    for (auto& s : S)
      if (!s.done) {
        s.step();
        any = true;
      }
    if (!any) break;
    for (auto& s : S)
      if (!s.done) {
        SPAQR_CUDA(cudaStreamSynchronize(s.h->st));
        s.stepped();
      }
  }
  for (auto& s : S) s.finish();
  for (auto& s : S) SPAQR_CUDA(cudaStreamSynchronize(s.h->st));
  for (auto& s : S) {
    ApplyPlan& P = *s.h->plan;
    int err = 0;
    if (P.d_err) {
      SPAQR_CUDA(cudaMemcpy(&err, P.d_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (err) {
        SPAQR_CUDA(cudaMemset(P.d_err, 0, sizeof(int)));
        SPAQR_CUDA(cudaMemset(P.d_bar, 0, 2 * sizeof(unsigned)));
        throw Error(SPAQR_ERR_TIMEOUT, "persistent apply: a grid barrier wait timed out");
      }
    }
  }
}

void cgls(Handle& h, const double* b_dev, double* x_dev, spaqr_solve_info* info) {
  std::vector<IterSolve> S(1);
  S[0].h = &h;
  S[0].kind = 0;
  S[0].rhs = b_dev;
  S[0].out = x_dev;
  S[0].tol = h.opt.tol;
  S[0].maxit = h.opt.maxit;
  run_iterative(S);
  S[0].report(info);
}

void csne(Handle& h, const double* b_dev, double* x_dev, spaqr_solve_info* info) {
  std::vector<IterSolve> S(1);
  S[0].h = &h;
  S[0].kind = 2;
  S[0].rhs = b_dev;
  S[0].out = x_dev;
  S[0].tol = h.opt.tol;
  S[0].maxit = h.opt.maxit;
  run_iterative(S);
  S[0].report(info);
}

void lstsq_grad(Handle& h, const double* b, const double* x, const double* lam, double* gb, double* gv) {
  lstsq_grad_kernel<<<blocks(h.m), kT, 0, h.st>>>(h.m, h.d_rowptr, h.d_colidx, h.d_vals, h.d_D, b, x, lam, gb, gv);
  SPAQR_CUDA(cudaGetLastError());
}

void set_values(Handle& h, const double* a_dev) {
  set_values_kernel<<<blocks(h.nnz), kT, 0, h.st>>>(h.nnz, a_dev, h.d_colidx, h.d_D, h.d_vals);
  gather_values_kernel<<<blocks(h.nnz), kT, 0, h.st>>>(h.nnz, h.d_vals, h.d_tperm, h.d_tvals);
  SPAQR_CUDA(cudaGetLastError());
}

}  // namespace spaqr
