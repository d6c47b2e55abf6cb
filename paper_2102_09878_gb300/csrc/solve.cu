// Apply of the stored factor W and the W-preconditioned CGLS (Section 4).
//
// W = W_1 ... W_L with W_l = (prod Q_p^T)(prod R_p)(prod R_s) for the
// operations of stage l (Section 2.7).  W^{-1} z replays the operations in
// reverse factorization order, W^{-T} z in factorization order.  Operations
// of one elimination round, of one scaling phase and of one step-2 phase act
// on disjoint slots and run as one batched launch each ("segment").  Every
// vector is FP64; the stored factor is FP64 or FP32 (mixed precision).
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

template <typename TW>
constexpr size_t kWarpSmem = (size_t)kW * 32 * 33 * sizeof(TW);  // staged R_ss per warp

template <typename TW>
struct ApplyOp {
  const TW* R;  // kind 0: c x (c + w) = [R_ss R_sn]; kind 1: c x c
  const TW* Qx; // kind 2, c > 32: explicit Q_pp (c x c, ld c)
  const TW* V;
  const TW* tau;
  const int* kdev;
  const int32_t* slots;
  const int32_t* nslots;
  const double* rdiag;  // kinds 0, 1: 1 / R_ii (FP64), computed once when the plan is built
  int c, w;
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Back substitution R y = rhs (R upper, ld c) on a shared vector y of length c,
// blocked by 32 rows: the 32 x 32 diagonal block is staged in shared memory
// (blk, 33 x 32 doubles) with parallel loads, warp 0 solves it with shuffles
// and the precomputed reciprocals, then all threads update the rows above.
template <typename TW>
__device__ void upper_solve(const TW* R, const double* rdiag, int c, double* y, double* blk) {
  const int lane = threadIdx.x & 31;
  for (int hi = c; hi > 0; hi -= 32) {
    const int lo = hi > 32 ? hi - 32 : 0;
    const int bs = hi - lo;
    __syncthreads();
    for (int e = threadIdx.x; e < bs * bs; e += kT) {
      const int r = e % bs, q = e / bs;  // coalesced over rows
      blk[r * 33 + q] = (double)R[(lo + r) + (int64_t)(lo + q) * c];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int r = lane;
      double x = r < bs ? y[lo + r] : 0.0;
      const double rd = r < bs ? rdiag[lo + r] : 0.0;
      for (int q = bs - 1; q >= 0; --q) {
        const double yq = __shfl_sync(0xffffffffu, x, q) * __shfl_sync(0xffffffffu, rd, q);
        if (r == q) x = yq;
        if (r < q) x -= blk[r * 33 + q] * yq;
      }
      if (r < bs) y[lo + r] = x;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < lo; i += kT) {
      double a0 = 0.0, a1 = 0.0;
      int j = lo;
      for (; j + 1 < hi; j += 2) {
        a0 += (double)R[i + (int64_t)j * c] * y[j];
        a1 += (double)R[i + (int64_t)(j + 1) * c] * y[j + 1];
      }
      if (j < hi) a0 += (double)R[i + (int64_t)j * c] * y[j];
      y[i] -= a0 + a1;
    }
  }
  __syncthreads();
}

// Forward substitution R^T y = rhs, blocked the same way.
template <typename TW>
__device__ void lower_t_solve(const TW* R, const double* rdiag, int c, double* y, double* blk) {
  const int lane = threadIdx.x & 31;
  for (int lo = 0; lo < c; lo += 32) {
    const int hi = lo + 32 < c ? lo + 32 : c;
    const int bs = hi - lo;
    __syncthreads();
    for (int e = threadIdx.x; e < bs * bs; e += kT) {
      const int r = e % bs, q = e / bs;
      blk[r * 33 + q] = (double)R[(lo + r) + (int64_t)(lo + q) * c];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int r = lane;
      double x = r < bs ? y[lo + r] : 0.0;
      const double rd = r < bs ? rdiag[lo + r] : 0.0;
      for (int q = 0; q < bs; ++q) {
        const double yq = __shfl_sync(0xffffffffu, x, q) * __shfl_sync(0xffffffffu, rd, q);
        if (r == q) x = yq;
        if (r > q && r < bs) x -= blk[q * 33 + r] * yq;
      }
      if (r < bs) y[lo + r] = x;
    }
    __syncthreads();
    for (int i = hi + threadIdx.x; i < c; i += kT) {
      const TW* col = R + (int64_t)i * c;
      double a0 = 0.0, a1 = 0.0;
      int j = lo;
      for (; j + 1 < hi; j += 2) {
        a0 += (double)col[j] * y[j];
        a1 += (double)col[j + 1] * y[j + 1];
      }
      if (j < hi) a0 += (double)col[j] * y[j];
      y[i] -= a0 + a1;
    }
  }
  __syncthreads();
}

// W^{-1}: z_s <- R_ss^{-1} (z_s - R_sn z_n)  (kind 0) or z_p <- R_pp^{-1} z_p (kind 1)
template <typename TW>
__global__ void __launch_bounds__(kT) r_inv_kernel(const ApplyOp<TW>* ops, const int* ids, double* z) {
  const ApplyOp<TW> op = ops[ids[blockIdx.x]];
  extern __shared__ double sh[];
  double* y = sh;          // c
  double* part = sh + op.c;  // kW * c partials
  __shared__ double blk[33 * 32];
  const int c = op.c, w = op.w;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kW * c; i += kT) part[i] = 0.0;
  __syncthreads();
  if (w > 0) {
    const TW* Rn = op.R + (int64_t)c * c;
    for (int i0 = 0; i0 < c; i0 += 32) {
      const int i = i0 + lane;
      double acc = 0.0;
      for (int j = warp; j < w; j += kW) {
        const double zj = z[op.nslots[j]];
        if (i < c) acc += (double)Rn[i + (int64_t)j * c] * zj;
      }
      if (i < c) part[warp * c + i] = acc;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < c; i += kT) {
    double s = z[op.slots[i]];
    for (int q = 0; q < kW; ++q) s -= part[q * c + i];
    y[i] = s;
  }
  upper_solve(op.R, op.rdiag, c, y, blk);
  for (int i = threadIdx.x; i < c; i += kT) z[op.slots[i]] = y[i];
}

// W^{-T}: y = R_ss^{-T} z_s, z_s <- y, z_n -= R_sn^T y (kind 0); z_p <- R_pp^{-T} z_p (kind 1)
template <typename TW>
__global__ void __launch_bounds__(kT) r_invT_kernel(const ApplyOp<TW>* ops, const int* ids, double* z) {
  const ApplyOp<TW> op = ops[ids[blockIdx.x]];
  extern __shared__ double sh[];
  double* y = sh;
  __shared__ double blk[33 * 32];
  const int c = op.c, w = op.w;
  for (int i = threadIdx.x; i < c; i += kT) y[i] = z[op.slots[i]];
  lower_t_solve(op.R, op.rdiag, c, y, blk);
  for (int i = threadIdx.x; i < c; i += kT) z[op.slots[i]] = y[i];
  if (w > 0) {
    const TW* Rn = op.R + (int64_t)c * c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < w; j += kW) {
      const TW* col = Rn + (int64_t)j * c;
      double s = 0.0;
      for (int i = lane; i < c; i += 32) s += (double)col[i] * y[i];
      s = wsum(s);
      if (lane == 0) atomicAdd(&z[op.nslots[j]], -s);
    }
  }
}

// Large Q_p ops use the explicit Q_pp formed after the factorization:
// W^{-1}: z_p <- Q_pp z_p;  W^{-T}: z_p <- Q_pp^T z_p  (one coalesced GEMV each).
template <typename TW>
__global__ void __launch_bounds__(kT) q_kernel(const ApplyOp<TW>* ops, const int* ids, double* z, int transpose) {
  const ApplyOp<TW> op = ops[ids[blockIdx.x]];
  extern __shared__ double sh[];
  double* x = sh;
  const int c = op.c;
  for (int i = threadIdx.x; i < c; i += kT) x[i] = z[op.slots[i]];
  __syncthreads();
  if (!transpose) {
    // y_i = sum_j Q[i, j] x_j: thread per row, columns in order (coalesced over i)
    for (int i0 = 0; i0 < c; i0 += kT) {
      const int i = i0 + threadIdx.x;
      if (i >= c) continue;
      double acc = 0.0;
      for (int j = 0; j < c; ++j) acc += (double)op.Qx[i + (int64_t)j * c] * x[j];
      z[op.slots[i]] = acc;
    }
  } else {
    // y_j = sum_i Q[i, j] x_i: warp per column, lanes over i (coalesced)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < c; j += kW) {
      const TW* col = op.Qx + (int64_t)j * c;
      double acc = 0.0;
      for (int i = lane; i < c; i += 32) acc += (double)col[i] * x[i];
      acc = wsum(acc);
      if (lane == 0) z[op.slots[j]] = acc;
    }
  }
}

// 1 / R_ii for every triangular op (one warp per op).
template <typename TW>
__global__ void __launch_bounds__(kT) recip_diag_kernel(const ApplyOp<TW>* ops, int nops) {
  const int gw = (int)((blockIdx.x * (unsigned)kT + threadIdx.x) >> 5);
  if (gw >= nops) return;
  const ApplyOp<TW> op = ops[gw];
  if (!op.rdiag) return;
  double* rd = const_cast<double*>(op.rdiag);
  for (int i = threadIdx.x & 31; i < op.c; i += 32) rd[i] = 1.0 / (double)op.R[i + (int64_t)i * op.c];
}

// Q = H_1 ... H_k applied to the identity, 32 columns per CTA (one warp per
// column at a time, the column held in shared memory).
template <typename TW>
__global__ void __launch_bounds__(kT) form_q_kernel(const ApplyOp<TW>* ops, const int* ids, TW* const* outs) {
  const ApplyOp<TW> op = ops[ids[blockIdx.y]];
  TW* Q = outs[blockIdx.y];
  const int c = op.c;
  const int k = *op.kdev;
  extern __shared__ double sh[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* y = sh + (size_t)warp * c;
  for (int jj = warp; jj < 32; jj += kW) {
    const int j = blockIdx.x * 32 + jj;
    if (j >= c) break;
    for (int i = lane; i < c; i += 32) y[i] = (i == j) ? 1.0 : 0.0;
    __syncwarp();
    for (int t = k - 1; t >= 0; --t) {  // Q e_j = H_1 (H_2 (... H_k e_j))
      const TW* v = op.V + (int64_t)t * c;
      double d = 0.0;
      for (int i = t + lane; i < c; i += 32) d += (i == t ? 1.0 : (double)v[i]) * y[i];
      d = wsum(d) * (double)op.tau[t];
      for (int i = t + lane; i < c; i += 32) y[i] -= d * (i == t ? 1.0 : (double)v[i]);
      __syncwarp();
    }
    for (int i = lane; i < c; i += 32) Q[i + (int64_t)j * c] = (TW)y[i];
    __syncwarp();
  }
}

// ------------------------------------------- warp-per-op kernels (c <= 32)
// One warp applies one stored op; lane i holds z_slots[i].  The triangular
// solves run by shuffles (no block barriers).
template <typename TW>
__global__ void __launch_bounds__(kT) r_inv_warp_kernel(const ApplyOp<TW>* ops, const int* ids, int count,
                                                        double* z) {
  const int gw = (int)((blockIdx.x * (unsigned)kT + threadIdx.x) >> 5);
  if (gw >= count) return;
  const ApplyOp<TW> op = ops[ids[gw]];
  const int lane = threadIdx.x & 31, c = op.c, w = op.w;
  double x = lane < c ? z[op.slots[lane]] : 0.0;
  if (w > 0) {
    const TW* Rn = op.R + (int64_t)c * c;
    double acc = 0.0;
    for (int j0 = 0; j0 < w; j0 += 32) {
      const double zl = (j0 + lane < w) ? z[op.nslots[j0 + lane]] : 0.0;
      const int jn = min(32, w - j0);
      for (int t = 0; t < jn; ++t) {
        const double zj = __shfl_sync(0xffffffffu, zl, t);
        if (lane < c) acc += (double)Rn[lane + (int64_t)(j0 + t) * c] * zj;
      }
    }
    x -= acc;
  }
  // stage R_ss (c x c) in this warp's shared region, then the back substitution
  extern __shared__ __align__(16) unsigned char wsm[];
  TW* B = reinterpret_cast<TW*>(wsm) + (size_t)(threadIdx.x >> 5) * (32 * 33);
  for (int q = 0; q < c; ++q)
    if (lane < c) B[lane * 33 + q] = op.R[lane + (int64_t)q * c];
  const double rd = lane < c ? op.rdiag[lane] : 0.0;
  __syncwarp();
  for (int j = c - 1; j >= 0; --j) {
    const double yj = __shfl_sync(0xffffffffu, x, j) * __shfl_sync(0xffffffffu, rd, j);
    if (lane == j) x = yj;
    if (lane < j) x -= (double)B[lane * 33 + j] * yj;
  }
  if (lane < c) z[op.slots[lane]] = x;
}

template <typename TW>
__global__ void __launch_bounds__(kT) r_invT_warp_kernel(const ApplyOp<TW>* ops, const int* ids, int count,
                                                         double* z) {
  const int gw = (int)((blockIdx.x * (unsigned)kT + threadIdx.x) >> 5);
  if (gw >= count) return;
  const ApplyOp<TW> op = ops[ids[gw]];
  const int lane = threadIdx.x & 31, c = op.c, w = op.w;
  double x = lane < c ? z[op.slots[lane]] : 0.0;
  extern __shared__ __align__(16) unsigned char wsm[];
  TW* B = reinterpret_cast<TW*>(wsm) + (size_t)(threadIdx.x >> 5) * (32 * 33);
  for (int q = 0; q < c; ++q)
    if (lane < c) B[lane * 33 + q] = op.R[lane + (int64_t)q * c];
  const double rd = lane < c ? op.rdiag[lane] : 0.0;
  __syncwarp();
  for (int i = 0; i < c; ++i) {
    const double yi = __shfl_sync(0xffffffffu, x, i) * __shfl_sync(0xffffffffu, rd, i);
    if (lane == i) x = yi;
    if (lane > i && lane < c) x -= (double)B[i * 33 + lane] * yi;
  }
  if (lane < c) z[op.slots[lane]] = x;
  if (w > 0) {
    const TW* Rn = op.R + (int64_t)c * c;
    for (int j = 0; j < w; ++j) {
      double sv = lane < c ? (double)Rn[lane + (int64_t)j * c] * x : 0.0;
      sv = wsum(sv);
      if (lane == 0) atomicAdd(&z[op.nslots[j]], -sv);
    }
  }
}

template <typename TW>
__global__ void __launch_bounds__(kT) q_warp_kernel(const ApplyOp<TW>* ops, const int* ids, int count, double* z,
                                                    int transpose) {
  const int gw = (int)((blockIdx.x * (unsigned)kT + threadIdx.x) >> 5);
  if (gw >= count) return;
  const ApplyOp<TW> op = ops[ids[gw]];
  const int lane = threadIdx.x & 31, c = op.c;
  const int k = *op.kdev;
  double x = lane < c ? z[op.slots[lane]] : 0.0;
  for (int t = 0; t < k; ++t) {
    const int i = transpose ? t : k - 1 - t;
    const double v = lane == i ? 1.0 : ((lane > i && lane < c) ? (double)op.V[lane + (int64_t)i * c] : 0.0);
    const double d = wsum(v * x) * (double)op.tau[i];
    x -= d * v;
  }
  if (lane < c) z[op.slots[lane]] = x;
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

__global__ void __launch_bounds__(kT) scale_kernel(int64_t n, const double* a, const double* d, double* out) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i < n) out[i] = a[i] * d[i];
}

int blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + kT - 1) / kT); }

}  // namespace

// ------------------------------------------------------------------ plan
struct Segment {
  int kind;        // 0 R_s, 1 R_p, 2 Q_p
  int n_small;     // ops with c <= 32 (one warp each), ids at small_ids
  int n_large;     // ops with c > 32 (one CTA each), ids at large_ids
  const int* small_ids;
  const int* large_ids;
  int smem;        // dynamic shared memory of the CTA kernels
};

struct ApplyPlan {
  cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* d_rdiag = nullptr;     // 1 / R_ii of every R_s and R_p op
  bool fp32 = false;
  void* d_ops = nullptr;         // ApplyOp<TW>[nops] (factorization order)
  int32_t* d_idx = nullptr;      // slot index arrays
  int* d_ids = nullptr;          // op ids of every segment (small ones, then large ones)
  std::vector<Segment> segs;     // factorization order
  cudaGraphExec_t graph = nullptr;
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

template <typename TW>
static void build_plan_t(Handle& h, ApplyPlan& P) {
  std::vector<int32_t> idx;
  std::vector<ApplyOp<TW>> ops;
  std::vector<size_t> soff, noff;
  for (auto& op : h.ops) {
    soff.push_back(idx.size());
    idx.insert(idx.end(), op.slots.begin(), op.slots.end());
    noff.push_back(idx.size());
    idx.insert(idx.end(), op.nslots.begin(), op.nslots.end());
  }
  SPAQR_CUDA(cudaMalloc(&P.d_idx, std::max<size_t>(idx.size(), 1) * sizeof(int32_t)));
  SPAQR_CUDA(cudaMemcpy(P.d_idx, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  std::vector<size_t> roff(h.ops.size(), 0);
  size_t nrd = 0;
  for (size_t i = 0; i < h.ops.size(); ++i)
    if (h.ops[i].kind != 2) {
      roff[i] = nrd;
      nrd += (size_t)h.ops[i].c;
    }
  SPAQR_CUDA(cudaMalloc(&P.d_rdiag, std::max<size_t>(nrd, 1) * sizeof(double)));
  for (size_t i = 0; i < h.ops.size(); ++i) {
    const WOp& op = h.ops[i];
    ApplyOp<TW> a{};
    a.rdiag = op.kind != 2 ? P.d_rdiag + roff[i] : nullptr;
    a.R = static_cast<const TW*>(op.R);
    a.Qx = static_cast<const TW*>(op.Qx);
    a.V = static_cast<const TW*>(op.V);
    a.tau = static_cast<const TW*>(op.tau);
    a.kdev = op.kdev;
    a.slots = P.d_idx + soff[i];
    a.nslots = P.d_idx + noff[i];
    a.c = op.c;
    a.w = op.kind == 0 ? op.w : 0;
    ops.push_back(a);
  }
  // explicit Q_pp for the Q_p ops too wide for one warp
  std::vector<int> qids;
  std::vector<TW*> qouts;
  int qmax = 0;
  for (size_t i = 0; i < h.ops.size(); ++i) {
    WOp& op = h.ops[i];
    if (op.kind != 2 || op.c <= 32) continue;
    op.Qx = h.wpool.alloc((size_t)op.c * op.c * sizeof(TW));
    ops[i].Qx = static_cast<const TW*>(op.Qx);
    qids.push_back((int)i);
    qouts.push_back(static_cast<TW*>(op.Qx));
    qmax = std::max(qmax, op.c);
  }
  SPAQR_CUDA(cudaMalloc(&P.d_ops, std::max<size_t>(ops.size(), 1) * sizeof(ApplyOp<TW>)));
  SPAQR_CUDA(cudaMemcpy(P.d_ops, ops.data(), ops.size() * sizeof(ApplyOp<TW>), cudaMemcpyHostToDevice));
  if (nrd) {
    recip_diag_kernel<TW><<<(unsigned)((h.ops.size() + kW - 1) / kW), kT, 0, h.st>>>(
        static_cast<const ApplyOp<TW>*>(P.d_ops), (int)h.ops.size());
    SPAQR_CUDA(cudaGetLastError());
  }
  if (!qids.empty()) {
    int* d_q = nullptr;
    TW** d_out = nullptr;
    SPAQR_CUDA(cudaMalloc(&d_q, qids.size() * sizeof(int)));
    SPAQR_CUDA(cudaMalloc(&d_out, qouts.size() * sizeof(TW*)));
    SPAQR_CUDA(cudaMemcpy(d_q, qids.data(), qids.size() * sizeof(int), cudaMemcpyHostToDevice));
    SPAQR_CUDA(cudaMemcpy(d_out, qouts.data(), qouts.size() * sizeof(TW*), cudaMemcpyHostToDevice));
    const size_t smem = (size_t)qmax * kW * sizeof(double);
    int mx = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((int)smem > mx - 1024) throw Error(SPAQR_ERR_CAPACITY, "apply: Q_pp too large to form");
    set_dyn_smem(form_q_kernel<TW>);
    for (size_t b0 = 0; b0 < qids.size(); b0 += 65535) {
      const unsigned nb = (unsigned)std::min<size_t>(65535, qids.size() - b0);
      form_q_kernel<TW><<<dim3((unsigned)((qmax + 31) / 32), nb), kT, smem, h.st>>>(
          static_cast<const ApplyOp<TW>*>(P.d_ops), d_q + b0, d_out + b0);
      SPAQR_CUDA(cudaGetLastError());
    }
    SPAQR_CUDA(cudaStreamSynchronize(h.st));
    cudaFree(d_q);
    cudaFree(d_out);
  }
  // segments: consecutive ops with equal (kind, stage, round for R_s)
  std::vector<int> ids;
  struct Tmp {
    int kind, ns, nl, maxc;
    size_t s0, l0;
  };
  std::vector<Tmp> tmp;
  size_t i = 0;
  while (i < h.ops.size()) {
    size_t j = i + 1;
    const WOp& a = h.ops[i];
    while (j < h.ops.size() && h.ops[j].kind == a.kind && h.ops[j].stage == a.stage &&
           (a.kind != 0 || h.ops[j].round == a.round))
      ++j;
    Tmp t{a.kind, 0, 0, 0, 0, 0};
    t.s0 = ids.size();
    for (size_t q = i; q < j; ++q)
      if (h.ops[q].c <= 32) {
        ids.push_back((int)q);
        t.ns++;
      }
    t.l0 = ids.size();
    for (size_t q = i; q < j; ++q)
      if (h.ops[q].c > 32) {
        ids.push_back((int)q);
        t.nl++;
        t.maxc = std::max(t.maxc, h.ops[q].c);
      }
    tmp.push_back(t);
    i = j;
  }
  SPAQR_CUDA(cudaMalloc(&P.d_ids, std::max<size_t>(ids.size(), 1) * sizeof(int)));
  SPAQR_CUDA(cudaMemcpy(P.d_ids, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice));
  for (auto& t : tmp) {
    Segment sg;
    sg.kind = t.kind;
    sg.n_small = t.ns;
    sg.n_large = t.nl;
    sg.small_ids = P.d_ids + t.s0;
    sg.large_ids = P.d_ids + t.l0;
    sg.smem = (int)((size_t)t.maxc * (kW + 1) * sizeof(double));
    P.segs.push_back(sg);
  }
}

void build_apply_plan(Handle& h) {
  free_apply_plan(h);
  h.plan = new ApplyPlan();
  h.plan->fp32 = h.precision == SPAQR_PREC_MIXED;
  if (h.plan->fp32)
    build_plan_t<float>(h, *h.plan);
  else
    build_plan_t<double>(h, *h.plan);
  int mx = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  mx -= 1024;  // margin for the kernels' static shared memory
  for (auto& s : h.plan->segs)
    if (s.smem > mx) throw Error(SPAQR_ERR_CAPACITY, "apply: cluster too large for shared memory");
  set_dyn_smem(r_inv_kernel<double>);
  set_dyn_smem(r_inv_kernel<float>);
  set_dyn_smem(r_invT_kernel<double>);
  set_dyn_smem(r_invT_kernel<float>);
  set_dyn_smem(q_kernel<double>);
  set_dyn_smem(q_kernel<float>);
  set_dyn_smem(r_inv_warp_kernel<double>);
  set_dyn_smem(r_invT_warp_kernel<double>);
  set_dyn_smem(r_inv_warp_kernel<float>);
  set_dyn_smem(r_invT_warp_kernel<float>);
  for (auto& e : h.plan->ev) SPAQR_CUDA(cudaEventCreate(&e));
  // algorithmic bytes of one W^{-1} plus one W^{-T} apply: every stored entry
  // once per direction, the slot indices, and the slot-vector reads/writes
  {
    const double es = h.plan->fp32 ? 4.0 : 8.0;
    double b = 0.0;
    for (auto& op : h.ops) {
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
  SPAQR_CUDA(cudaMalloc(&h.plan->d_scal, 8 * sizeof(double)));
  SPAQR_CUDA(cudaMalloc(&h.plan->d_part, (size_t)h.plan->part_n * sizeof(double)));
}

void free_apply_plan(Handle& h) {
  if (!h.plan) return;
  for (auto& e : h.plan->ev)
    if (e) cudaEventDestroy(e);
  if (h.plan->graph) cudaGraphExecDestroy(h.plan->graph);
  cudaFree(h.plan->d_ops);
  cudaFree(h.plan->d_idx);
  cudaFree(h.plan->d_ids);
  cudaFree(h.plan->d_rdiag);
  cudaFree(h.plan->d_scal);
  cudaFree(h.plan->d_part);
  delete h.plan;
  h.plan = nullptr;
}

template <typename TW>
static void apply_t(Handle& h, double* z, int transpose) {
  ApplyPlan& P = *h.plan;
  const ApplyOp<TW>* ops = static_cast<const ApplyOp<TW>*>(P.d_ops);
  const int nseg = (int)P.segs.size();
  for (int t = 0; t < nseg; ++t) {
    const Segment& s = P.segs[(size_t)(transpose ? t : nseg - 1 - t)];
    if (s.n_small) {
      const int grid = (s.n_small + kW - 1) / kW;
      if (s.kind == 2)
        q_warp_kernel<TW><<<grid, kT, 0, h.st>>>(ops, s.small_ids, s.n_small, z, transpose);
      else if (transpose)
        r_invT_warp_kernel<TW><<<grid, kT, kWarpSmem<TW>, h.st>>>(ops, s.small_ids, s.n_small, z);
      else
        r_inv_warp_kernel<TW><<<grid, kT, kWarpSmem<TW>, h.st>>>(ops, s.small_ids, s.n_small, z);
    }
    if (s.n_large) {
      if (s.kind == 2)
        q_kernel<TW><<<s.n_large, kT, (size_t)s.smem, h.st>>>(ops, s.large_ids, z, transpose);
      else if (transpose)
        r_invT_kernel<TW><<<s.n_large, kT, (size_t)s.smem, h.st>>>(ops, s.large_ids, z);
      else
        r_inv_kernel<TW><<<s.n_large, kT, (size_t)s.smem, h.st>>>(ops, s.large_ids, z);
    }
  }
  SPAQR_CUDA(cudaGetLastError());
}

// Diagnostic (SPAQR_PROFILE_APPLY=1): one W^{-1} and one W^{-T} with CUDA events
// around every segment, printed to stderr as stage/kind/ops/microseconds.
template <typename TW>
static void profile_apply_t(Handle& h, double* z) {
  ApplyPlan& P = *h.plan;
  const ApplyOp<TW>* ops = static_cast<const ApplyOp<TW>*>(P.d_ops);
  const int nseg = (int)P.segs.size();
  std::vector<cudaEvent_t> ev(2 * (size_t)nseg + 2);
  for (auto& e : ev) SPAQR_CUDA(cudaEventCreate(&e));
  for (int transpose = 0; transpose < 2; ++transpose) {
    for (int t = 0; t < nseg; ++t) {
      const int si = transpose ? t : nseg - 1 - t;
      const Segment& s = P.segs[(size_t)si];
      SPAQR_CUDA(cudaEventRecord(ev[2 * (size_t)t], h.st));
      if (s.n_small) {
        const int grid = (s.n_small + kW - 1) / kW;
        if (s.kind == 2)
          q_warp_kernel<TW><<<grid, kT, 0, h.st>>>(ops, s.small_ids, s.n_small, z, transpose);
        else if (transpose)
          r_invT_warp_kernel<TW><<<grid, kT, kWarpSmem<TW>, h.st>>>(ops, s.small_ids, s.n_small, z);
        else
          r_inv_warp_kernel<TW><<<grid, kT, kWarpSmem<TW>, h.st>>>(ops, s.small_ids, s.n_small, z);
      }
      if (s.n_large) {
        if (s.kind == 2)
          q_kernel<TW><<<s.n_large, kT, (size_t)s.smem, h.st>>>(ops, s.large_ids, z, transpose);
        else if (transpose)
          r_invT_kernel<TW><<<s.n_large, kT, (size_t)s.smem, h.st>>>(ops, s.large_ids, z);
        else
          r_inv_kernel<TW><<<s.n_large, kT, (size_t)s.smem, h.st>>>(ops, s.large_ids, z);
      }
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
        std::fprintf(stderr, "[spaqr] apply %s seg %3d kind %d small %6d large %5d: %8.1f us\n",
                     transpose ? "W^-T" : "W^-1", si, s.kind, s.n_small, s.n_large, ms * 1e3);
    }
    std::fprintf(stderr, "[spaqr] apply %s total %.3f ms over %d segments\n", transpose ? "W^-T" : "W^-1", tot, nseg);
  }
  for (auto& e : ev) cudaEventDestroy(e);
}

void profile_apply(Handle& h, double* z) {
  if (h.plan->fp32)
    profile_apply_t<float>(h, z);
  else
    profile_apply_t<double>(h, z);
}

void apply_Winv(Handle& h, double* z, int transpose) {
  if (!h.plan) throw Error(SPAQR_ERR_INVALID_ARG, "no factorization");
  if (h.plan->fp32)
    apply_t<float>(h, z, transpose);
  else
    apply_t<double>(h, z, transpose);
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
    int64_t launches = 0;
    for (auto& sg : P.segs) launches += (sg.n_small > 0) + (sg.n_large > 0);
    h.stats.n_kernel[4] += 2 * launches;
    h.stats.t_kernel[5] += (c + d) * 1e-3;
    h.stats.n_kernel[5] += 2;
  } else {
    cudaGetLastError();
  }
}

void cgls(Handle& h, const double* b_dev, double* x_dev, spaqr_solve_info* info) {
  auto t0 = std::chrono::steady_clock::now();
  ApplyPlan& P = *h.plan;
  const int64_t m = h.m, n = h.n;
  const size_t need = (size_t)3 * m + (size_t)5 * n;
  if (h.work_elems < need) {
    if (h.d_work) cudaFree(h.d_work);
    SPAQR_CUDA(cudaMalloc(&h.d_work, need * sizeof(double)));
    h.work_elems = need;
    if (P.graph) {
      cudaGraphExecDestroy(P.graph);
      P.graph = nullptr;
    }
  }
  double* r = h.d_work;
  double* q = r + m;
  double* xt = q + m;
  double* p = xt + n;
  double* t = p + n;
  double* u = t + n;
  double* s = u + n;
  (void)s;
  double* sv = s;
  const double* Dinv_w = h.d_D;  // |D^{-1} u| = |u / D|
  {
    const char* e = std::getenv("SPAQR_PROFILE_APPLY");
    if (e && e[0] == '1') {
      SPAQR_CUDA(cudaMemsetAsync(t, 0, (size_t)n * sizeof(double), h.st));
      profile_apply(h, t);
    }
  }
  SPAQR_CUDA(cudaMemsetAsync(xt, 0, (size_t)n * sizeof(double), h.st));
  SPAQR_CUDA(cudaMemcpyAsync(r, b_dev, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, h.st));
  spmv_kernel<<<blocks(n), kT, 0, h.st>>>(n, h.d_trowptr, h.d_tcolidx, h.d_tvals, r, u, Dinv_w, P.d_part);
  finish_sum_kernel<<<1, kT, 0, h.st>>>(blocks(n), P.d_part, P.d_scal + 2);
  SPAQR_CUDA(cudaMemcpyAsync(sv, u, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h.st));
  apply_Winv(h, sv, 1);
  SPAQR_CUDA(cudaMemcpyAsync(p, sv, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, h.st));
  sumsq_kernel<<<std::min(blocks(n), P.part_n), kT, 0, h.st>>>(n, sv, P.d_part);
  finish_sum_kernel<<<1, kT, 0, h.st>>>(std::min(blocks(n), P.part_n), P.d_part, P.d_scal + 0);
  double res0 = 0.0;
  SPAQR_CUDA(cudaMemcpyAsync(&res0, P.d_scal + 2, sizeof(double), cudaMemcpyDeviceToHost, h.st));
  SPAQR_CUDA(cudaStreamSynchronize(h.st));
  const double norm0 = std::sqrt(res0);
  h.stats.t_kernel[4] = h.stats.t_kernel[5] = 0.0;
  h.stats.n_kernel[4] = h.stats.n_kernel[5] = 0;
  int it = 0;
  double rel = norm0 > 0.0 ? 1.0 : 0.0;
  if (norm0 > 0.0) {
    const bool graphs = h.opt.use_graphs != 0;
    if (graphs && !P.graph) {
      cudaGraph_t g;
      SPAQR_CUDA(cudaStreamBeginCapture(h.st, cudaStreamCaptureModeThreadLocal));
      cgls_body(h, xt, r, p, t, q, u, sv, Dinv_w, true);
      SPAQR_CUDA(cudaStreamEndCapture(h.st, &g));
      SPAQR_CUDA(cudaGraphInstantiate(&P.graph, g, 0));
      cudaGraphDestroy(g);
    }
    for (it = 1; it <= h.opt.maxit; ++it) {
      if (graphs)
        SPAQR_CUDA(cudaGraphLaunch(P.graph, h.st));
      else
        cgls_body(h, xt, r, p, t, q, u, sv, Dinv_w, false);
      double res = 0.0;
      SPAQR_CUDA(cudaMemcpyAsync(&res, P.d_scal + 2, sizeof(double), cudaMemcpyDeviceToHost, h.st));
      SPAQR_CUDA(cudaStreamSynchronize(h.st));
      accumulate_solve_timers(h);
      rel = std::sqrt(res) / norm0;
      if (!(rel >= h.opt.tol)) break;
    }
    if (it > h.opt.maxit) it = h.opt.maxit;
  }
  scale_kernel<<<blocks(n), kT, 0, h.st>>>(n, xt, h.d_D, x_dev);
  SPAQR_CUDA(cudaGetLastError());
  SPAQR_CUDA(cudaStreamSynchronize(h.st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  h.stats.t_solve = secs;
  h.stats.iters = it;
  if (info) {
    info->iters = it;
    info->rel_resid = rel;
    info->converged = rel < h.opt.tol;
    info->seconds = secs;
  }
}

}  // namespace spaqr
