// Dense device kernels of the spaQR factorization (sm_103a).
//
//  * front QR (Section 2.3, 2.4): Householder QR of the eliminated columns of
//    a batch of uneven fronts.  Fronts that fit run entirely in shared memory,
//    one CTA each, with warp-shuffle reductions; larger fronts run blocked:
//    a panel kernel (reflectors + the compact-WY factor T) and a multi-CTA
//    trailing update C <- C - V (T^T (V^T C)).
//  * column-pivoted QR (Section 2.5, the rank-revealing QR of Section 4):
//    a warp, a CTA, a thread-block cluster or a group of CTAs per matrix with
//    column slabs in shared memory, pivot by the largest remaining column norm
//    (norms in the data's precision), stop at |R_ii| < eps |R_11| (R_ii and
//    the test to FP64 accuracy).
//  * reflector application (compact WY blocks for FP32 row vectors),
//    triangular solve X R^{-1}, batched block copies and the max-norm row
//    assignment (Section 2.2).
#include <cooperative_groups.h>

#include <atomic>
#include <mutex>
#include <cuda_runtime.h>

#include <cfloat>
#include <climits>
#include <cstdint>
#include <type_traits>
#include <vector>

namespace cg = cooperative_groups;

#include "kernels.h"

namespace spaqr {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr double kRecompute = 1e-8;  // exact norm recomputation threshold

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ copies
constexpr int kCopyChunk = kThreads * 8;  // elements per CTA

// One CTA per chunk of kCopyChunk elements; chunk_start[i] is the first chunk
// of descriptor i (prefix sums over the descriptors, chunk_start[count] = total).
template <typename T>
__global__ void __launch_bounds__(kThreads) copy_kernel(const CopyDesc<T>* descs, const int* chunk_start, int count) {
  int lo = 0, hi = count - 1;
  const int b = (int)blockIdx.x;
  while (lo < hi) {  // last i with chunk_start[i] <= b
    const int mid = (lo + hi + 1) >> 1;
    if (chunk_start[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  const CopyDesc<T> d = descs[lo];
  if (d.transpose) {
    // tile (32 rows x 64 columns) of the source through shared memory: read
    // along the source's columns, written along the destination's columns
    __shared__ T tile[64][33];
    const int tiles_r = (d.rows + 31) / 32;
    const int t = b - chunk_start[lo];
    const int r0 = (t % tiles_r) * 32, c0 = (t / tiles_r) * 64;
    const int lr = threadIdx.x & 31, lc = threadIdx.x >> 5;  // 32 rows x 8 columns per pass
    for (int cc = lc; cc < 64; cc += kThreads / 32) {
      const int r = r0 + lr, c = c0 + cc;
      T v = T(0);
      if (r < d.rows && c < d.cols && d.src) {
        const int sr = d.rowidx ? d.rowidx[r] : r;
        v = d.src[sr + (int64_t)c * d.sld];
      }
      tile[cc][lr] = v;
    }
    __syncthreads();
    // destination entry (c, r) at dst[c + r * dld]: lanes over c
    for (int e = threadIdx.x; e < 64 * 32; e += kThreads) {
      const int cc = e & 63, rr = e >> 6;
      const int r = r0 + rr, c = c0 + cc;
      if (r < d.rows && c < d.cols) d.dst[c + (int64_t)r * d.dld] = tile[cc][rr];
    }
    return;
  }
  // flat column-major index e = r + c * rows (a block holds fewer than 2^31
  // entries); (r, c) of the thread's first entry by one 32-bit division, then
  // stepped by kThreads rows (a division per step for blocks of fewer rows)
  const uint32_t rows = (uint32_t)d.rows;
  const uint32_t total = rows * (uint32_t)d.cols;
  const uint32_t beg = (uint32_t)(b - chunk_start[lo]) * kCopyChunk;
  if (beg >= total) return;
  const uint32_t end = beg + kCopyChunk < total ? beg + kCopyChunk : total;
  uint32_t e = beg + threadIdx.x;
  uint32_t c = e / rows, r = e - c * rows;
  for (; e < end; e += kThreads) {
    T v = T(0);
    if (d.src) {
      const int sr = d.rowidx ? d.rowidx[r] : (int)r;
      v = d.src[sr + (int64_t)c * d.sld];
    }
    if (d.transpose)
      d.dst[c + (int64_t)r * d.dld] = v;
    else
      d.dst[r + (int64_t)c * d.dld] = v;
    if (rows >= (uint32_t)kThreads) {
      r += kThreads;
      if (r >= rows) {
        r -= rows;
        ++c;
      }
    } else {
      const uint32_t n = e + kThreads;
      c = n / rows;
      r = n - c * rows;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) identity_kernel(const CopyDesc<T>* descs) {
  const CopyDesc<T> d = descs[blockIdx.x];
  const int64_t total = (int64_t)d.rows * d.cols;
  for (int64_t e = threadIdx.x; e < total; e += kThreads) {
    const int r = (int)(e % d.rows);
    const int c = (int)(e / d.rows);
    d.dst[r + (int64_t)c * d.dld] = (r == c) ? T(1) : T(0);
  }
}

// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi) / 2), the operations built from the error-free
// two-sum (Knuth) and two-product (one fused multiply-add) transformations
// (Dekker 1971; Ogita, Rump and Oishi 2005).  About 44 significant bits.  The
// FP32 pivoted QR forms R_ii and takes the rank decision with it: on this GPU
// every FP64 instruction of a warp holds the FP64 pipe for tens of cycles, so
// a handful of them per pivot step would dominate the step.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_quick(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float z = s - a;
  return DF{s, (a - (s - z)) + (b - z)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  return df_quick(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_sqr(float a) {
  const float p = a * a;
  return DF{p, fmaf(a, a, -p)};
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  return df_quick(p, e + (a.hi * b.lo + a.lo * b.hi));
}
__device__ __forceinline__ DF df_sqrt(DF a) {  // a >= 0; one Newton step from the FP32 root
  if (!(a.hi > 0.f)) return DF{0.f, 0.f};
  const float r = sqrtf(a.hi);
  const float res = fmaf(-r, r, a.hi) + a.lo;
  return df_quick(r, res * (0.5f / r));
}
__device__ __forceinline__ bool df_less(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// Sum of squares of the entries of a column to FP64 accuracy.  For FP32 data
// every term x^2 is split exactly into p + e (p = fl(x^2), e = fma(x, x, -p))
// and accumulated with two-sums, the rounding errors collected in a second
// FP32 word (the Sum2 scheme of Ogita, Rump and Oishi): s + c is the exact sum
// up to relative errors of order (n u)^2, u = 2^-24.  FP64 data are summed in
// FP64.  warp_total() leaves the warp's total, as a (hi, lo) pair, in every lane.
template <typename T>
struct SqSum;
template <>
struct SqSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s = fma(x, x, s); }
  __device__ __forceinline__ void warp_total(double& hi, double& lo) {
    hi = warp_sum(s);
    lo = 0.0;
  }
};
template <>
struct SqSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const DF p = df_sqr(x);
    const DF t = df_two_sum(s, p.hi);
    c += t.lo + p.lo;
    s = t.hi;
  }
  __device__ __forceinline__ void warp_total(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
      const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
      const DF t = df_two_sum(s, s2);
      c = (c + c2) + t.lo;
      s = t.hi;
    }
    const DF r = df_quick(s, c);
    hi = r.hi;
    lo = r.lo;
  }
};

// The Householder data of a pivot step from alpha (the diagonal entry) and the
// sum of squares below it (sh + sl): R_ii = beta = -sign(alpha) sqrt(alpha^2 +
// sigma), tau = (beta - alpha) / beta, den = alpha - beta (the reflector is the
// column below alpha divided by den), and the rank test |R_ii| < eps |R_11|
// (stop; also when beta = 0).  r11 holds |R_11| from step 0 on (set when
// first = true).  FP64 data: in FP64.  FP32 data: in double-float.
template <typename T>
struct HouseStep {
  T beta, tau, den;
  bool stop;
  T bh, bl;  // |beta| in the arithmetic of the rank test (bl = 0 for FP64)
};
__device__ __forceinline__ HouseStep<double> house_step(double alpha, double sh, double, double eps, double& r11,
                                                        bool first) {
  HouseStep<double> h;
  if (sh == 0.0) {
    h.beta = alpha;
    h.tau = 0.0;
    h.den = 0.0;
  } else {
    const double nrm = sqrt(alpha * alpha + sh);
    h.beta = alpha >= 0.0 ? -nrm : nrm;
    h.tau = (h.beta - alpha) / h.beta;
    h.den = alpha - h.beta;
  }
  const double ab = fabs(h.beta);
  if (first) r11 = ab;
  h.stop = h.beta == 0.0 || ab < eps * r11;
  h.bh = ab;
  h.bl = 0.0;
  return h;
}
__device__ __forceinline__ HouseStep<float> house_step(float alpha, float sh, float sl, DF eps, DF& r11, bool first) {
  HouseStep<float> h;
  DF b;  // |beta|
  if (sh == 0.f && sl == 0.f) {
    b = DF{fabsf(alpha), 0.f};
    h.beta = alpha;
    h.tau = 0.f;
    h.den = 0.f;
  } else {
    b = df_sqrt(df_add(df_sqr(alpha), DF{sh, sl}));
    const float sg = alpha >= 0.f ? -1.f : 1.f;  // beta = sg * b
    const DF den = df_add(DF{alpha, 0.f}, DF{-sg * b.hi, -sg * b.lo});  // alpha - beta, no cancellation
    h.beta = sg * (b.hi + b.lo);
    h.den = den.hi + den.lo;
    h.tau = -h.den / h.beta;  // (beta - alpha) / beta
  }
  if (first) r11 = b;
  h.stop = (b.hi == 0.f) || df_less(b, df_mul(eps, r11));
  h.bh = b.hi;
  h.bl = b.lo;
  return h;
}

// Householder data of a front column (no rank test): FP64 for FP64 data,
// double-float for FP32 data, as in the pivoted QR.
__device__ __forceinline__ HouseStep<double> front_house(double alpha, double sh, double sl) {
  double r11 = 0.0;
  return house_step(alpha, sh, sl, 0.0, r11, true);
}
__device__ __forceinline__ HouseStep<float> front_house(float alpha, float sh, float sl) {
  DF r11{0.f, 0.f};
  return house_step(alpha, sh, sl, DF{0.f, 0.f}, r11, true);
}

// (hi, lo) sums of squares combined in a fixed order: double-float for FP32,
// plain addition for FP64 (lo = 0)
__device__ __forceinline__ void sq_combine(float& h, float& l, float h2, float l2) {
  const DF t = df_add(DF{h, l}, DF{h2, l2});
  h = t.hi;
  l = t.lo;
}
__device__ __forceinline__ void sq_combine(double& h, double& l, double h2, double) { h += h2; (void)l; }

// --------------------------------------------------------- reflector maths
// Computes the Householder reflector of x = X[j:m, j] (column j of X with
// leading dimension ld) by warp 0: beta = -sign(alpha) ||x|| (sign(0) = +1),
// v = x / (alpha - beta) below the diagonal, tau = (beta - alpha) / beta;
// tau = 0 (H = I) when x[1:] = 0.  Writes v in place and beta at X[j, j].
// Returns (through shared memory) tau and beta.
template <typename T>
__device__ void make_reflector_warp0(T* X, int ld, int m, int j, T* s_tau, T* s_beta) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  T* col = X + (int64_t)j * ld;
  SqSum<T> acc;
  for (int i = j + 1 + lane; i < m; i += 32) acc.add(col[i]);
  T sh, sl;
  acc.warp_total(sh, sl);
  const HouseStep<T> h = front_house(col[j], sh, sl);
  if (h.tau != T(0))
    for (int i = j + 1 + lane; i < m; i += 32) col[i] = col[i] / h.den;
  __syncwarp();
  if (lane == 0) {
    col[j] = h.beta;
    *s_tau = h.tau;
    *s_beta = h.beta;
  }
}

// Applies H_j = I - tau v v^T (v stored in column j below the diagonal, v_j = 1)
// to columns [c0, c1) of X, rows j..m-1; one warp per column.
template <typename T>
__device__ void apply_reflector_cols(T* X, int ld, int m, int j, T tau, int c0, int c1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* v = X + (int64_t)j * ld;
  for (int cc = c0 + warp; cc < c1; cc += kWarps) {
    T* col = X + (int64_t)cc * ld;
    T s = T(0);
    for (int i = j + 1 + lane; i < m; i += 32) s += v[i] * col[i];
    s = warp_sum(s);
    const T w = tau * (col[j] + s);
    if (lane == 0) col[j] -= w;
    for (int i = j + 1 + lane; i < m; i += 32) col[i] -= w * v[i];
  }
}

// Applies H_j to column cc alone (one warp).
template <typename T>
__device__ __forceinline__ void apply_reflector_col(T* X, int ld, int m, int j, T tau, int cc) {
  const int lane = threadIdx.x & 31;
  const T* v = X + (int64_t)j * ld;
  T* col = X + (int64_t)cc * ld;
  T s = T(0);
  for (int i = j + 1 + lane; i < m; i += 32) s += v[i] * col[i];
  s = warp_sum(s);
  const T w = tau * (col[j] + s);
  if (lane == 0) col[j] -= w;
  for (int i = j + 1 + lane; i < m; i += 32) col[i] -= w * v[i];
}

// ------------------------------------------------- front QR, shared memory
// One CTA per front.  Look-ahead by one column: while warps 1..7 apply H_j to
// columns j+2.., warp 0 applies it to column j+1 and forms H_{j+1} from it,
// so the reflector's reductions overlap the trailing update (one CTA barrier
// per column).
template <typename T>
__global__ void __launch_bounds__(kThreads) front_qr_smem_kernel(const FrontDesc<T>* descs) {
  const FrontDesc<T> d = descs[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);
  __shared__ T s_tau2[2], s_beta2[2];  // reflector data by column parity
  const int m = d.m, n = d.n, c = d.c;
  if (m == 0 || n == 0) return;
  const int64_t tot = (int64_t)m * n;
  for (int64_t e = threadIdx.x; e < tot; e += kThreads) {
    const int r = (int)(e % m), cc = (int)(e / m);
    S[e] = d.ptr[r + (int64_t)cc * d.ld];
  }
  unsigned* negmask = reinterpret_cast<unsigned*>(S + tot);  // sign bits of R_ii
  for (int t = threadIdx.x; t < (c + 31) / 32; t += kThreads) negmask[t] = 0u;
  __syncthreads();
  const int steps = c < m ? c : m;
  const int warp = threadIdx.x >> 5;
  if (steps > 0) make_reflector_warp0(S, m, m, 0, &s_tau2[0], &s_beta2[0]);
  __syncthreads();
  for (int j = 0; j < steps; ++j) {
    const T tau = s_tau2[j & 1];
    if (warp == 0) {
      if (threadIdx.x == 0 && s_beta2[j & 1] < T(0)) negmask[j >> 5] |= 1u << (j & 31);
      if (j + 1 < n) {
        if (tau != T(0)) apply_reflector_col(S, m, m, j, tau, j + 1);
        if (j + 1 < steps) {
          __syncwarp();
          make_reflector_warp0(S, m, m, j + 1, &s_tau2[(j + 1) & 1], &s_beta2[(j + 1) & 1]);
        }
      }
    } else if (tau != T(0)) {
      // two columns per pass: their dot products and warp sums are independent
      const int lane = threadIdx.x & 31;
      const T* v = S + (int64_t)j * m;
      int cc = j + 2 + (warp - 1);
      for (; cc + (kWarps - 1) < n; cc += 2 * (kWarps - 1)) {
        T* c0 = S + (int64_t)cc * m;
        T* c1 = S + (int64_t)(cc + kWarps - 1) * m;
        T a0 = T(0), a1 = T(0);
        for (int i = j + 1 + lane; i < m; i += 32) {
          const T vi = v[i];
          a0 += vi * c0[i];
          a1 += vi * c1[i];
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        const T w0 = tau * (c0[j] + a0), w1 = tau * (c1[j] + a1);
        if (lane == 0) {
          c0[j] -= w0;
          c1[j] -= w1;
        }
        for (int i = j + 1 + lane; i < m; i += 32) {
          const T vi = v[i];
          c0[i] -= w0 * vi;
          c1[i] -= w1 * vi;
        }
      }
      if (cc < n) apply_reflector_col(S, m, m, j, tau, cc);
    }
    __syncthreads();
  }
  // zero below the diagonal of the eliminated columns; flip rows with R_ii < 0
  for (int64_t e = threadIdx.x; e < tot; e += kThreads) {
    const int r = (int)(e % m), cc = (int)(e / m);
    T v = S[e];
    if (cc < steps && r > cc) v = T(0);
    if (r < steps && ((negmask[r >> 5] >> (r & 31)) & 1u)) v = -v;
    d.ptr[r + (int64_t)cc * d.ld] = v;
  }
}

// ----------------------------------------------- front QR, one warp each
// For small fronts: every warp of the CTA factors its own front in its own
// shared-memory region (ld = m | 1, odd, so that lane-per-column accesses are
// conflict-free).  Reflector norms by warp shuffles; trailing updates one lane
// per column; only __syncwarp, no block barriers.
template <typename T>
__global__ void __launch_bounds__(kThreads) front_qr_warp_kernel(const FrontDesc<T>* descs, int count,
                                                                 int per_warp_elems) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * kWarps + warp;
  if (f >= count) return;
  const FrontDesc<T> d = descs[f];
  extern __shared__ __align__(16) unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw) + (size_t)warp * per_warp_elems;
  const int m = d.m, n = d.n, c = d.c;
  const int ld = m | 1;
  for (int cc = 0; cc < n; ++cc)
    for (int r = lane; r < m; r += 32) S[r + cc * ld] = d.ptr[r + (int64_t)cc * d.ld];
  __syncwarp();
  const int steps = c < m ? c : m;
  unsigned neg = 0u;  // sign bits of R_ii, bit j of lane (j & 31) for j >> 5 == word... kept per 32-block
  unsigned negs[4] = {0u, 0u, 0u, 0u};  // steps <= 128 for this kernel
  for (int j = 0; j < steps; ++j) {
    T* col = S + j * ld;
    SqSum<T> acc;
    for (int r = j + 1 + lane; r < m; r += 32) acc.add(col[r]);
    T sh, sl;
    acc.warp_total(sh, sl);
    const HouseStep<T> h = front_house(col[j], sh, sl);
    if (h.tau != T(0))
      for (int r = j + 1 + lane; r < m; r += 32) col[r] = col[r] / h.den;
    if (h.beta < T(0)) negs[j >> 5] |= 1u << (j & 31);
    __syncwarp();
    if (lane == 0) col[j] = h.beta;
    __syncwarp();
    if (h.tau != T(0)) {
      const T tt = h.tau;
      for (int cc = j + 1 + lane; cc < n; cc += 32) {
        T* x = S + cc * ld;
        // four independent partial sums (rows j+1.. in steps of four)
        T s0 = x[j], s1 = T(0), s2 = T(0), s3 = T(0);
        int r = j + 1;
        for (; r + 3 < m; r += 4) {
          s0 += col[r] * x[r];
          s1 += col[r + 1] * x[r + 1];
          s2 += col[r + 2] * x[r + 2];
          s3 += col[r + 3] * x[r + 3];
        }
        for (; r < m; ++r) s0 += col[r] * x[r];
        const T sacc = (s0 + s1) + (s2 + s3);
        const T w = tt * sacc;
        x[j] -= w;
        for (int r = j + 1; r < m; ++r) x[r] -= w * col[r];
      }
    }
    __syncwarp();
  }
  (void)neg;
  for (int cc = 0; cc < n; ++cc)
    for (int r = lane; r < m; r += 32) {
      T v = S[r + cc * ld];
      if (cc < steps && r > cc) v = T(0);
      if (r < steps && ((negs[r >> 5] >> (r & 31)) & 1u)) v = -v;
      d.ptr[r + (int64_t)cc * d.ld] = v;
    }
}

// ----------------------------------------------------- front QR, blocked
// Panel: reflectors j0..j0+b-1 in global memory, then T (b x b, upper) with
// Q_panel = I - V T V^T, stored at Tbuf + f*nb*nb (ld nb).
template <typename T>
__global__ void __launch_bounds__(kThreads) front_panel_kernel(const FrontDesc<T>* descs, int j0, int nb,
                                                               T* Tbuf) {
  const FrontDesc<T> d = descs[blockIdx.x];
  const int steps = d.c < d.m ? d.c : d.m;
  const int b = min(nb, steps - j0);
  if (b <= 0) return;
  __shared__ T s_tau, s_beta;
  __shared__ T taus[64];
  __shared__ T G[64 * 64];  // G[l + i*64] = V_l . V_i (l < i)
  T* X = d.ptr;
  const int m = d.m, ld = d.ld;
  for (int jj = 0; jj < b; ++jj) {
    const int j = j0 + jj;
    make_reflector_warp0(X, ld, m, j, &s_tau, &s_beta);
    __syncthreads();
    const T tau = s_tau;
    if (threadIdx.x == 0) taus[jj] = tau;
    if (tau != T(0)) apply_reflector_cols(X, ld, m, j, tau, j + 1, j0 + b);
    __syncthreads();
  }
  // Gram entries of the unit-lower V (rows j0..m-1): G[l,i] = sum_r V[r,l] V[r,i], l < i
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int p = warp; p < b * b; p += kWarps) {
    const int l = p % b, i = p / b;
    if (l >= i) continue;
    const T* vl = X + (int64_t)(j0 + l) * ld;
    const T* vi = X + (int64_t)(j0 + i) * ld;
    T s = T(0);
    // row j0+i: V[., i] = 1; rows > j0+i: stored values; V[., l] stored below j0+l
    for (int r = j0 + i + lane; r < m; r += 32) s += vl[r] * (r == j0 + i ? T(1) : vi[r]);
    s = warp_sum(s);
    if (lane == 0) G[l + i * 64] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T* Tm = Tbuf + (int64_t)blockIdx.x * nb * nb;
    for (int i = 0; i < b; ++i) {
      Tm[i + i * nb] = taus[i];
      for (int l = 0; l < i; ++l) {
        // (T[0:i,0:i] G[0:i,i])_l
        T s = T(0);
        for (int q = l; q < i; ++q) s += Tm[l + q * nb] * G[q + i * 64];
        Tm[l + i * nb] = -taus[i] * s;
      }
      for (int l = i + 1; l < nb; ++l) Tm[l + i * nb] = T(0);
    }
  }
}

// Panel of the blocked QR on a thread-block cluster (tall panels): the rows
// j0..m-1 of the panel columns are split over the CS CTAs of the cluster and
// staged in shared memory (column-major, odd leading dimension).  Per column:
// every CTA pushes its partial sum of squares (FP64-accurate) and, for the
// owner of the diagonal, the diagonal entry into every CTA's shared memory;
// after a cluster barrier every thread forms the same reflector from them
// (summed in rank order); the partial products with the remaining panel
// columns are pushed the same way; after the second cluster barrier each CTA
// applies the rank-1 update to its own rows (the reflector's scaling by
// 1 / (alpha - beta) is folded into the reads and written back one column
// later) -- two cluster barriers and no remote loads per column.  The Gram
// matrix of the reflectors is reduced through distributed shared memory once
// per panel and T (Q = I - V T V^T) is formed warp-parallel by CTA 0.
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) front_panel_cluster_kernel(const FrontDesc<T>* descs, int j0, int nb,
                                                                           T* Tbuf, int per_max) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int f = blockIdx.x / CS;
  const FrontDesc<T> d = descs[f];
  const int steps = d.c < d.m ? d.c : d.m;
  const int b = min(nb, steps - j0);
  if (b <= 0) return;  // the same for every CTA of the cluster
  const int mrows = d.m - j0;
  const int per = (mrows + CS - 1) / CS;
  const int r0 = j0 + rank * per, r1 = min(d.m, r0 + per);
  const int nr = max(0, r1 - r0);
  const int ld = per_max | 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);  // nr x b, ld
  // exchange areas, written by the other CTAs of the cluster (index = source rank):
  // partial sums of squares (hi, lo) with the diagonal entry, and partial products
  // (pd shares its storage with the Gram partials Gp used after the last column)
  __shared__ T px_h[16], px_l[16], px_a[16];
  __shared__ T xbuf[32 * 33];
  T(*pd)[32] = reinterpret_cast<T(*)[32]>(xbuf);  // [16][32]
  T* Gp = xbuf;
  __shared__ T taus[32];
  __shared__ T red_h[kWarps], red_l[kWarps];
  __shared__ T wsum[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* X = d.ptr;
  for (int e = threadIdx.x; e < nr * b; e += kThreads) {
    const int r = e % nr, jj = e / nr;
    P[r + jj * ld] = X[(r0 + r) + (int64_t)(j0 + jj) * d.ld];
  }
  __syncthreads();
  T prev_rden = T(0);  // scale of the previous column's reflector, applied one step late
  for (int jj = 0; jj < b; ++jj) {
    const int j = j0 + jj;
    T* pc = P + jj * ld;
    if (jj > 0 && prev_rden != T(1)) {  // the previous reflector: its rows below its diagonal scaled in place
      T* pp = P + (jj - 1) * ld;
      for (int r = max(r0, j) + threadIdx.x; r < r1; r += kThreads) pp[r - r0] *= prev_rden;
    }
    // (1) this CTA's sum of squares below the diagonal (FP64-accurate), pushed
    // with the diagonal entry (owner) into every CTA of the cluster
    {
      SqSum<T> acc;
      for (int r = max(r0, j + 1) + threadIdx.x; r < r1; r += kThreads) acc.add(pc[r - r0]);
      T h, l;
      acc.warp_total(h, l);
      if (lane == 0) {
        red_h[warp] = h;
        red_l[warp] = l;
      }
    }
    __syncthreads();
    if (warp == 0) {
      T h = red_h[0], l = red_l[0];
      for (int w = 1; w < kWarps; ++w) sq_combine(h, l, red_h[w], red_l[w]);
      const T a = (j >= r0 && j < r1) ? pc[j - r0] : T(0);
      if (lane < CS) {
        *cl.map_shared_rank(&px_h[rank], lane) = h;
        *cl.map_shared_rank(&px_l[rank], lane) = l;
        *cl.map_shared_rank(&px_a[rank], lane) = a;
      }
    }
    cl.sync();  // (A) every CTA's partial norm and the diagonal entry are local
    const int owner = (j - j0) / per;
    // every thread: the partials combined in rank order, the Householder data
    T th = px_h[0], tl = px_l[0];
    for (int q = 1; q < CS; ++q) sq_combine(th, tl, px_h[q], px_l[q]);
    const HouseStep<T> hs = front_house(px_a[owner], th, tl);
    const T tau = hs.tau;
    const T rden = tau != T(0) ? T(1) / hs.den : T(1);  // v = x / (alpha - beta) below the diagonal
    if (threadIdx.x == 0) taus[jj] = tau;
    if (rank == owner && threadIdx.x == 0) pc[j - r0] = hs.beta;  // row j is read as v_j = 1 from here on
    // partial products v . x_c for the panel columns c > jj (v_j = 1), pushed
    // into every CTA of the cluster
    for (int c = jj + 1 + warp; c < b; c += kWarps) {
      const T* xc = P + c * ld;
      T acc = T(0);
      for (int r = max(r0, j) + lane; r < r1; r += 32) acc += (r == j ? T(1) : pc[r - r0] * rden) * xc[r - r0];
      acc = warp_sum(acc);
      if (lane < CS) *cl.map_shared_rank(&pd[rank][c], lane) = acc;
    }
    cl.sync();  // (B) every CTA's partial products are local
    if (threadIdx.x > jj && threadIdx.x < b) {
      T w = T(0);
      for (int q = 0; q < CS; ++q) w += pd[q][threadIdx.x];  // rank order
      wsum[threadIdx.x] = tau * w;
    }
    __syncthreads();
    if (tau != T(0)) {
      // rank-1 update of this CTA's rows: a warp per column, lanes over rows
      const int rbeg = max(r0, j);
      for (int c = jj + 1 + warp; c < b; c += kWarps) {
        T* xc = P + c * ld;
        const T wc = wsum[c];
        for (int r = rbeg + lane; r < r1; r += 32) {
          const T vr = r == j ? T(1) : pc[r - r0] * rden;
          xc[r - r0] -= wc * vr;
        }
      }
    }
    prev_rden = rden;
    __syncthreads();
  }
  if (prev_rden != T(1)) {  // the last reflector's rows below its diagonal
    T* pp = P + (b - 1) * ld;
    for (int r = max(r0, j0 + b) + threadIdx.x; r < r1; r += kThreads) pp[r - r0] *= prev_rden;
  }
  __syncthreads();
  // Gram of the unit-lower reflectors over this CTA's rows: G[l, i] = v_l . v_i, l < i
  for (int pq = warp; pq < b * b; pq += kWarps) {
    const int l = pq % b, i = pq / b;
    if (l >= i) continue;
    T acc = T(0);
    for (int r = max(r0, j0 + i) + lane; r < r1; r += 32) {
      const T vi = r == j0 + i ? T(1) : P[(r - r0) + i * ld];
      acc += P[(r - r0) + l * ld] * vi;
    }
    acc = warp_sum(acc);
    if (lane == 0) Gp[l + i * 33] = acc;
  }
  cl.sync();  // (C) partial Gram matrices visible
  if (rank == 0) {
    // G summed over the cluster: one thread per (l, i) pair, its CS remote
    // loads issued together and added in rank order, in place (no other CTA
    // reads CTA 0's partials)
    for (int pq = threadIdx.x; pq < b * b; pq += kThreads) {
      const int l = pq % b, i = pq / b;
      if (l >= i) continue;
      T v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = q < CS ? *cl.map_shared_rank(&Gp[l + i * 33], q) : T(0);
      T g = T(0);
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (q < CS) g += v[q];
      Gp[l + i * 33] = g;
    }
    __syncthreads();
    if (warp == 0) {
      // T column by column, in place over G (column i of G is read into wsum
      // before column i of T replaces it; later columns need only their own
      // column of G and the finished columns of T):
      // T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i]
      for (int i = 0; i < b; ++i) {
        wsum[lane] = lane < i ? Gp[lane + i * 33] : T(0);  // G[lane, i]
        __syncwarp();
        T acc = T(0);
        if (lane < i)
          for (int qq = lane; qq < i; ++qq) acc += Gp[lane + qq * 33] * wsum[qq];
        __syncwarp();
        Gp[lane + i * 33] = lane < i ? -taus[i] * acc : (lane == i ? taus[i] : T(0));
        __syncwarp();
      }
      T* Tg = Tbuf + (int64_t)f * nb * nb;
      for (int i = 0; i < nb; ++i)
        if (lane < nb) Tg[lane + i * nb] = (i < b && lane < b) ? Gp[lane + i * 33] : T(0);
    }
  }
  // the panel back to global memory (R above, reflectors below the diagonal)
  for (int e = threadIdx.x; e < nr * b; e += kThreads) {
    const int r = e % nr, jj = e / nr;
    X[(r0 + r) + (int64_t)(j0 + jj) * d.ld] = P[r + jj * ld];
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Trailing update of columns [j0+b, n) in tiles of 32 columns per CTA:
// C <- C - V (T^T (V^T C)), rows j0..m-1.
constexpr int kTN = 32;
constexpr int kRC = 64;
template <typename T>
__global__ void __launch_bounds__(kThreads) front_trailing_kernel(const FrontDesc<T>* descs, int j0, int nb,
                                                                  const T* Tbuf) {
  const FrontDesc<T> d = descs[blockIdx.y];
  const int steps = d.c < d.m ? d.c : d.m;
  const int b = min(nb, steps - j0);
  if (b <= 0) return;
  const int col0 = j0 + b + blockIdx.x * kTN;
  if (col0 >= d.n) return;
  const int tn = min(kTN, d.n - col0);
  __shared__ T Vs[kRC][33];
  __shared__ T Cs[kRC][kTN + 1];
  __shared__ T Ws[32][kTN + 1];
  __shared__ T Tm[32 * 32];
  const T* Tg = Tbuf + (int64_t)blockIdx.y * nb * nb;
  for (int e = threadIdx.x; e < nb * nb && e < 32 * 32; e += kThreads) Tm[e] = (e % nb < b && e / nb < b) ? Tg[e] : T(0);
  T* X = d.ptr;
  const int ld = d.ld, m = d.m;
  const int tcol = threadIdx.x & 31;  // tile column
  const int trow = threadIdx.x >> 5;  // 0..7
  T acc[4] = {T(0), T(0), T(0), T(0)};  // W[trow + 8q][tcol]
  for (int r0 = j0; r0 < m; r0 += kRC) {
    const int rc = min(kRC, m - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < kRC * 32; e += kThreads) {
      const int r = e % kRC, i = e / kRC;
      T v = T(0);
      if (r < rc && i < b) {
        const int gr = r0 + r, gc = j0 + i;
        v = gr < gc ? T(0) : (gr == gc ? T(1) : X[gr + (int64_t)gc * ld]);
      }
      Vs[r][i] = v;
    }
    for (int e = threadIdx.x; e < kRC * kTN; e += kThreads) {
      const int r = e % kRC, cc = e / kRC;
      Cs[r][cc] = (r < rc && cc < tn) ? X[(r0 + r) + (int64_t)(col0 + cc) * ld] : T(0);
    }
    __syncthreads();
    for (int r = 0; r < rc; ++r) {
      const T cv = Cs[r][tcol];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += Vs[r][trow + 8 * q] * cv;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) Ws[trow + 8 * q][tcol] = acc[q];
  __syncthreads();
  // W2 = T^T W  (T upper => T^T lower): W2[i] = sum_{l<=i} T[l,i] W[l]
  T w2[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = trow + 8 * q;
    T s = T(0);
    for (int l = 0; l <= i && l < b; ++l) s += Tm[l + i * nb] * Ws[l][tcol];
    w2[q] = i < b ? s : T(0);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) Ws[trow + 8 * q][tcol] = w2[q];
  __syncthreads();
  for (int r0 = j0; r0 < m; r0 += kRC) {
    const int rc = min(kRC, m - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < kRC * 32; e += kThreads) {
      const int r = e % kRC, i = e / kRC;
      T v = T(0);
      if (r < rc && i < b) {
        const int gr = r0 + r, gc = j0 + i;
        v = gr < gc ? T(0) : (gr == gc ? T(1) : X[gr + (int64_t)gc * ld]);
      }
      Vs[r][i] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kRC * kTN; e += kThreads) {
      const int r = e % kRC, cc = e / kRC;
      if (r < rc && cc < tn) {
        T s = T(0);
        for (int i = 0; i < b; ++i) s += Vs[r][i] * Ws[i][cc];
        X[(r0 + r) + (int64_t)(col0 + cc) * ld] -= s;
      }
    }
  }
}

// After the panels: zero below the diagonal of the eliminated columns and flip
// rows of R with a negative diagonal.
// The signs of the diagonal entries R_ii of every front, as bit masks (front f
// at masks + f * words_per_front), taken before any row is flipped.
template <typename T>
__global__ void __launch_bounds__(kThreads) front_signs_kernel(const FrontDesc<T>* descs, unsigned* masks,
                                                               int words_per_front) {
  const FrontDesc<T> d = descs[blockIdx.x];
  const int steps = d.c < d.m ? d.c : d.m;
  const int words = (steps + 31) / 32;
  __shared__ unsigned sm[kThreads];
  unsigned* out = masks + (size_t)blockIdx.x * words_per_front;
  for (int w0 = 0; w0 < words; w0 += kThreads) {
    __syncthreads();
    if (w0 + (int)threadIdx.x < words) sm[threadIdx.x] = 0u;
    __syncthreads();
    for (int i = w0 * 32 + threadIdx.x; i < steps && i < (w0 + kThreads) * 32; i += kThreads)
      if (d.ptr[i + (int64_t)i * d.ld] < T(0)) atomicOr(&sm[(i >> 5) - w0], 1u << (i & 31));
    __syncthreads();
    if (w0 + (int)threadIdx.x < words) out[w0 + threadIdx.x] = sm[threadIdx.x];
  }
}

// Blocked fronts, after the last panel: rows i with R_ii < 0 are negated from
// column i on (diag(R) >= 0), and the eliminated columns are zeroed below the
// diagonal.  CTA (f, y) takes 32 columns of front f, threads over rows.
template <typename T>
__global__ void __launch_bounds__(kThreads) front_finish_kernel(const FrontDesc<T>* descs, const unsigned* masks,
                                                                int words_per_front) {
  const FrontDesc<T> d = descs[blockIdx.x];
  const int c0 = blockIdx.y * 32;
  if (c0 >= d.n) return;
  const int c1 = min(d.n, c0 + 32);
  const int steps = d.c < d.m ? d.c : d.m;
  const unsigned* mk = masks + (size_t)blockIdx.x * words_per_front;
  T* X = d.ptr;
  for (int cc = c0; cc < c1; ++cc) {
    const int rows = cc < steps ? d.m : steps;  // zeroing below the diagonal only in eliminated columns
    T* col = X + (int64_t)cc * d.ld;
    for (int r = threadIdx.x; r < rows; r += kThreads) {
      if (r > cc) {
        col[r] = T(0);
      } else if (r < steps && ((__ldg(&mk[r >> 5]) >> (r & 31)) & 1u)) {
        col[r] = -col[r];
      }
    }
  }
}

// Transposed butterfly over a warp: lanes hold a[0..G) (G a power of two
// <= 32); log2(G) halving exchanges (lanes with bit lvl set keep the upper
// half) then plain exchanges leave every lane with the warp-wide sum of
// column butterfly_col(lane); butterfly_lane(j) is the lowest lane holding it.
template <int G>
__device__ __forceinline__ int butterfly_col(int lane) {
  int j = 0, half = G / 2;
  for (int lvl = 16; half >= 1; lvl >>= 1, half >>= 1)
    if (lane & lvl) j += half;
  return j;
}
template <int G>
__device__ __forceinline__ int butterfly_lane(int j) {
  int l = 0, half = G / 2;
  for (int lvl = 16; half >= 1; lvl >>= 1, half >>= 1)
    if (j & half) l += lvl;
  return l;
}
template <int G, typename T>
__device__ __forceinline__ T butterfly_reduce(T (&a)[G], int lane) {
  int lvl = 16;
#pragma unroll
  for (int cnt = G; cnt > 1; cnt >>= 1, lvl >>= 1) {
    const bool up = lane & lvl;
#pragma unroll
    for (int q = 0; q < cnt / 2; ++q)
      a[q] = (up ? a[q + cnt / 2] : a[q]) + __shfl_xor_sync(0xffffffffu, up ? a[q] : a[q + cnt / 2], lvl);
  }
  T v = a[0];
  for (; lvl >= 1; lvl >>= 1) v += __shfl_xor_sync(0xffffffffu, v, lvl);
  return v;
}

// Partial column norms are downdated and recomputed exactly once they have
// lost more than this fraction of the last exact value: the reference
// algorithm's FP64 threshold, and sqrt(FP32 epsilon) (single-precision LAPACK's
// tol3z) for norms kept in FP32.
template <typename N>
__device__ __forceinline__ N recompute_frac();
template <>
__device__ __forceinline__ double recompute_frac<double>() {
  return kRecompute;
}
template <>
__device__ __forceinline__ float recompute_frac<float>() {
  return 3.4527e-4f;
}

// One warp's proposal for the next pivot step, as the slab QRCP exchanges it:
// the squared partial norm that orders the pivots (v), the column (j, original
// index; INT_MAX = none), its entry at the next diagonal position (alpha) and
// the FP64-accurate sum of squares of its entries below (sh + sl).
template <typename T, typename N>
struct QrcpProp {
  N v;
  int j;
  T alpha, sh, sl;
};

// Lowest original column index among equal norms: the pivot rule of the oracle.
template <typename N>
__device__ __forceinline__ bool prop_better(N v, int j, N bv, int bj) {
  return v > bv || (v == bv && j < bj);
}

// Every lane of the warp ends with the best of the warp's (v, j) and the lane
// holding it.
template <typename N>
__device__ __forceinline__ int warp_argmax(N& v, int& j) {
  int who = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const N ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oj = __shfl_xor_sync(0xffffffffu, j, o);
    const int ow = __shfl_xor_sync(0xffffffffu, who, o);
    if (prop_better(ov, oj, v, j)) {
      v = ov;
      j = oj;
      who = ow;
    }
  }
  return who;
}

// 16-byte shared-memory vectors: four FP32 or two FP64 consecutive rows
template <typename T>
__device__ __forceinline__ void ld16(const T* p, T (&a)[16 / sizeof(T)]);
template <>
__device__ __forceinline__ void ld16<float>(const float* p, float (&a)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a[0] = v.x;
  a[1] = v.y;
  a[2] = v.z;
  a[3] = v.w;
}
template <>
__device__ __forceinline__ void ld16<double>(const double* p, double (&a)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a[0] = v.x;
  a[1] = v.y;
}
template <typename T>
__device__ __forceinline__ void st16(T* p, const T (&a)[16 / sizeof(T)]);
template <>
__device__ __forceinline__ void st16<float>(float* p, const float (&a)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(a[0], a[1], a[2], a[3]);
}
template <>
__device__ __forceinline__ void st16<double>(double* p, const double (&a)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(a[0], a[1]);
}

// ------------------------------------------------------------------- QRCP
// Column-pivoted Householder QR stopped at the rank, one thread-block cluster
// of CS CTAs (CS = 1 allowed) per matrix.  CTA r of the cluster owns the
// column slab [r*nl, (r+1)*nl) (nl = ceil(n/CS)) in its shared memory, columns
// of ldx = m rounded up to four rows (zero below m).  Columns never move.  One
// pivot step is
//   B1  every warp has left, from its share of the previous update, its best
//       column (partial norm, index); CTA barrier; every thread reduces them to
//       the CTA's best, all threads sum the squares below the next diagonal
//       entry of that column (FP64-accurate), B1b combines the warps' parts in
//       a fixed order: the CTA's record (norm, index, sum, diagonal entry);
//   with CS > 1 each CTA pushes its record into every CTA's shared memory and,
//       after one cluster barrier, every warp reduces the CS records the same
//       way (local reads only);
//   R_ii = beta and tau follow from the winner's record alone (FP64, or
//       double-float for FP32 data), the rank test |R_ii| >= eps |R_11| stops
//       the loop uniformly;
//   every thread scales its rows of the winner's column, read from the owner's
//       slab (distributed shared memory), into the local reflector buffer, which
//       is indexed by row (zero above row i, one at row i);
//   B2  CTA barrier; the update x_j <- x_j - tau (v^T x_j) v of the unpivoted
//       columns (compact list act[]) in 16-byte row vectors with the downdate of
//       their partial norms, and each warp's best column for the next step.
// The owner writes beta and the reflector into the pivot column once no CTA
// can still read it: at once when CS = 1, otherwise after the next cluster
// barrier (double-buffered records and reflector buffers keep every read of
// step i apart from the writes of step i + 1).
template <typename T, int KG, int NT>
__global__ void __launch_bounds__(NT, 1) qrcp_slab_kernel(const QrcpDesc<T>* descs, double eps, int nl_max,
                                                       int m_max) {
  constexpr int NW = NT / 32;
  constexpr int VW = 16 / (int)sizeof(T);
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const QrcpDesc<T> d = descs[blockIdx.x / CS];
  const int m = d.m, n = d.n;
  const int ldx = qrcp_ldx(m);
  const int nl = (n + CS - 1) / CS;
  const int j0 = min(n, rank * nl), j1 = min(n, j0 + nl);
  const int nloc = j1 - j0;
  extern __shared__ __align__(16) unsigned char smraw[];
  using N = T;  // partial column norms and pivot order in the data's precision
  N* nu = reinterpret_cast<N*>(smraw);  // nl_max
  N* nuref = nu + nl_max;               // nl_max
  int* step_of = reinterpret_cast<int*>(nuref + nl_max);  // nl_max
  int* act = step_of + nl_max;                            // unpivoted local columns, nl_max
  int* pos = act + nl_max;                                // position of each column in act
  const int vstride = qrcp_vstride(m_max);
  T* vbuf = reinterpret_cast<T*>(smraw + (((size_t)nl_max * 28 + 15) / 16) * 16);  // 2 x vstride
  T* taus = vbuf + 2 * vstride;                                                    // vstride
  T* X = taus + vstride;                                                           // ldx x nloc slab
  __shared__ N wb_v[NW];  // every warp's best (v, j) after an update
  __shared__ int wb_j[NW];
  __shared__ T red_h[NW], red_l[NW];        // partial sums of squares of the CTA's best column
  __shared__ QrcpProp<T, N> pubs[2][16];  // every CTA's best of the step, pushed here by its owner (by parity)
  __shared__ int s_nact;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t e = threadIdx.x; e < (int64_t)ldx * nloc; e += NT) {
    const int r = (int)(e % ldx), c = (int)(e / ldx);
    X[e] = r < m ? d.src[r + (int64_t)(j0 + c) * d.ld] : T(0);
  }
  for (int e = threadIdx.x; e < 2 * vstride; e += NT) vbuf[e] = T(0);
  __syncthreads();
  for (int c = warp; c < nloc; c += NW) {
    N sq = N(0);
    for (int r = lane; r < m; r += 32) {
      const N v = (N)X[r + (int64_t)c * ldx];
      sq += v * v;
    }
    sq = warp_sum(sq);
    if (lane == 0) {
      nu[c] = sq;
      nuref[c] = sq;
      step_of[c] = -1;
    }
  }
  for (int c = threadIdx.x; c < nloc; c += NT) {
    act[c] = c;
    pos[c] = c;
  }
  if (threadIdx.x == 0) s_nact = nloc;
  const int kmax = m < n ? m : n;
  __syncthreads();
  {  // records for step 0: every warp over its columns c = warp + NW * (lane + 32 t)
    N wv = N(-1);
    int wj = INT_MAX;
    for (int c = warp + lane * NW; c < nloc; c += 32 * NW)
      if (prop_better(nu[c], j0 + c, wv, wj)) {
        wv = nu[c];
        wj = j0 + c;
      }
    warp_argmax(wv, wj);
    if (lane == 0) {
      wb_v[warp] = wv;
      wb_j[warp] = wj;
    }
  }
  // eps and |R_11| in the arithmetic of the rank test (FP64, or double-float for FP32 data)
  using Acc = typename std::conditional<sizeof(T) == 8, double, DF>::type;
  Acc eps_x, r11;
  if constexpr (sizeof(T) == 8) {
    eps_x = eps;
    r11 = 0.0;
  } else {
    const float e_hi = (float)eps;
    eps_x = DF{e_hi, (float)(eps - (double)e_hi)};
    r11 = DF{0.f, 0.f};
  }
  int k = 0;
  int pend_p = -1, pend_i = -1;  // pivot column this CTA still has to write (CS > 1)
  T pend_beta = T(0);
  const int jl = butterfly_col<KG>(lane);  // the column whose sum this lane ends with
  const bool lead = lane == butterfly_lane<KG>(jl);
  for (int i = 0; i < kmax; ++i) {
    const int par = i & 1;
    T* vb = vbuf + par * vstride;
    __syncthreads();  // B1: the warps' proposals of step i
    // the CTA's best column (every thread reduces the warps' proposals) and the
    // sum of squares below row i of that column, by all threads
    QrcpProp<T, N> best{N(-1), INT_MAX, T(0), T(0), T(0)};
    for (int w = 0; w < NW; ++w)
      if (prop_better(wb_v[w], wb_j[w], best.v, best.j)) {
        best.v = wb_v[w];
        best.j = wb_j[w];
      }
    if (best.j != INT_MAX) {
      const T* col = X + (int64_t)(best.j - j0) * ldx;
      SqSum<T> acc;
      for (int r = i + 1 + threadIdx.x; r < m; r += NT) acc.add(col[r]);
      T h, l;
      acc.warp_total(h, l);
      if (lane == 0) {
        red_h[warp] = h;
        red_l[warp] = l;
      }
    }
    __syncthreads();  // B1b
    if (best.j != INT_MAX) {
      T h = red_h[0], l = red_l[0];
      for (int w = 1; w < NW; ++w) sq_combine(h, l, red_h[w], red_l[w]);
      best.sh = h;
      best.sl = l;
      best.alpha = X[i + (int64_t)(best.j - j0) * ldx];
    }
    if (CS > 1) {
      // the CTA's best pushed into every CTA's shared memory (lane q: CTA q);
      // after the cluster barrier all bests of the step are local
      if (warp == 0 && lane < CS) *cl.map_shared_rank(&pubs[par][rank], lane) = best;
      cl.sync();  // the CTAs' bests of step i visible cluster-wide; step i - 1 reads finished
      QrcpProp<T, N> o{N(-1), INT_MAX, T(0), T(0), T(0)};
      if (lane < CS) o = pubs[par][lane];
      N v = o.v;
      int j = o.j;
      const int who = warp_argmax(v, j);
      best.alpha = __shfl_sync(0xffffffffu, o.alpha, who);
      best.sh = __shfl_sync(0xffffffffu, o.sh, who);
      best.sl = __shfl_sync(0xffffffffu, o.sl, who);
      best.v = v;
      best.j = j;
      if (pend_p >= 0) {  // the previous pivot column: nobody reads it any more
        T* col = X + (int64_t)(pend_p - j0) * ldx;
        const T* vp = vbuf + (pend_i & 1) * vstride;
        for (int r = pend_i + 1 + threadIdx.x; r < m; r += NT) col[r] = vp[r];
        if (threadIdx.x == 0) col[pend_i] = pend_beta;
        pend_p = -1;
      }
    }
    const int p = best.j;
    if (p == INT_MAX) break;  // no proposal (non-finite norms): the same p everywhere
    const int owner = p / nl;
    const int rb = i & ~(VW - 1);  // first row of the vectors the update touches
    const T* Xo = owner == rank ? X : cl.map_shared_rank(X, owner);
    const T* src = Xo + (int64_t)(p - owner * nl) * ldx;
    // this thread's first kPre rows of the winner's column, loaded before the
    // Householder arithmetic so that the (remote) loads overlap it
    constexpr int kPre = 8;
    T pre[kPre];
#pragma unroll
    for (int q = 0; q < kPre; ++q) {
      const int r = rb + (int)threadIdx.x + q * NT;
      pre[q] = (r > i && r < m) ? src[r] : T(0);
    }
    // R_ii, tau and the rank test, the same arithmetic in every thread
    const HouseStep<T> hs = house_step(best.alpha, best.sh, best.sl, eps_x, r11, i == 0);
    if (hs.stop) break;  // rank reached: the same decision everywhere
    const T den = hs.den;
    const T tau_t = hs.tau;
    const T beta_t = hs.beta;
    {  // the reflector by row: 0 above row i, 1 at row i, the scaled column below
      const T rden = den != T(0) ? T(1) / den : T(0);  // the reflector scaled by 1 / (alpha - beta)
#pragma unroll
      for (int q = 0; q < kPre; ++q) {
        const int r = rb + (int)threadIdx.x + q * NT;
        if (r < ldx) vb[r] = r < i ? T(0) : (r == i ? T(1) : pre[q] * rden);
      }
      for (int r = rb + (int)threadIdx.x + kPre * NT; r < ldx; r += NT)
        vb[r] = r < m ? src[r] * rden : T(0);
      if (threadIdx.x == 0) taus[i] = copysign(tau_t, beta_t);  // tau >= 0; the sign is that of R_ii
    }
    if (rank == owner && threadIdx.x == 0) {
      const int pl = p - j0;
      const int q = pos[pl], last = act[s_nact - 1];
      step_of[pl] = i;
      act[q] = last;
      pos[last] = q;
      s_nact = s_nact - 1;
    }
    __syncthreads();  // B2: vb complete, act[] updated
    if (rank == owner) {
      if (CS == 1) {
        T* col = X + (int64_t)(p - j0) * ldx;
        for (int r = i + 1 + threadIdx.x; r < m; r += NT) col[r] = vb[r];
        if (threadIdx.x == 0) col[i] = beta_t;
      } else {
        pend_p = p;
        pend_i = i;
        pend_beta = beta_t;
      }
    }
    // apply H_i to the CTA's unpivoted columns: every warp takes groups of KG
    // columns, each lane VW consecutive rows per 16-byte access, KG independent
    // accumulators; the KG dot products (row i included: v_i = 1) are reduced
    // by one transposed butterfly (lane L(j) ends with column j's sum),
    // w_j = tau v^T x_j is broadcast, the rows are updated, and lane L(j)
    // downdates the squared norm of column j (recomputed warp-parallel when it
    // lost too many digits)
    N wv = N(-1);
    int wj = INT_MAX;
    const int nact = s_nact;
    for (int g0 = warp * KG; g0 < nact; g0 += NW * KG) {
      const int ng = min(KG, nact - g0);
      T* cols[KG];
#pragma unroll
      for (int j = 0; j < KG; ++j) cols[j] = X + (int64_t)act[g0 + (j < ng ? j : 0)] * ldx;
      T acc[KG];
#pragma unroll
      for (int j = 0; j < KG; ++j) acc[j] = T(0);
      if (tau_t != T(0)) {
        for (int r = rb + lane * VW; r < ldx; r += 32 * VW) {
          T v[VW];
          ld16(vb + r, v);
#pragma unroll
          for (int j = 0; j < KG; ++j) {
            T x[VW];
            ld16(cols[j] + r, x);
#pragma unroll
            for (int q = 0; q < VW; ++q) acc[j] += v[q] * x[q];
          }
        }
      }
      const T dsum = butterfly_reduce<KG>(acc, lane);
      const int cme = jl < ng ? act[g0 + jl] : 0;
      const T wmine = jl < ng ? tau_t * dsum : T(0);
      T wv8[KG];
#pragma unroll
      for (int j = 0; j < KG; ++j) wv8[j] = __shfl_sync(0xffffffffu, wmine, butterfly_lane<KG>(j));
      if (tau_t != T(0)) {
        for (int r = rb + lane * VW; r < ldx; r += 32 * VW) {
          T v[VW];
          ld16(vb + r, v);
#pragma unroll
          for (int j = 0; j < KG; ++j)
            if (j < ng) {
              T x[VW];
              ld16(cols[j] + r, x);
#pragma unroll
              for (int q = 0; q < VW; ++q) x[q] -= wv8[j] * v[q];
              st16(cols[j] + r, x);
            }
        }
      }
      __syncwarp();
      N v = N(-1);
      bool redo = false;
      if (lead && jl < ng) {
        const N xnew = (N)X[i + (int64_t)cme * ldx];
        v = nu[cme] - xnew * xnew;
        redo = v < recompute_frac<N>() * nuref[cme];
      }
      unsigned flagged = __ballot_sync(0xffffffffu, redo);
      while (flagged) {
        const int l = __ffs(flagged) - 1;
        flagged &= flagged - 1;
        const int cc = __shfl_sync(0xffffffffu, cme, l);
        const T* col = X + (int64_t)cc * ldx;
        N sq = N(0);
        for (int r = i + 1 + lane; r < m; r += 32) {
          const N y = (N)col[r];
          sq += y * y;
        }
        sq = warp_sum(sq);
        if (lane == l) {
          v = sq;
          nuref[cc] = sq;
        }
      }
      if (lead && jl < ng) {
        nu[cme] = v;
        if (prop_better(v, j0 + cme, wv, wj)) {
          wv = v;
          wj = j0 + cme;
        }
      }
    }
    // the warp's proposal for step i + 1 (its columns are all updated: __syncwarp above)
    warp_argmax(wv, wj);
    if (lane == 0) {
      wb_v[warp] = wv;
      wb_j[warp] = wj;
    }
    k = i + 1;
  }
  if (CS > 1) {
    cl.sync();  // every read of the last pivot column is done
    if (pend_p >= 0) {
      T* col = X + (int64_t)(pend_p - j0) * ldx;
      const T* vp = vbuf + (pend_i & 1) * vstride;
      for (int r = pend_i + 1 + threadIdx.x; r < m; r += NT) col[r] = vp[r];
      if (threadIdx.x == 0) col[pend_i] = pend_beta;
    }
  }
  __syncthreads();
  if (rank == 0 && threadIdx.x == 0) d.rank[0] = k;
  if (d.V) {
    for (int64_t e = threadIdx.x; e < (int64_t)m * nloc; e += NT) {
      const int r = (int)(e % m), c = (int)(e / m);
      const int t = step_of[c];
      if (t < 0 || t >= k) continue;
      d.V[r + (int64_t)t * m] = r < t ? T(0) : (r == t ? T(1) : X[r + (int64_t)c * ldx]);
    }
    if (rank == 0)
      for (int t = threadIdx.x; t < k; t += NT) d.tau[t] = fabs(taus[t]);
  }
  // the first k rows of Q^T A in the original column order, only when k < m
  if (d.out && (k < m || (d.flags & kQrcpAlwaysOut))) {
    const bool fix = d.flags & kQrcpSignFix;
    for (int64_t e = threadIdx.x; e < (int64_t)k * nloc; e += NT) {
      const int r = (int)(e % k), c = (int)(e / k);
      const int t = step_of[c];
      const T x = (t >= 0 && r > t) ? T(0) : X[r + (int64_t)c * ldx];
      d.out[r + (int64_t)(j0 + c) * d.ldo] = fix && signbit(taus[r]) ? -x : x;
    }
  }
  if (CS > 1) cl.sync();  // no CTA leaves while another may still read its shared memory
}

// ------------------------------------------- QRCP over a group of CTAs
// The same slab-in-shared-memory pivoted QR for matrices whose slabs need more
// CTAs than one cluster holds: matrix f of a launch takes CTAs
// [cta0, cta0 + ctas) (all resident at once: cooperative launch) and the
// cluster barrier plus distributed-shared-memory reads become a message
// exchange through global memory (L2).  At step i every CTA writes its
// proposal and the speculative reflector of its best column into buffer
// (i & 1), then adds one to that buffer's arrival counter; every CTA waits
// until the counter shows all G arrivals of the step (a bounded wait: on
// expiry it raises the matrix's timeout tag, writes rank -1 and returns), picks the same
// winner and copies the winner's reflector.  A CTA can only reach step i + 2,
// which rewrites buffer (i & 1), after every CTA has arrived at step i + 1,
// i.e. after every CTA has finished reading step i.
// One CTA's proposal of a grid-mode step as it sits in global memory (the 32
// bytes of a QrcpSlot): the squared partial norm and column of its best
// column, that column's Householder data and rank decision, and |beta| in the
// arithmetic of the rank test (double-float for FP32: R_11 at step 0).
template <typename T>
struct GridSlot;
template <>
struct GridSlot<double> {
  double v, beta, tau;
  int j, stop;
  __device__ __forceinline__ void set_b(double, double) {}
  __device__ __forceinline__ void load_b(const GridSlot*) {}
  __device__ __forceinline__ double b_acc() const { return fabs(beta); }
};
template <>
struct GridSlot<float> {
  float v, beta, tau, bh, bl;
  int j, stop, pad;
  __device__ __forceinline__ void set_b(float h, float l) {
    bh = h;
    bl = l;
  }
  __device__ __forceinline__ void load_b(const GridSlot* s) {
    bh = __ldcg(&s->bh);
    bl = __ldcg(&s->bl);
  }
  __device__ __forceinline__ DF b_acc() const { return DF{bh, bl}; }
};
static_assert(sizeof(GridSlot<double>) == sizeof(QrcpSlot) && sizeof(GridSlot<float>) == sizeof(QrcpSlot),
              "grid slots keep the QrcpSlot size");

constexpr int kQrcpLateTag = 48;  // int of a matrix's tag area raised when a wait expired

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void add_release(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T, int KG, bool SMEM>
__global__ void __launch_bounds__(kThreads, 1) qrcp_grid_kernel(const QrcpDesc<T>* descs, const QrcpGridDesc* gds,
                                                             int count, double eps, int nl_max, int m_max,
                                                             long long wait_cycles, int missing) {
  int f = 0;
  {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (gds[mid].cta0 <= (int)blockIdx.x)
        lo = mid;
      else
        hi = mid - 1;
    }
    f = lo;
  }
  const QrcpGridDesc gd = gds[f];
  const int G = gd.ctas;
  const int rank = (int)blockIdx.x - gd.cta0;
  const QrcpDesc<T> d = descs[f];
  const int m = d.m, n = d.n;
  const int nl = (n + G - 1) / G;
  const int j0 = min(n, rank * nl), j1 = min(n, j0 + nl);
  const int nloc = j1 - j0;
  const int vstride = (m_max + 3) & ~1;
  int* tags = gd.tags;                        // arrival counters of the two buffers, 128 bytes apart
  GridSlot<T>* slots = reinterpret_cast<GridSlot<T>*>(gd.slots);  // [2][G]
  T* vg = static_cast<T*>(gd.vg);             // [2][G][vstride]
  extern __shared__ __align__(16) unsigned char smraw[];
  using N = T;  // partial column norms and pivot proposals in the data's precision
  N* nu = reinterpret_cast<N*>(smraw);
  N* nuref = nu + nl_max;
  int* step_of = reinterpret_cast<int*>(nuref + nl_max);
  int* act = step_of + nl_max;
  int* pos = act + nl_max;
  T* vbuf = reinterpret_cast<T*>(smraw + (((size_t)nl_max * 28 + 15) / 16) * 16);  // 2 x vstride
  T* taus = vbuf + 2 * vstride;
  T* X = SMEM ? taus + vstride : d.work + (size_t)j0 * m;  // the slab, or this CTA's columns of the work copy
  __shared__ int s_nact, s_late;
  __shared__ N wb_v[kWarps];             // every warp's best (v, j) after an update
  __shared__ int wb_j[kWarps];
  __shared__ T red_h[kWarps], red_l[kWarps];  // partial sums of squares of the CTA's best column
  __shared__ GridSlot<T> wslot[kWarps];  // best slot among each warp's 32 (winner search)
  __shared__ T s_part[kWarps * KG];  // partial dot products (few-column apply)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t e = threadIdx.x; e < (int64_t)m * nloc; e += kThreads) {
    const int r = (int)(e % m), c = (int)(e / m);
    X[e] = d.src[r + (int64_t)(j0 + c) * d.ld];
  }
  __syncthreads();
  for (int c = warp; c < nloc; c += kWarps) {
    N sq = N(0);
    for (int r = lane; r < m; r += 32) {
      const N v = (N)X[r + (int64_t)c * m];
      sq += v * v;
    }
    sq = warp_sum(sq);
    if (lane == 0) {
      nu[c] = sq;
      nuref[c] = sq;
      step_of[c] = -1;
    }
  }
  for (int c = threadIdx.x; c < nloc; c += kThreads) {
    act[c] = c;
    pos[c] = c;
  }
  if (threadIdx.x == 0) {
    s_nact = nloc;
    s_late = 0;
  }
  const int kmax = m < n ? m : n;
  // eps and |R_11| in the arithmetic of the rank test (FP64, or double-float for FP32 data)
  using Acc = typename std::conditional<sizeof(T) == 8, double, DF>::type;
  Acc eps_x, r11;
  if constexpr (sizeof(T) == 8) {
    eps_x = eps;
    r11 = 0.0;
  } else {
    const float e_hi = (float)eps;
    eps_x = DF{e_hi, (float)(eps - (double)e_hi)};
    r11 = DF{0.f, 0.f};
  }
  int k = 0;
  __syncthreads();
  {  // proposals for step 0: every warp over its columns c = warp + kWarps * (lane + 32 t)
    N wv = N(-1);
    int wj = INT_MAX;
    for (int c = warp + lane * kWarps; c < nloc; c += 32 * kWarps)
      if (prop_better(nu[c], j0 + c, wv, wj)) {
        wv = nu[c];
        wj = j0 + c;
      }
    warp_argmax(wv, wj);
    if (lane == 0) {
      wb_v[warp] = wv;
      wb_j[warp] = wj;
    }
  }
  for (int i = 0; i < kmax; ++i) {
    const int par = i & 1;
    T* vb = vbuf + par * vstride;
    T* vmine = vg + ((size_t)par * G + rank) * vstride;
    GridSlot<T>* myslot = slots + (size_t)par * G + rank;
    __syncthreads();  // B1: the warps' proposals of step i
    // (1) the CTA's best column (every thread reduces the warps' proposals),
    // the sum of squares below row i of that column by all threads, then its
    // Householder data (every thread, the same arithmetic), its speculative
    // reflector into vb and the CTA's global buffer, its slot
    QrcpProp<T, N> best{N(-1), INT_MAX, T(0), T(0), T(0)};
    for (int w = 0; w < kWarps; ++w)
      if (prop_better(wb_v[w], wb_j[w], best.v, best.j)) {
        best.v = wb_v[w];
        best.j = wb_j[w];
      }
    if (best.j != INT_MAX) {
      const T* col = X + (int64_t)(best.j - j0) * m;
      SqSum<T> acc;
      for (int r = i + 1 + threadIdx.x; r < m; r += kThreads) acc.add(col[r]);
      T h, l;
      acc.warp_total(h, l);
      if (lane == 0) {
        red_h[warp] = h;
        red_l[warp] = l;
      }
    }
    __syncthreads();  // B1b
    if (best.j != INT_MAX) {
      T h = red_h[0], l = red_l[0];
      for (int w = 1; w < kWarps; ++w) sq_combine(h, l, red_h[w], red_l[w]);
      best.sh = h;
      best.sl = l;
      best.alpha = X[i + (int64_t)(best.j - j0) * m];
    }
    const int jloc = best.j;
    if (jloc != INT_MAX) {
      Acc r11c = r11;  // at step 0 the winner's |R_11| is known only after the exchange
      const HouseStep<T> hs = house_step(best.alpha, best.sh, best.sl, eps_x, r11c, i == 0);
      const T* col = X + (int64_t)(jloc - j0) * m;
      const T rden = hs.den != T(0) ? T(1) / hs.den : T(0);  // the reflector scaled by 1 / (alpha - beta)
      for (int r = i + 1 + threadIdx.x; r < m; r += kThreads) {
        const T x = col[r] * rden;
        vb[r - i] = x;
        vmine[r - i] = x;
      }
      if (threadIdx.x == 0) {
        vb[0] = T(1);
        vmine[0] = T(1);
        GridSlot<T> sl;
        sl.v = best.v;
        sl.beta = hs.beta;
        sl.tau = hs.tau;
        sl.set_b(hs.bh, hs.bl);
        sl.j = jloc;
        sl.stop = hs.stop ? 1 : 0;
        *myslot = sl;
      }
    } else if (threadIdx.x == 0) {
      GridSlot<T> sl;
      sl.v = N(-1);
      sl.beta = T(0);
      sl.tau = T(0);
      sl.set_b(T(0), T(0));
      sl.j = INT_MAX;
      sl.stop = 1;
      *myslot = sl;
    }
    // (2) publish: the CTA barrier orders every thread's stores before thread 0's
    // release increment of the step counter (cumulative at gpu scope); buffer
    // par counts G arrivals every second step
    __syncthreads();  // B2
    if (threadIdx.x == 0) {
      add_release(tags + 32 * par, 1);
      // (3) wait for every CTA of the matrix (bounded); the acquire load makes
      // the step's slots and reflectors visible to the CTA after the barrier
      const int target = G * (i / 2 + 1) + missing;  // missing > 0 only in failure-path tests
      const long long t0 = clock64();
      int spins = 0;
      while (ld_acquire(tags + 32 * par) < target) {
        if (((++spins) & 255) == 0 && clock64() - t0 > wait_cycles) {
          s_late = 1;
          break;
        }
      }
    }
    __syncthreads();  // B3
    if (s_late) {
      if (threadIdx.x == 0) {
        atomicExch(tags + kQrcpLateTag, 1);
        d.rank[0] = -1;
      }
      return;
    }
    // (4) the winner (lowest column index on ties): warp w loads slots
    // 32 w .. 32 w + 31 (one per lane, all in one round), keeps its best whole
    // slot; after a barrier every thread reduces those
    const int nsw = (G + 31) >> 5;
    if (warp < nsw) {
      const int t = (warp << 5) + lane;
      GridSlot<T> mine;
      mine.v = N(-1);
      mine.j = INT_MAX;
      if (t < G) {
        const GridSlot<T>* sl = slots + (size_t)par * G + t;
        mine.v = __ldcg(&sl->v);
        mine.j = __ldcg(&sl->j);
        mine.beta = __ldcg(&sl->beta);
        mine.tau = __ldcg(&sl->tau);
        mine.stop = __ldcg(&sl->stop);
        mine.load_b(sl);
      }
      N v = mine.v;
      int j = mine.j;
      const int who = warp_argmax(v, j);
      if (lane == who) wslot[warp] = mine;
    }
    __syncthreads();  // B3b
    int owner = -1;
    GridSlot<T> win;
    win.v = N(-1);
    win.j = INT_MAX;
    for (int w = 0; w < nsw; ++w)
      if (prop_better(wslot[w].v, wslot[w].j, win.v, win.j)) win = wslot[w];
    if (win.j != INT_MAX) owner = win.j / nl;  // CTA t holds columns [t nl, (t + 1) nl)
    if (owner < 0) break;  // no proposal (non-finite norms): every CTA sees the same
    if (i == 0) r11 = win.b_acc();
    if (win.stop) break;  // rank reached: the same decision everywhere
    const int p = win.j;
    if (rank != owner) {
      const T* vo = vg + ((size_t)par * G + owner) * vstride;
      for (int r = threadIdx.x; r < m - i; r += kThreads) vb[r] = __ldcg(vo + r);
    }
    const T tau = win.tau;
    if (threadIdx.x == 0) taus[i] = copysign(tau, win.beta);  // tau >= 0; the sign is that of R_ii
    if (rank == owner && threadIdx.x == 0) {
      const int pl = p - j0;
      const int q = pos[pl], last = act[s_nact - 1];
      step_of[pl] = i;
      act[q] = last;
      pos[last] = q;
      s_nact = s_nact - 1;
    }
    __syncthreads();  // B4: vb complete, act[] updated
    if (rank == owner) {  // the pivot column (out of act[]: no warp updates it)
      T* col = X + (int64_t)(p - j0) * m;
      for (int r = i + 1 + threadIdx.x; r < m; r += kThreads) col[r] = vb[r - i];
      if (threadIdx.x == 0) col[i] = win.beta;
    }
    // (6) apply H_i to the CTA's unpivoted columns.  Many columns: warps take
    // groups of KG columns as in the cluster kernel.  Few columns (at most four
    // groups): RS warps share a group, each over every RS-th 32-row block; the
    // partial dot products meet in shared memory, every warp of the group forms
    // the same w_j (same summation order) and updates its rows, and after a
    // barrier the group's first warp updates row i, the norms and the proposal.
    N wv = N(-1);
    int wj = INT_MAX;
    const int nact = s_nact;
    const int jl = butterfly_col<KG>(lane);
    const bool lead = lane == butterfly_lane<KG>(jl);
    const int ngrp = (nact + KG - 1) / KG;
    int RS = 1;
    if (ngrp > 0)
      while (RS * 2 * ngrp <= kWarps) RS *= 2;
    if (nact <= 2 * kWarps) {
      // at most two columns per warp: warp w updates columns act[w] and
      // act[w + kWarps] alone (lanes over rows, no CTA barrier), downdates
      // their norms and proposes the better one
      for (int q = warp; q < nact; q += kWarps) {
        const int cme = act[q];
        T* col = X + (int64_t)cme * m;
        // four rows per lane per iteration (independent loads and sums): with
        // one CTA per SM there are too few warps to hide shared-memory latency
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        int r = i + 1 + lane;
        if (tau != T(0)) {
          for (; r + 96 < m; r += 128) {
            a0 += vb[r - i] * col[r];
            a1 += vb[r + 32 - i] * col[r + 32];
            a2 += vb[r + 64 - i] * col[r + 64];
            a3 += vb[r + 96 - i] * col[r + 96];
          }
          for (; r < m; r += 32) a0 += vb[r - i] * col[r];
        }
        const T acc = warp_sum((a0 + a1) + (a2 + a3));
        const T xi = col[i];
        const T w = tau * (xi + acc);
        const N xnew = (N)(xi - w);
        if (tau != T(0)) {
          r = i + 1 + lane;
          for (; r + 96 < m; r += 128) {
            const T c0 = col[r], c1 = col[r + 32], c2 = col[r + 64], c3 = col[r + 96];
            col[r] = c0 - w * vb[r - i];
            col[r + 32] = c1 - w * vb[r + 32 - i];
            col[r + 64] = c2 - w * vb[r + 64 - i];
            col[r + 96] = c3 - w * vb[r + 96 - i];
          }
          for (; r < m; r += 32) col[r] -= w * vb[r - i];
        }
        __syncwarp();
        if (lane == 0) col[i] = (T)xnew;
        N v = nu[cme] - xnew * xnew;
        if (v < recompute_frac<N>() * nuref[cme]) {  // the same decision in every lane
          N sq = N(0);
          for (int r = i + 1 + lane; r < m; r += 32) {
            const N y = (N)col[r];
            sq += y * y;
          }
          v = warp_sum(sq);
          if (lane == 0) nuref[cme] = v;
        }
        if (lane == 0) nu[cme] = v;
        if (prop_better(v, j0 + cme, wv, wj)) {
          wv = v;
          wj = j0 + cme;
        }
      }
    } else if (RS == 1) {
      for (int g0 = warp * KG; g0 < nact; g0 += kWarps * KG) {
        const int ng = min(KG, nact - g0);
        T* cols[KG];
  #pragma unroll
        for (int j = 0; j < KG; ++j) cols[j] = X + (int64_t)act[g0 + (j < ng ? j : 0)] * m;
        T acc[KG];
  #pragma unroll
        for (int j = 0; j < KG; ++j) acc[j] = T(0);
        if (tau != T(0)) {
          for (int r = i + 1 + lane; r < m; r += 32) {
            const T vr = vb[r - i];
  #pragma unroll
            for (int j = 0; j < KG; ++j) acc[j] += vr * cols[j][r];
          }
        }
        const T dsum = butterfly_reduce<KG>(acc, lane);
        const int cme = jl < ng ? act[g0 + jl] : 0;
        T* colme = X + (int64_t)cme * m;
        T wmine = T(0);
        N xnew = N(0);
        if (jl < ng) {
          const T xi = colme[i];
          wmine = tau * (xi + dsum);
          xnew = (N)(xi - wmine);
        }
        T wv8[KG];
  #pragma unroll
        for (int j = 0; j < KG; ++j) wv8[j] = __shfl_sync(0xffffffffu, wmine, butterfly_lane<KG>(j));
        __syncwarp();
        if (lead && jl < ng) colme[i] = (T)xnew;
        if (tau != T(0)) {
          for (int r = i + 1 + lane; r < m; r += 32) {
            const T vr = vb[r - i];
  #pragma unroll
            for (int j = 0; j < KG; ++j)
              if (j < ng) cols[j][r] -= wv8[j] * vr;
          }
        }
        __syncwarp();
        N v = N(-1);
        bool redo = false;
        if (lead && jl < ng) {
          v = nu[cme] - xnew * xnew;
          redo = v < recompute_frac<N>() * nuref[cme];
        }
        unsigned flagged = __ballot_sync(0xffffffffu, redo);
        while (flagged) {
          const int l = __ffs(flagged) - 1;
          flagged &= flagged - 1;
          const int cc = __shfl_sync(0xffffffffu, cme, l);
          const T* col = X + (int64_t)cc * m;
          N sq = N(0);
          for (int r = i + 1 + lane; r < m; r += 32) {
            const N y = (N)col[r];
            sq += y * y;
          }
          sq = warp_sum(sq);
          if (lane == l) {
            v = sq;
            nuref[cc] = sq;
          }
        }
        if (lead && jl < ng) {
          nu[cme] = v;
          if (v > wv || (v == wv && j0 + cme < wj)) {
            wv = v;
            wj = j0 + cme;
          }
        }
      }
    } else {
      const int cg = warp / RS, rs = warp % RS;
      const bool active = cg < ngrp;
      const int g0 = cg * KG;
      const int ng = active ? min(KG, nact - g0) : 0;
      T* cols[KG];
#pragma unroll
      for (int j = 0; j < KG; ++j) cols[j] = X + (int64_t)act[active ? g0 + (j < ng ? j : 0) : 0] * m;
      T acc[KG];
#pragma unroll
      for (int j = 0; j < KG; ++j) acc[j] = T(0);
      if (active && tau != T(0)) {
        for (int r = i + 1 + lane + 32 * rs; r < m; r += 32 * RS) {
          const T vr = vb[r - i];
#pragma unroll
          for (int j = 0; j < KG; ++j) acc[j] += vr * cols[j][r];
        }
      }
      const T dpart = butterfly_reduce<KG>(acc, lane);
      if (active && lead && jl < ng) s_part[(g0 + jl) * RS + rs] = dpart;
      __syncthreads();
      const int cme = (active && jl < ng) ? act[g0 + jl] : 0;
      T* colme = X + (int64_t)cme * m;
      T wmine = T(0);
      N xnew = N(0);
      if (active && jl < ng) {
        T dsum = T(0);
        for (int q = 0; q < RS; ++q) dsum += s_part[(g0 + jl) * RS + q];
        const T xi = colme[i];
        wmine = tau * (xi + dsum);
        xnew = (N)(xi - wmine);
      }
      T wv8[KG];
#pragma unroll
      for (int j = 0; j < KG; ++j) wv8[j] = __shfl_sync(0xffffffffu, wmine, butterfly_lane<KG>(j));
      if (active && tau != T(0)) {
        for (int r = i + 1 + lane + 32 * rs; r < m; r += 32 * RS) {
          const T vr = vb[r - i];
#pragma unroll
          for (int j = 0; j < KG; ++j)
            if (j < ng) cols[j][r] -= wv8[j] * vr;
        }
      }
      __syncthreads();  // every row slice is updated before row i and the norms
      if (active && rs == 0) {
        if (lead && jl < ng) colme[i] = (T)xnew;
        N v = N(-1);
        bool redo = false;
        if (lead && jl < ng) {
          v = nu[cme] - xnew * xnew;
          redo = v < recompute_frac<N>() * nuref[cme];
        }
        unsigned flagged = __ballot_sync(0xffffffffu, redo);
        while (flagged) {
          const int l = __ffs(flagged) - 1;
          flagged &= flagged - 1;
          const int cc = __shfl_sync(0xffffffffu, cme, l);
          const T* col = X + (int64_t)cc * m;
          N sq = N(0);
          for (int r = i + 1 + lane; r < m; r += 32) {
            const N y = (N)col[r];
            sq += y * y;
          }
          sq = warp_sum(sq);
          if (lane == l) {
            v = sq;
            nuref[cc] = sq;
          }
        }
        if (lead && jl < ng) {
          nu[cme] = v;
          if (v > wv || (v == wv && j0 + cme < wj)) {
            wv = v;
            wj = j0 + cme;
          }
        }
      }
    }
    // the warp's proposal for step i + 1 (every thread is past B1b: wb_* of step i are read)
    warp_argmax(wv, wj);
    if (lane == 0) {
      wb_v[warp] = wv;
      wb_j[warp] = wj;
    }
    k = i + 1;
  }
  __syncthreads();
  // a CTA whose wait expired has written rank -1; keep it
  if (rank == 0 && threadIdx.x == 0 && ld_acquire(tags + kQrcpLateTag) == 0) d.rank[0] = k;
  if (d.V) {
    for (int64_t e = threadIdx.x; e < (int64_t)m * nloc; e += kThreads) {
      const int r = (int)(e % m), c = (int)(e / m);
      const int t = step_of[c];
      if (t < 0 || t >= k) continue;
      d.V[r + (int64_t)t * m] = r < t ? T(0) : (r == t ? T(1) : X[r + (int64_t)c * m]);
    }
    if (rank == 0)
      for (int t = threadIdx.x; t < k; t += kThreads) d.tau[t] = fabs(taus[t]);
  }
  if (d.out && (k < m || (d.flags & kQrcpAlwaysOut))) {
    const bool fix = d.flags & kQrcpSignFix;
    for (int64_t e = threadIdx.x; e < (int64_t)k * nloc; e += kThreads) {
      const int r = (int)(e % k), c = (int)(e / k);
      const int t = step_of[c];
      const T x = (t >= 0 && r > t) ? T(0) : X[r + (int64_t)c * m];
      d.out[r + (int64_t)(j0 + c) * d.ldo] = fix && signbit(taus[r]) ? -x : x;
    }
  }
}

// --------------------------------------------- QRCP with delayed updates
// The global-work variant (slabs too large for shared memory): the pivots,
// reflectors and rank rule of qrcp_slab_kernel, but the reflectors of a
// panel of up to kQrcpNB steps reach the unpivoted columns only at the end of
// the panel, as one rank-kQrcpNB update.  Within a panel each step reads every
// unpivoted column once (v^T a) and keeps per column the coefficients f_t of
// a_upd = a - sum_t v_t f_t, with f_j = tau_j (v_j^T a - sum_{t<j} (v_t^T v_j) f_t)
// (the delayed-update form of column-pivoted Householder QR; Quintana-Orti,
// Sun and Bischof, 1998).  The pivot column is brought up to date before its
// reflector is formed, and the row-i entries that the norm downdates need are
// formed from the coefficients.  Reflector storage: the pivot columns of the
// shared work copy, read by every CTA of the cluster.
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads, 1) qrcp_delayed_kernel(const QrcpDesc<T>* descs, double eps, int nl_max,
                                                                int m_max) {
  constexpr int KG = 8;
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const QrcpDesc<T> d = descs[blockIdx.x / CS];
  const int m = d.m, n = d.n;
  const int nl = (n + CS - 1) / CS;
  const int j0 = min(n, rank * nl), j1 = min(n, j0 + nl);
  const int nloc = j1 - j0;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* nu = reinterpret_cast<double*>(smraw);
  double* nuref = nu + nl_max;
  int* step_of = reinterpret_cast<int*>(nuref + nl_max);
  int* act = step_of + nl_max;
  int* pos = act + nl_max;
  T* F = reinterpret_cast<T*>(smraw + (((size_t)nl_max * 28 + 15) / 16) * 16);  // NB coefficients per column
  T* cbuf = F + (size_t)nl_max * NB;    // rows i0..m-1: owner's pivot column, then the reflector (m_max + 2)
  T* taus = cbuf + ((m_max + 3) & ~1);  // kmax + 2
  T* W = d.work;                        // the whole matrix, ld m
  T* X = W + (size_t)j0 * m;            // this CTA's columns
  __shared__ double cand_v;
  __shared__ int cand_j;
  __shared__ double s_beta;
  __shared__ T s_tau;
  __shared__ int s_stop, s_piv, s_nact;
  __shared__ double red_v[kWarps];
  __shared__ int red_i[kWarps];
  __shared__ int piv[NB];  // global column of each reflector of the panel
  __shared__ T gco[NB];    // v_t^T v_j for the panel's earlier reflectors t
  __shared__ T gred[kWarps * NB];
  __shared__ T s_den;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t e = threadIdx.x; e < (int64_t)m * nloc; e += kThreads) {
    const int r = (int)(e % m), c = (int)(e / m);
    X[e] = d.src[r + (int64_t)(j0 + c) * d.ld];
  }
  __syncthreads();
  for (int c = warp; c < nloc; c += kWarps) {
    double sq = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double v = (double)X[r + (int64_t)c * m];
      sq += v * v;
    }
    sq = warp_sum(sq);
    if (lane == 0) {
      nu[c] = sq;
      nuref[c] = sq;
      step_of[c] = -1;
    }
  }
  for (int c = threadIdx.x; c < nloc; c += kThreads) {
    act[c] = c;
    pos[c] = c;
  }
  if (threadIdx.x == 0) s_nact = nloc;
  for (int e = threadIdx.x; e < nl_max * NB; e += kThreads) F[e] = T(0);
  const int kmax = m < n ? m : n;
  double r11 = 0.0;
  int k = 0;
  __syncthreads();
  double wv = -1.0;
  int wj = INT_MAX;
  for (int c = warp + lane * kWarps; c < nloc; c += 32 * kWarps) {
    const double v = nu[c];
    if (v > wv || (v == wv && j0 + c < wj)) {
      wv = v;
      wj = j0 + c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, wv, o);
    const int oj = __shfl_xor_sync(0xffffffffu, wj, o);
    if (ov > wv || (ov == wv && oj < wj)) {
      wv = ov;
      wj = oj;
    }
  }
  // a_c <- a_c - sum_{t<nb} V[:, t] F[c, t] over rows i0..m-1 for every unpivoted
  // column: thread per row, V[r, 0:NB] in registers, F[c, :] read as vectors
  auto block_update = [&](int i0, int nb) {
    __syncthreads();
    const int nact = s_nact;
    for (int r = i0 + threadIdx.x; r < m; r += kThreads) {
      T vr[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t)
        vr[t] = (t >= nb || r < i0 + t) ? T(0) : (r == i0 + t ? T(1) : __ldcg(W + r + (int64_t)piv[t] * m));
      // four columns per pass: their loads are issued before any store
      int q = 0;
      for (; q + 3 < nact; q += 4) {
        T* p4[4];
        T a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          p4[u] = X + r + (int64_t)act[q + u] * m;
          a[u] = *p4[u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const T* Fc = F + (size_t)act[q + u] * NB;
#pragma unroll
          for (int t = 0; t < NB; ++t) a[u] -= vr[t] * Fc[t];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) *p4[u] = a[u];
      }
      for (; q < nact; ++q) {
        const int c = act[q];
        const T* Fc = F + (size_t)c * NB;
        T a = X[r + (int64_t)c * m];
#pragma unroll
        for (int t = 0; t < NB; ++t) a -= vr[t] * Fc[t];
        X[r + (int64_t)c * m] = a;
      }
    }
    __syncthreads();
  };
  int i0 = 0, jj = 0;
  for (int i = 0; i < kmax; ++i) {
    if (lane == 0) {
      red_v[warp] = wv;
      red_i[warp] = wj;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = red_v[0];
      int j = red_i[0];
      for (int w = 1; w < kWarps; ++w)
        if (red_v[w] > v || (red_v[w] == v && red_i[w] < j)) {
          v = red_v[w];
          j = red_i[w];
        }
      cand_v = v;
      cand_j = j;
    }
    cl.sync();  // (A) proposals visible cluster-wide
    if (threadIdx.x < 32) {
      double v = -1.0;
      int j = INT_MAX;
      if (lane < CS) {
        v = *cl.map_shared_rank(&cand_v, lane);
        j = *cl.map_shared_rank(&cand_j, lane);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (ov > v || (ov == v && oj < j)) {
          v = ov;
          j = oj;
        }
      }
      if (lane == 0) s_piv = j;
    }
    __syncthreads();
    const int p = s_piv;
    if (p == INT_MAX) break;
    const int owner = p / nl;
    if (rank == owner) {
      // the pivot column brought up to date over rows i0..m-1 (into cbuf)
      const int pl = p - j0;
      T* col = X + (int64_t)pl * m;
      const T* Fp = F + (size_t)pl * NB;
      for (int r = i0 + threadIdx.x; r < m; r += kThreads) {
        T a = col[r];
        for (int t = 0; t < jj && r >= i0 + t; ++t) {
          const T vrt = r == i0 + t ? T(1) : __ldcg(W + r + (int64_t)piv[t] * m);
          a -= vrt * Fp[t];
        }
        cbuf[r - i0] = a;
      }
      __syncthreads();
      T* cv = cbuf + (i - i0);  // cv[r - i], rows i..m-1
      {
        // squared norm below the diagonal: the whole CTA, then one thread forms the reflector
        double sq = 0.0;
        for (int r = i + 1 + threadIdx.x; r < m; r += kThreads) {
          const double v = (double)cv[r - i];
          sq += v * v;
        }
        sq = warp_sum(sq);
        if (lane == 0) red_v[warp] = sq;
        __syncthreads();
        if (threadIdx.x == 0) {
          double sig = 0.0;
          for (int w = 0; w < kWarps; ++w) sig += red_v[w];
          const double alpha = (double)cv[0];
          double beta, tau;
          if (sig == 0.0) {
            beta = alpha;
            tau = 0.0;
          } else {
            const double nrm = sqrt(alpha * alpha + sig);
            beta = alpha >= 0.0 ? -nrm : nrm;
            tau = (beta - alpha) / beta;
          }
          const double ab = fabs(beta);
          const double r11_here = (i == 0) ? ab : r11;
          const int stop = (beta == 0.0 || ab < eps * r11_here) ? 1 : 0;
          s_tau = (T)tau;
          s_beta = beta;
          s_stop = stop;
          s_den = (!stop && sig != 0.0) ? (T)(alpha - beta) : T(0);
        }
        __syncthreads();
        const T den = s_den;
        for (int r = i + 1 + threadIdx.x; r < m; r += kThreads) cv[r - i] = den != T(0) ? cv[r - i] / den : T(0);
      }
      __syncthreads();
      if (!s_stop) {
        // rows i0..i-1: R entries; row i: beta; below: the reflector
        for (int r = i0 + threadIdx.x; r < m; r += kThreads) col[r] = r == i ? (T)s_beta : cbuf[r - i0];
      }
      __syncthreads();
      if (threadIdx.x == 0) cv[0] = T(1);
    }
    cl.sync();  // (C) reflector ready (owner's cbuf and the work copy)
    if (rank != owner) {
      for (int r = i + threadIdx.x; r < m; r += kThreads) cbuf[r - i0] = *cl.map_shared_rank(cbuf + (r - i0), owner);
      if (threadIdx.x == 0) {
        s_tau = *cl.map_shared_rank(&s_tau, owner);
        s_beta = *cl.map_shared_rank(&s_beta, owner);
        s_stop = *cl.map_shared_rank(&s_stop, owner);
      }
    }
    __syncthreads();
    if (i == 0) r11 = fabs(s_beta);
    if (s_stop) break;
    const T tau = s_tau;
    if (threadIdx.x == 0) {
      taus[i] = copysign(tau, (T)s_beta);  // tau >= 0; the sign is that of R_ii
      piv[jj] = p;
    }
    if (rank == owner && threadIdx.x == 0) {
      const int pl = p - j0, q = pos[pl], last = act[s_nact - 1];
      step_of[pl] = i;
      act[q] = last;
      pos[last] = q;
      s_nact = s_nact - 1;
    }
    // g_t = v_t^T v_i (rows i..m-1) for the panel's earlier reflectors: one pass
    // over the rows for all t (independent loads), then a CTA reduction per t
    if (jj > 0) {
      T gacc[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) gacc[t] = T(0);
      for (int r = i + threadIdx.x; r < m; r += kThreads) {
        const T vr = cbuf[r - i0];
#pragma unroll
        for (int t = 0; t < NB; ++t)
          if (t < jj) gacc[t] += __ldcg(W + r + (int64_t)piv[t] * m) * vr;
      }
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        if (t >= jj) break;
        const T v = warp_sum(gacc[t]);
        if (lane == 0) gred[warp * NB + t] = v;
      }
      __syncthreads();
      if (threadIdx.x < jj) {
        T v = T(0);
        for (int w = 0; w < kWarps; ++w) v += gred[w * NB + threadIdx.x];
        gco[threadIdx.x] = v;
      }
    }
    __syncthreads();
    // every unpivoted column: v^T a (stale a), its coefficient f, its row-i entry, the norm downdate
    wv = -1.0;
    wj = INT_MAX;
    const int nact = s_nact;
    const int jl = butterfly_col<KG>(lane);
    const bool lead = lane == butterfly_lane<KG>(jl);
    const T* vcur = cbuf + (i - i0);  // vcur[r - i]
    for (int g0 = warp * KG; g0 < nact; g0 += kWarps * KG) {
      const int ng = min(KG, nact - g0);
      const T* cols[KG];
#pragma unroll
      for (int j = 0; j < KG; ++j) cols[j] = X + (int64_t)act[g0 + (j < ng ? j : 0)] * m;
      T acc[KG];
#pragma unroll
      for (int j = 0; j < KG; ++j) acc[j] = T(0);
      if (tau != T(0)) {
        // four rows per lane per pass: 4 x KG independent loads in flight
        int r = i + lane;
        for (; r + 96 < m; r += 128) {
          T vr[4], x[4][KG];
#pragma unroll
          for (int u = 0; u < 4; ++u) vr[u] = vcur[r + 32 * u - i];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < KG; ++j) x[u][j] = cols[j][r + 32 * u];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < KG; ++j) acc[j] += vr[u] * x[u][j];
        }
        for (; r < m; r += 32) {
          const T vr = vcur[r - i];
#pragma unroll
          for (int j = 0; j < KG; ++j) acc[j] += vr * cols[j][r];
        }
      }
      const T dsum = butterfly_reduce<KG>(acc, lane);
      const int cme = jl < ng ? act[g0 + jl] : 0;
      double v = -1.0;
      bool redo = false;
      if (lead && jl < ng) {
        T* Fc = F + (size_t)cme * NB;
        T corr = T(0);
        for (int t = 0; t < jj; ++t) corr += gco[t] * Fc[t];
        const T f = tau * (dsum - corr);
        Fc[jj] = f;
        T xi = X[i + (int64_t)cme * m];
        for (int t = 0; t < jj; ++t) xi -= __ldcg(W + i + (int64_t)piv[t] * m) * Fc[t];
        xi -= f;
        const double x = (double)xi;
        v = nu[cme] - x * x;
        redo = v < kRecompute * nuref[cme];
      }
      unsigned flagged = __ballot_sync(0xffffffffu, redo);
      while (flagged) {
        const int l = __ffs(flagged) - 1;
        flagged &= flagged - 1;
        const int cc = __shfl_sync(0xffffffffu, cme, l);
        const T* col = X + (int64_t)cc * m;
        const T* Fc = F + (size_t)cc * NB;
        double sq = 0.0;
        for (int r = i + 1 + lane; r < m; r += 32) {
          T a = col[r] - vcur[r - i] * Fc[jj];
          for (int t = 0; t < jj; ++t) a -= __ldcg(W + r + (int64_t)piv[t] * m) * Fc[t];
          const double y = (double)a;
          sq += y * y;
        }
        sq = warp_sum(sq);
        if (lane == l) {
          v = sq;
          nuref[cc] = sq;
        }
      }
      if (lead && jl < ng) {
        nu[cme] = v;
        if (v > wv || (v == wv && j0 + cme < wj)) {
          wv = v;
          wj = j0 + cme;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, wv, o);
      const int oj = __shfl_xor_sync(0xffffffffu, wj, o);
      if (ov > wv || (ov == wv && oj < wj)) {
        wv = ov;
        wj = oj;
      }
    }
    k = i + 1;
    if (++jj == NB) {
      block_update(i0, jj);
      i0 = i + 1;
      jj = 0;
    }
  }
  if (jj > 0) block_update(i0, jj);
  __syncthreads();
  if (rank == 0 && threadIdx.x == 0) d.rank[0] = k;
  if (d.V) {
    for (int64_t e = threadIdx.x; e < (int64_t)m * nloc; e += kThreads) {
      const int r = (int)(e % m), c = (int)(e / m);
      const int t = step_of[c];
      if (t < 0 || t >= k) continue;
      d.V[r + (int64_t)t * m] = r < t ? T(0) : (r == t ? T(1) : X[r + (int64_t)c * m]);
    }
    if (rank == 0)
      for (int t = threadIdx.x; t < k; t += kThreads) d.tau[t] = fabs(taus[t]);
  }
  if (d.out && (k < m || (d.flags & kQrcpAlwaysOut))) {
    const bool fix = d.flags & kQrcpSignFix;
    for (int64_t e = threadIdx.x; e < (int64_t)k * nloc; e += kThreads) {
      const int r = (int)(e % k), c = (int)(e / k);
      const int t = step_of[c];
      const T x = (t >= 0 && r > t) ? T(0) : X[r + (int64_t)c * m];
      d.out[r + (int64_t)(j0 + c) * d.ldo] = fix && signbit(taus[r]) ? -x : x;
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// ----------------------------------------------------- QRCP, one warp each
// The same swap-free column-pivoted QR for small matrices: every warp owns one
// matrix in its shared-memory region (ld = m | 1), lanes own columns for the
// norms, the pivot search and the reflector application; no block barriers.
template <typename T>
__global__ void __launch_bounds__(kThreads) qrcp_warp_kernel(const QrcpDesc<T>* descs, int count, double eps,
                                                             int per_warp_bytes) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * kWarps + warp;
  if (f >= count) return;
  const QrcpDesc<T> d = descs[f];
  const int m = d.m, n = d.n, ld = m | 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* base = smraw + (size_t)warp * per_warp_bytes;
  double* nu = reinterpret_cast<double*>(base);
  double* nuref = nu + n;
  int* step_of = reinterpret_cast<int*>(nuref + n);
  T* taus = reinterpret_cast<T*>(base + (((size_t)n * 20 + 15) / 16) * 16);
  const int kmax = m < n ? m : n;
  T* X = taus + ((kmax + 3) & ~1);
  for (int c = 0; c < n; ++c)
    for (int r = lane; r < m; r += 32) X[r + c * ld] = d.src[r + (int64_t)c * d.ld];
  __syncwarp();
  for (int c = lane; c < n; c += 32) {
    double sq = 0.0;
    for (int r = 0; r < m; ++r) {
      const double v = (double)X[r + c * ld];
      sq += v * v;
    }
    nu[c] = sq;
    nuref[c] = sq;
    step_of[c] = -1;
  }
  __syncwarp();
  double r11 = 0.0;
  int k = 0;
  for (int i = 0; i < kmax; ++i) {
    double bv = -1.0;
    int bj = INT_MAX;
    for (int c = lane; c < n; c += 32) {
      if (step_of[c] >= 0) continue;
      if (nu[c] > bv) {
        bv = nu[c];
        bj = c;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ov > bv || (ov == bv && oj < bj)) {
        bv = ov;
        bj = oj;
      }
    }
    const int p = bj;
    if (p == INT_MAX) break;  // no proposal (non-finite norms)
    T* col = X + p * ld;
    double sig = 0.0;
    for (int r = i + 1 + lane; r < m; r += 32) {
      const double v = (double)col[r];
      sig += v * v;
    }
    sig = warp_sum(sig);
    const double alpha = (double)col[i];
    double beta, tau;
    if (sig == 0.0) {
      beta = alpha;
      tau = 0.0;
    } else {
      const double nrm = sqrt(alpha * alpha + sig);
      beta = alpha >= 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
    }
    const double ab = fabs(beta);
    if (i == 0) r11 = ab;
    if (beta == 0.0 || ab < eps * r11) break;
    if (sig != 0.0) {
      const T den = (T)(alpha - beta);
      for (int r = i + 1 + lane; r < m; r += 32) col[r] = col[r] / den;
    }
    __syncwarp();
    if (lane == 0) {
      col[i] = (T)beta;
      taus[i] = copysign((T)tau, (T)beta);  // tau >= 0; the sign is that of R_ii
      step_of[p] = i;
    }
    __syncwarp();
    const T tt = (T)tau;
    for (int c = lane; c < n; c += 32) {
      if (step_of[c] >= 0) continue;
      T* x = X + c * ld;
      if (tt != T(0)) {
        T sacc = x[i];
        for (int r = i + 1; r < m; ++r) sacc += col[r] * x[r];
        const T w = tt * sacc;
        x[i] -= w;
        for (int r = i + 1; r < m; ++r) x[r] -= w * col[r];
      }
      const double xv = (double)x[i];
      double v = nu[c] - xv * xv;
      if (v < kRecompute * nuref[c]) {
        v = 0.0;
        for (int r = i + 1; r < m; ++r) {
          const double y = (double)x[r];
          v += y * y;
        }
        nuref[c] = v;
      }
      nu[c] = v;
    }
    __syncwarp();
    k = i + 1;
  }
  __syncwarp();
  if (lane == 0) d.rank[0] = k;
  if (d.V) {
    for (int c = 0; c < n; ++c) {
      const int t = step_of[c];
      if (t < 0 || t >= k) continue;
      for (int r = lane; r < m; r += 32)
        d.V[r + (int64_t)t * m] = r < t ? T(0) : (r == t ? T(1) : X[r + c * ld]);
    }
    for (int t = lane; t < k; t += 32) d.tau[t] = fabs(taus[t]);
  }
  if (d.out && (k < m || (d.flags & kQrcpAlwaysOut))) {
    const bool fix = d.flags & kQrcpSignFix;
    for (int c = 0; c < n; ++c) {
      const int t = step_of[c];
      for (int r = lane; r < k; r += 32) {
        const T x = (t >= 0 && r > t) ? T(0) : X[r + c * ld];
        d.out[r + (int64_t)c * d.ldo] = fix && signbit(taus[r]) ? -x : x;
      }
    }
  }
}

// ------------------------------------------------------ reflector applies
// Row vectors (mode 0, rows of a block with leading dimension ld): one thread
// per row, the reflectors in blocks of kWyB as I - V T V^T (compact WY form;
// T from the block's Gram matrix, as in the front panels): w = V^T x,
// w' = T^T w, x <- x - V w', with V staged in shared memory in chunks of rows
// (the rows' entries are read coalesced across threads; 2 kWyB flops per
// entry and pass instead of a warp reduction per reflector).
constexpr int kWyB = 32;
constexpr int kWyChunk = 64;
template <typename T>
__device__ void refl_rows_blocked(const ReflDesc<T>& d, int k, int row0) {
  __shared__ T Vs[kWyChunk][kWyB + 1];
  __shared__ T Gs[kWyB][kWyB + 1];  // the block's Gram matrix, then T in place
  __shared__ T tcol[kWyB];
  const int len = d.len;
  const int r = row0 + (int)threadIdx.x;
  const bool live = r < d.nvec;
  T* x = d.ptr + (live ? r : 0);  // entry l at x[l * ld]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto stage = [&](int i0, int nb, int l0, int nl) {  // V rows l0.., reflectors i0.. (unit lower)
    for (int e = threadIdx.x; e < kWyChunk * kWyB; e += kThreads) {
      const int ll = e % kWyChunk, q = e / kWyChunk;
      const int l = l0 + ll, i = i0 + q;
      T v = T(0);
      if (ll < nl && q < nb) v = l < i ? T(0) : (l == i ? T(1) : d.V[l + (int64_t)i * len]);
      Vs[ll][q] = v;
    }
  };
  for (int i0 = 0; i0 < k; i0 += kWyB) {
    const int nb = min(kWyB, k - i0);
    T w[kWyB];
#pragma unroll
    for (int q = 0; q < kWyB; ++q) w[q] = T(0);
    T g4[4] = {T(0), T(0), T(0), T(0)};  // Gram entries (lane, warp + 8 j)
    for (int l0 = i0; l0 < len; l0 += kWyChunk) {
      const int nl = min(kWyChunk, len - l0);
      __syncthreads();
      stage(i0, nb, l0, nl);
      __syncthreads();
      for (int ll = 0; ll < nl; ++ll) {
#pragma unroll
        for (int j = 0; j < 4; ++j) g4[j] += Vs[ll][lane] * Vs[ll][warp + 8 * j];
      }
      if (live)
        for (int ll = 0; ll < nl; ++ll) {
          const T xl = x[(int64_t)(l0 + ll) * d.ld];
#pragma unroll
          for (int q = 0; q < kWyB; ++q) w[q] += xl * Vs[ll][q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) Gs[lane][warp + 8 * j] = g4[j];
    __syncthreads();
    if (warp == 0) {  // T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i], in place over G
      for (int i = 0; i < kWyB; ++i) {
        const T tau_i = i < nb ? d.tau[i0 + i] : T(0);
        tcol[lane] = lane < i ? Gs[lane][i] : T(0);
        __syncwarp();
        T acc = T(0);
        if (lane < i)
          for (int qq = lane; qq < i; ++qq) acc += Gs[lane][qq] * tcol[qq];
        __syncwarp();
        Gs[lane][i] = lane < i ? -tau_i * acc : (lane == i ? tau_i : T(0));
        __syncwarp();
      }
    }
    __syncthreads();
    T w2[kWyB];  // T^T w
#pragma unroll
    for (int q = 0; q < kWyB; ++q) {
      T acc = T(0);
#pragma unroll
      for (int p = 0; p <= q; ++p) acc += Gs[p][q] * w[p];
      w2[q] = acc;
    }
    for (int l0 = i0; l0 < len; l0 += kWyChunk) {
      const int nl = min(kWyChunk, len - l0);
      __syncthreads();
      stage(i0, nb, l0, nl);
      __syncthreads();
      if (live)
        for (int ll = 0; ll < nl; ++ll) {
          T xl = x[(int64_t)(l0 + ll) * d.ld];
#pragma unroll
          for (int q = 0; q < kWyB; ++q) xl -= Vs[ll][q] * w2[q];
          x[(int64_t)(l0 + ll) * d.ld] = xl;
        }
    }
  }
  if (live)
    for (int l = k; l < len; ++l) x[(int64_t)l * d.ld] = T(0);
}

// Column vectors (mode 1, contiguous), and every vector in FP64: one warp per
// vector, lanes over its entries, the reflectors one after the other.  FP32
// row vectors take the blocked path above (items of kReflRowsPerItem rows).
template <typename T>
__global__ void __launch_bounds__(kThreads) refl_kernel(const ReflDesc<T>* descs, const int2* items) {
  const int2 it = items[blockIdx.x];  // (descriptor, first vector)
  const ReflDesc<T> d = descs[it.x];
  const int k = *d.k;
  const int len = d.len;
  if (k >= len) return;  // the same for the whole CTA
  if constexpr (sizeof(T) == 4) {
    if (d.mode == 0) {
      refl_rows_blocked(d, k, it.y);
      return;
    }
  }
  // one warp per vector (FP64 rows too: the blocked form is bound by the FP64
  // pipe, the per-reflector form was measured faster there)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vec = it.y + warp;
  if (vec >= d.nvec) return;
  const int64_t sl = d.mode == 0 ? d.ld : 1;  // stride between a vector's entries
  T* y = d.ptr + (d.mode == 0 ? (int64_t)vec : (int64_t)vec * d.ld);
  for (int i = 0; i < k; ++i) {
    const T* v = d.V + (int64_t)i * len;
    T s = T(0);
    for (int l = i + lane; l < len; l += 32) s += y[l * sl] * (l == i ? T(1) : v[l]);
    s = warp_sum(s) * d.tau[i];
    for (int l = i + lane; l < len; l += 32) y[l * sl] -= s * (l == i ? T(1) : v[l]);
  }
  for (int l = k + lane; l < len; l += 32) y[l * sl] = T(0);
}

// ---------------------------------------------------------- X <- X R^{-1}
// One thread per row of X, the columns in blocks of 32: a block's 32 entries
// are accumulated in registers, first minus the solved blocks times the
// matching tiles of R (staged in shared memory, shared by the CTA's rows),
// then solved against the block's diagonal triangle.
constexpr int kTrsmB = 32;
template <typename T>
__global__ void __launch_bounds__(kThreads) trsm_kernel(const TrsmDesc<T>* descs, const int2* items) {
  const int2 it = items[blockIdx.x];  // (descriptor, first row)
  const TrsmDesc<T> d = descs[it.x];
  const int r = it.y + threadIdx.x;
  if constexpr (sizeof(T) == 8) {
    // FP64: column by column (the blocked form is bound by the FP64 pipe and
    // was measured slower)
    if (r >= d.rows) return;
    T* x = d.ptr + r;
    for (int j = 0; j < d.c; ++j) {
      const T* Rj = d.R + (int64_t)j * d.rld;
      T s = x[(int64_t)j * d.ld];
      for (int i = 0; i < j; ++i) s -= x[(int64_t)i * d.ld] * Rj[i];
      x[(int64_t)j * d.ld] = s / Rj[j];
    }
    return;
  }
  const bool live = r < d.rows;
  __shared__ T Rt[kTrsmB][kTrsmB + 1];  // Rt[i][k] = R[i0 + i, j0 + k]
  T* x = d.ptr + (live ? r : 0);
  for (int j0 = 0; j0 < d.c; j0 += kTrsmB) {
    const int nb = min(kTrsmB, d.c - j0);
    T s[kTrsmB];
#pragma unroll
    for (int k = 0; k < kTrsmB; ++k) s[k] = (live && k < nb) ? x[(int64_t)(j0 + k) * d.ld] : T(0);
    for (int i0 = 0; i0 < j0; i0 += kTrsmB) {  // s_k -= x_i R[i, j0 + k] over the solved blocks
      __syncthreads();
      for (int e = threadIdx.x; e < kTrsmB * kTrsmB; e += kThreads) {
        const int i = e % kTrsmB, k = e / kTrsmB;
        Rt[i][k] = k < nb ? d.R[(i0 + i) + (int64_t)(j0 + k) * d.rld] : T(0);
      }
      __syncthreads();
      if (live) {
#pragma unroll 4
        for (int i = 0; i < kTrsmB; ++i) {
          const T xi = x[(int64_t)(i0 + i) * d.ld];
#pragma unroll
          for (int k = 0; k < kTrsmB; ++k) s[k] -= xi * Rt[i][k];
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kTrsmB * kTrsmB; e += kThreads) {
      const int i = e % kTrsmB, k = e / kTrsmB;
      Rt[i][k] = (i < nb && k < nb) ? d.R[(j0 + i) + (int64_t)(j0 + k) * d.rld] : T(1);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTrsmB; ++k) {  // the diagonal triangle: s[i], i < k, already solved
      T v = s[k];
#pragma unroll
      for (int i = 0; i < k; ++i) v -= s[i] * Rt[i][k];
      s[k] = v / Rt[k][k];
    }
    if (live)
#pragma unroll
      for (int k = 0; k < kTrsmB; ++k)
        if (k < nb) x[(int64_t)(j0 + k) * d.ld] = s[k];
  }
}

// ----------------------------------------------------- max-norm row rule
template <typename T>
__global__ void __launch_bounds__(kThreads) argmax_kernel(const ArgmaxDesc<T>* descs, const int2* items) {
  const int2 it = items[blockIdx.x];  // (descriptor, first row offset)
  const ArgmaxDesc<T> d = descs[it.x];
  const int r = d.r0 + it.y + threadIdx.x;
  if (r >= d.r1) return;
  double best = -1.0;
  int bl = -1, bid = 0x7fffffff, bt = -1;
  for (int t = 0; t < d.ncl; ++t) {
    if (d.lvl[t] < 0) continue;  // not a candidate
    double s = 0.0;
    for (int c = d.coff[t]; c < d.coff[t + 1]; ++c) {
      const double v = (double)d.F[r + (int64_t)c * d.ld];
      s += v * v;
    }
    const int lv = d.lvl[t], id = d.cid[t];
    if (s > best || (s == best && (lv > bl || (lv == bl && id < bid)))) {
      best = s;
      bl = lv;
      bid = id;
      bt = t;
    }
  }
  d.out[r - d.r0] = bt;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) scatter_values_kernel(T* base, const int64_t* dest, const T* vals, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (e < n) base[dest[e]] = vals[e];
}

// Raise the kernel's dynamic shared-memory limit to the opt-in maximum minus
// its static shared memory (the two together may not exceed the opt-in size).
template <typename K>
void allow_smem(K kernel) {
  int dev = 0;
  cudaGetDevice(&dev);
  int mx = 0;
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, kernel);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
}

}  // namespace

int max_smem_optin() {
  // dynamic shared memory any kernel here may request: the opt-in maximum
  // less a margin that covers the largest static footprint of the
  // dynamic-smem pivoted-QR kernels (at most 1.5 KB: the FP64 slab kernel's
  // per-CTA records of a 16-CTA cluster)
  int dev = 0, mx = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return mx - 2048;
}

template <typename T>
cudaError_t launch_copy(const CopyDesc<T>* d, const int* chunk_start, int count, int total_chunks, cudaStream_t st) {
  if (count <= 0 || total_chunks <= 0) return cudaSuccess;
  copy_kernel<T><<<(unsigned)total_chunks, kThreads, 0, st>>>(d, chunk_start, count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_identity(const CopyDesc<T>* d, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  identity_kernel<T><<<(unsigned)count, kThreads, 0, st>>>(d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_front_qr_smem(const FrontDesc<T>* d, int count, int smem_bytes, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  static std::once_flag init;  // attributes set once, whichever host thread launches first
  std::call_once(init, [] {
    allow_smem(front_qr_smem_kernel<T>);
  });
  front_qr_smem_kernel<T><<<(unsigned)count, kThreads, (size_t)smem_bytes, st>>>(d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_front_qr_warp(const FrontDesc<T>* d, int count, int per_warp_elems, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  static std::once_flag init;  // attributes set once, whichever host thread launches first
  std::call_once(init, [] {
    allow_smem(front_qr_warp_kernel<T>);
  });
  const size_t smem = (size_t)per_warp_elems * sizeof(T) * kWarps;
  front_qr_warp_kernel<T><<<(unsigned)((count + kWarps - 1) / kWarps), kThreads, smem, st>>>(d, count, per_warp_elems);
  return cudaGetLastError();
}

// rows_max = the largest m - j0 of the batch: panels that fit the shared memory
// of at most 16 CTAs take the cluster kernel, others the one-CTA kernel.
template <typename T>
cudaError_t launch_front_panel(const FrontDesc<T>* d, int count, int j0, int nb, T* Tbuf, cudaStream_t st,
                               int rows_max) {
  if (count <= 0) return cudaSuccess;
  const int lim = max_smem_optin() - 12 * 1024;  // room for the kernel's static shared memory
  const int per_cap = lim / (nb * (int)sizeof(T)) - 1;
  int cs = 1;
  while (cs < 16 && (rows_max + cs - 1) / cs > per_cap) cs *= 2;
  // a few fronts: spread their rows over larger clusters (the per-column loops
  // shorten with the rows per CTA; the two cluster barriers per column do not
  // grow), while the batch stays within one wave of clusters (about 128 SMs)
  // and every CTA keeps at least 64 rows
  while (cs < 16 && (int64_t)count * cs * 2 <= 128 && rows_max / (cs * 2) >= 64) cs *= 2;
  const int per_max = (rows_max + cs - 1) / cs;
  if (rows_max <= 0 || per_max > per_cap) {
    front_panel_kernel<T><<<(unsigned)count, kThreads, 0, st>>>(d, j0, nb, Tbuf);
    return cudaGetLastError();
  }
  static std::once_flag init;  // attributes set once, whichever host thread launches first
  std::call_once(init, [] {
    allow_smem(front_panel_cluster_kernel<T>);
    cudaFuncSetAttribute(front_panel_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  });
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(count * cs));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = (size_t)(per_max | 1) * nb * sizeof(T);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, front_panel_cluster_kernel<T>, d, j0, nb, Tbuf, per_max);
}

template <typename T>
cudaError_t launch_front_trailing(const FrontDesc<T>* d, int count, int j0, int nb, const T* Tbuf, int max_tiles,
                                  cudaStream_t st) {
  if (count <= 0 || max_tiles <= 0) return cudaSuccess;
  front_trailing_kernel<T><<<dim3((unsigned)max_tiles, (unsigned)count), kThreads, 0, st>>>(d, j0, nb, Tbuf);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_front_finish(const FrontDesc<T>* d, int count, int max_c, int max_n, unsigned* masks,
                                cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int words = (max_c + 31) / 32;
  front_signs_kernel<T><<<(unsigned)count, kThreads, 0, st>>>(d, masks, words);
  front_finish_kernel<T><<<dim3((unsigned)count, (unsigned)((max_n + 31) / 32)), kThreads, 0, st>>>(d, masks, words);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_cluster(void (*kernel)(const QrcpDesc<T>*, double, int, int), std::once_flag& init, unsigned grid,
                                  int cs, int smem, cudaStream_t st, const QrcpDesc<T>* d, double eps, int nl_max,
                                  int m_max, int threads = kThreads) {
  std::call_once(init, [kernel] {
    allow_smem(kernel);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  });
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, d, eps, nl_max, m_max);
}

template <typename T>
cudaError_t launch_qrcp(const QrcpDesc<T>* d, int count, double eps, int cs, int nl_max, int m_max, bool smem_slab,
                        cudaStream_t st, int nb) {
  if (count <= 0) return cudaSuccess;
  if (cs == 0) {  // one warp per matrix; nl_max = per-warp bytes
    static std::once_flag init;  // attributes set once, whichever host thread launches first
    std::call_once(init, [] {
      allow_smem(qrcp_warp_kernel<T>);
    });
    qrcp_warp_kernel<T><<<(unsigned)((count + kWarps - 1) / kWarps), kThreads, (size_t)nl_max * kWarps, st>>>(
        d, count, eps, nl_max);
    return cudaGetLastError();
  }
  const int smem = qrcp_smem_bytes(m_max, nl_max, (int)sizeof(T), smem_slab, nb);
  const unsigned grid = (unsigned)(count * cs);
  if (smem_slab) {
    static std::once_flag init_s;
    return launch_cluster(qrcp_slab_kernel<T, 8, kThreads>, init_s, grid, cs, smem, st, d, eps, nl_max, m_max, kThreads);
  }
  switch (nb) {
    case 16: {
      static std::once_flag i16;
      return launch_cluster(qrcp_delayed_kernel<T, 16>, i16, grid, cs, smem, st, d, eps, nl_max, m_max);
    }
    case 8: {
      static std::once_flag i8;
      return launch_cluster(qrcp_delayed_kernel<T, 8>, i8, grid, cs, smem, st, d, eps, nl_max, m_max);
    }
    case 4: {
      static std::once_flag i4;
      return launch_cluster(qrcp_delayed_kernel<T, 4>, i4, grid, cs, smem, st, d, eps, nl_max, m_max);
    }
    case 2: {
      static std::once_flag i2;
      return launch_cluster(qrcp_delayed_kernel<T, 2>, i2, grid, cs, smem, st, d, eps, nl_max, m_max);
    }
    default: {
      static std::once_flag i1;
      return launch_cluster(qrcp_delayed_kernel<T, 1>, i1, grid, cs, smem, st, d, eps, nl_max, m_max);
    }
  }
}

int qrcp_grid_capacity(int smem_bytes, int elem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (elem == 4) {
    allow_smem(qrcp_grid_kernel<float, 8, true>);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, qrcp_grid_kernel<float, 8, true>, kThreads, smem_bytes);
  } else {
    allow_smem(qrcp_grid_kernel<double, 8, true>);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, qrcp_grid_kernel<double, 8, true>, kThreads, smem_bytes);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    per = 0;
  }
  return std::min(sms * per, kThreads);  // the winner search takes one thread per CTA of a matrix
}

// Wait limit and missing arrivals of the CTA-group exchange (failure-path tests
// lower the limit and ask for an arrival that never comes).
std::atomic<long long> g_grid_wait_cycles{kQrcpGridWaitCyclesDefault};
std::atomic<int> g_grid_missing{0};

void qrcp_grid_set_wait(long long cycles, int missing) {
  g_grid_wait_cycles.store(cycles > 0 ? cycles : kQrcpGridWaitCyclesDefault);
  g_grid_missing.store(missing > 0 ? missing : 0);
}

template <typename T>
cudaError_t launch_qrcp_grid(const QrcpDesc<T>* d, const QrcpGridDesc* gd, int count, int total_ctas, double eps,
                             int nl_max, int m_max, bool smem_slab, cudaStream_t st) {
  if (count <= 0 || total_ctas <= 0) return cudaSuccess;
  const int smem = qrcp_grid_smem_bytes(m_max, nl_max, (int)sizeof(T), smem_slab);
  static std::once_flag init_s, init_g;
  auto kernel = smem_slab ? qrcp_grid_kernel<T, 8, true> : qrcp_grid_kernel<T, 8, false>;
  std::call_once(smem_slab ? init_s : init_g, [kernel] { allow_smem(kernel); });
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)total_ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const long long wait = g_grid_wait_cycles.load();
  const int missing = g_grid_missing.load();
  return cudaLaunchKernelEx(&cfg, kernel, d, gd, count, eps, nl_max, m_max, wait, missing);
}

template <typename T>
cudaError_t launch_refl(const ReflDesc<T>* d, const int2* items, int nitems, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  refl_kernel<T><<<(unsigned)nitems, kThreads, 0, st>>>(d, items);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_trsm(const TrsmDesc<T>* d, const int2* items, int nitems, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  trsm_kernel<T><<<(unsigned)nitems, kThreads, 0, st>>>(d, items);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_argmax(const ArgmaxDesc<T>* d, const int2* items, int nitems, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  argmax_kernel<T><<<(unsigned)nitems, kThreads, 0, st>>>(d, items);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_values(T* base, const int64_t* dest, const T* vals, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  scatter_values_kernel<T><<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(base, dest, vals, n);
  return cudaGetLastError();
}

// The tensor-core panel steps of one blocked group: for every panel j0 the
// fronts still active, with P / Wp carved from the scratch after the
// descriptors (the same P / Wp region serves every panel: the panels run in
// stream order).  Returns the descriptors [panel][front] and per-panel offsets.
template <typename T>
static size_t tc_group_layout(const std::vector<FrontDesc<T>>& fronts, const T* Tbuf, unsigned char* base,
                              std::vector<TcPanel>& all, std::vector<size_t>& first, int* flag = nullptr) {
  constexpr int nb = 32;
  int steps_max = 0;
  for (auto& f : fronts) steps_max = std::max(steps_max, std::min(f.c, f.m));
  const int npan = (steps_max + nb - 1) / nb;
  all.clear();
  first.assign((size_t)npan + 1, 0);
  size_t work_max = 0;
  for (int p = 0; p < npan; ++p) {
    const int j0 = p * nb;
    first[(size_t)p] = all.size();
    size_t off = 0;
    for (size_t fi = 0; fi < fronts.size(); ++fi) {
      const auto& f = fronts[fi];
      const int steps = std::min(f.c, f.m);
      if (j0 >= steps) continue;
      TcPanel t{};
      t.b = std::min(nb, steps - j0);
      t.ncols = f.n - j0 - t.b;
      t.mr = f.m - j0;
      if (t.ncols <= 0 || t.mr <= 0) continue;
      t.X = reinterpret_cast<float*>(f.ptr);
      t.Tm = reinterpret_cast<const float*>(Tbuf) + fi * nb * nb;
      t.ld = f.ld;
      t.j0 = j0;
      t.flag = flag;
      tc_plan_panel(t);
      t.P = reinterpret_cast<float*>(base) + off;  // offsets relative to the work region, fixed below
      off += tc_panel_scratch(t);
      t.Wp = t.P + (size_t)t.nsl * t.ncols * 32;
      all.push_back(t);
    }
    work_max = std::max(work_max, off);
  }
  first[(size_t)npan] = all.size();
  return work_max;
}

template <typename T>
size_t front_groups_tc_bytes(const std::vector<FrontGroup>& groups, const std::vector<std::vector<FrontDesc<T>>>& host) {
  if (sizeof(T) != sizeof(float)) return 0;
  size_t need = 0;
  for (size_t g = 0; g < groups.size(); ++g) {
    if (groups[g].kind != 2) continue;
    std::vector<TcPanel> all;
    std::vector<size_t> first;
    const size_t work = tc_group_layout<T>(host[g], nullptr, nullptr, all, first);
    const size_t desc = (all.size() * sizeof(TcPanel) + 255) / 256 * 256;
    need = std::max(need, desc + work * sizeof(float));
  }
  return need;
}

template <typename T>
cudaError_t launch_front_groups(const std::vector<FrontGroup>& groups, const std::vector<const FrontDesc<T>*>& d,
                                const std::vector<std::vector<FrontDesc<T>>>& host, T* Tbuf, cudaStream_t st,
                                int64_t* launches, void* tc_scratch, int* tc_flag) {
  cudaError_t e = cudaSuccess;
  for (size_t g = 0; g < groups.size() && e == cudaSuccess; ++g) {
    const FrontGroup& G = groups[g];
    const int cnt = (int)G.idx.size();
    if (G.kind == 0) {
      e = launch_front_qr_warp<T>(d[g], cnt, G.param, st);
      ++*launches;
    } else if (G.kind == 1) {
      e = launch_front_qr_smem<T>(const_cast<FrontDesc<T>*>(d[g]), cnt, G.param, st);
      ++*launches;
    } else {
      const int nb = 32;
      const bool tc = sizeof(T) == sizeof(float) && tc_scratch != nullptr;
      std::vector<TcPanel> all;
      std::vector<size_t> first;
      TcPanel* d_all = nullptr;
      if (tc) {
        // descriptors first, then the P / Wp work region
        std::vector<TcPanel> probe;
        std::vector<size_t> pf;
        tc_group_layout<T>(host[g], Tbuf, nullptr, probe, pf);
        const size_t dbytes = (probe.size() * sizeof(TcPanel) + 255) / 256 * 256;
        unsigned char* work = static_cast<unsigned char*>(tc_scratch) + dbytes;
        tc_group_layout<T>(host[g], Tbuf, work, all, first, tc_flag);
        d_all = static_cast<TcPanel*>(tc_scratch);
        if (!all.empty()) e = cudaMemcpyAsync(d_all, all.data(), all.size() * sizeof(TcPanel), cudaMemcpyHostToDevice, st);
      }
      int p = 0;
      for (int j0 = 0; j0 < G.param && e == cudaSuccess; j0 += nb, ++p) {
        int rows_max = 0;
        for (auto& f : host[g])
          if (j0 < std::min(f.c, f.m)) rows_max = std::max(rows_max, f.m - j0);
        e = launch_front_panel<T>(d[g], cnt, j0, nb, Tbuf, st, rows_max);
        ++*launches;
        if (e != cudaSuccess) break;
        if (tc) {
          const size_t a = first[(size_t)p], b = first[(size_t)p + 1];
          if (b > a) {
            std::vector<TcPanel> cur(all.begin() + (long)a, all.begin() + (long)b);
            e = launch_tc_panels(d_all + a, cur, st);
            *launches += 3;
          }
        } else {
          int maxtiles = 0;
          for (auto& f : host[g]) {
            const int steps = f.c < f.m ? f.c : f.m;
            if (j0 >= steps) continue;
            const int b = steps - j0 < nb ? steps - j0 : nb;
            const int tiles = (f.n - (j0 + b) + 31) / 32;
            maxtiles = tiles > maxtiles ? tiles : maxtiles;
          }
          e = launch_front_trailing<T>(d[g], cnt, j0, nb, Tbuf, maxtiles, st);
          ++*launches;
        }
      }
      // the sign masks go where the panels' T factors were (no longer needed):
      // count x 32 x 32 elements hold ceil(max c / 32) words per front
      int max_n = 0;
      for (auto& f : host[g]) max_n = std::max(max_n, f.n);
      if (e == cudaSuccess)
        e = launch_front_finish<T>(d[g], cnt, G.param, max_n, reinterpret_cast<unsigned*>(Tbuf), st);
      *launches += 2;
    }
  }
  return e;
}

#define SPAQR_INST(T)                                                                                     \
  template cudaError_t launch_front_groups<T>(const std::vector<FrontGroup>&, const std::vector<const FrontDesc<T>*>&, \
                                              const std::vector<std::vector<FrontDesc<T>>>&, T*, cudaStream_t,       \
                                              int64_t*, void*, int*);                                                \
  template size_t front_groups_tc_bytes<T>(const std::vector<FrontGroup>&,                                          \
                                           const std::vector<std::vector<FrontDesc<T>>>&);                         \
  template cudaError_t launch_scatter_values<T>(T*, const int64_t*, const T*, int64_t, cudaStream_t);    \
  template cudaError_t launch_copy<T>(const CopyDesc<T>*, const int*, int, int, cudaStream_t);           \
  template cudaError_t launch_identity<T>(const CopyDesc<T>*, int, cudaStream_t);                        \
  template cudaError_t launch_front_qr_smem<T>(const FrontDesc<T>*, int, int, cudaStream_t);             \
  template cudaError_t launch_front_qr_warp<T>(const FrontDesc<T>*, int, int, cudaStream_t);             \
  template cudaError_t launch_front_panel<T>(const FrontDesc<T>*, int, int, int, T*, cudaStream_t, int); \
  template cudaError_t launch_front_trailing<T>(const FrontDesc<T>*, int, int, int, const T*, int,       \
                                                cudaStream_t);                                           \
  template cudaError_t launch_front_finish<T>(const FrontDesc<T>*, int, int, int, unsigned*, cudaStream_t);                   \
  template cudaError_t launch_qrcp<T>(const QrcpDesc<T>*, int, double, int, int, int, bool, cudaStream_t, int); \
  template cudaError_t launch_qrcp_grid<T>(const QrcpDesc<T>*, const QrcpGridDesc*, int, int, double, int, int,    \
                                           bool, cudaStream_t);                                                   \
  template cudaError_t launch_refl<T>(const ReflDesc<T>*, const int2*, int, cudaStream_t);               \
  template cudaError_t launch_trsm<T>(const TrsmDesc<T>*, const int2*, int, cudaStream_t);               \
  template cudaError_t launch_argmax<T>(const ArgmaxDesc<T>*, const int2*, int, cudaStream_t);

SPAQR_INST(double)
SPAQR_INST(float)

}  // namespace spaqr
