// Dense device kernels of the spaQR factorization (sm_103a).
//
//  * front QR (Section 2.3, 2.4): Householder QR of the eliminated columns of
//    a batch of uneven fronts.  Fronts that fit run entirely in shared memory,
//    one CTA each, with warp-shuffle reductions; larger fronts run blocked:
//    a panel kernel (reflectors + the compact-WY factor T) and a multi-CTA
//    trailing update C <- C - V (T^T (V^T C)).
//  * column-pivoted QR (Section 2.5, the rank-revealing QR of Section 4):
//    one CTA per matrix, pivot by the largest remaining column norm (norms
//    kept in FP64), stop at |R_ii| < eps |R_11|.
//  * reflector application, triangular solve X R^{-1}, batched block copies
//    and the max-norm row assignment (Section 2.2).
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

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
  const int64_t total = (int64_t)d.rows * d.cols;
  const int64_t beg = (int64_t)(b - chunk_start[lo]) * kCopyChunk;
  if (beg >= total) return;
  const int64_t end = beg + kCopyChunk < total ? beg + kCopyChunk : total;
  for (int64_t e = beg + threadIdx.x; e < end; e += kThreads) {
    const int r = (int)(e % d.rows);
    const int c = (int)(e / d.rows);
    T v = T(0);
    if (d.src) {
      const int sr = d.rowidx ? d.rowidx[r] : r;
      v = d.src[sr + (int64_t)c * d.sld];
    }
    if (d.transpose)
      d.dst[c + (int64_t)r * d.dld] = v;
    else
      d.dst[r + (int64_t)c * d.dld] = v;
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

// --------------------------------------------------------- reflector maths
// Computes the Householder reflector of x = X[j:m, j] (column j of X with
// leading dimension ld) by warp 0: beta = -sign(alpha) ||x|| (sign(0) = +1),
// v = x / (alpha - beta) below the diagonal, tau = (beta - alpha) / beta;
// tau = 0 (H = I) when x[1:] = 0.  Writes v in place and beta at X[j, j].
// Returns (through shared memory) tau and beta.
template <typename T>
__device__ void make_reflector_warp0(T* X, int ld, int m, int j, T* s_tau, double* s_beta) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  T* col = X + (int64_t)j * ld;
  double sig = 0.0;
  for (int i = j + 1 + lane; i < m; i += 32) {
    const double v = (double)col[i];
    sig += v * v;
  }
  sig = warp_sum(sig);
  const double alpha = (double)col[j];
  double beta, tau;
  if (sig == 0.0) {
    beta = alpha;
    tau = 0.0;
  } else {
    const double nrm = sqrt(alpha * alpha + sig);
    beta = alpha >= 0.0 ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    const T den = (T)(alpha - beta);
    for (int i = j + 1 + lane; i < m; i += 32) col[i] = col[i] / den;
  }
  __syncwarp();
  if (lane == 0) {
    col[j] = (T)beta;
    *s_tau = (T)tau;
    *s_beta = beta;
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

// ------------------------------------------------- front QR, shared memory
template <typename T>
__global__ void __launch_bounds__(kThreads) front_qr_smem_kernel(const FrontDesc<T>* descs) {
  const FrontDesc<T> d = descs[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smraw[];
  T* S = reinterpret_cast<T*>(smraw);
  __shared__ T s_tau;
  __shared__ double s_beta;
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
  for (int j = 0; j < steps; ++j) {
    make_reflector_warp0(S, m, m, j, &s_tau, &s_beta);
    __syncthreads();
    const T tau = s_tau;
    if (threadIdx.x == 0 && s_beta < 0.0) negmask[j >> 5] |= 1u << (j & 31);
    if (tau != T(0)) apply_reflector_cols(S, m, m, j, tau, j + 1, n);
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
  __shared__ T s_tau;
  __shared__ double s_beta;
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
template <typename T>
__global__ void __launch_bounds__(kThreads) front_finish_kernel(const FrontDesc<T>* descs) {
  const FrontDesc<T> d = descs[blockIdx.x];
  const int steps = d.c < d.m ? d.c : d.m;
  T* X = d.ptr;
  extern __shared__ unsigned negmask[];  // ceil(steps / 32) words
  for (int t = threadIdx.x; t < (steps + 31) / 32; t += kThreads) negmask[t] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < steps; i += kThreads)
    if (X[i + (int64_t)i * d.ld] < T(0)) atomicOr(&negmask[i >> 5], 1u << (i & 31));
  __syncthreads();
  // rows r < steps, columns >= r: flip; columns < steps, rows > column: zero
  for (int64_t e = threadIdx.x; e < (int64_t)steps * d.n; e += kThreads) {
    const int r = (int)(e % steps), cc = (int)(e / steps);
    if (cc >= r && ((negmask[r >> 5] >> (r & 31)) & 1u)) X[r + (int64_t)cc * d.ld] = -X[r + (int64_t)cc * d.ld];
  }
  for (int64_t e = threadIdx.x; e < (int64_t)d.m * steps; e += kThreads) {
    const int r = (int)(e % d.m), cc = (int)(e / d.m);
    if (r > cc) X[r + (int64_t)cc * d.ld] = T(0);
  }
}

// ------------------------------------------------------------------- QRCP
template <typename T, bool SMEM>
__global__ void __launch_bounds__(kThreads) qrcp_kernel(const QrcpDesc<T>* descs, double eps) {
  const QrcpDesc<T> d = descs[blockIdx.x];
  const int m = d.m, n = d.n;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* nu = reinterpret_cast<double*>(smraw);
  double* nuref = nu + n;
  int* perm = reinterpret_cast<int*>(nuref + n);
  T* taus = reinterpret_cast<T*>(smraw + (((size_t)n * 20 + 15) / 16) * 16);
  const int kmax = m < n ? m : n;
  T* X;
  const int ld = m;
  if (SMEM) {
    X = taus + ((kmax + 1) & ~1) + 2;
  } else {
    X = d.work;  // m x n, ld m
  }
  for (int64_t e = threadIdx.x; e < (int64_t)m * n; e += kThreads) {
    const int r = (int)(e % m), cc = (int)(e / m);
    X[e] = d.src[r + (int64_t)cc * d.ld];
  }
  __shared__ T s_tau;
  __shared__ double s_beta;
  __shared__ double s_r11;
  __shared__ int s_piv;
  __shared__ int s_stop;
  __shared__ double red_v[kWarps];
  __shared__ int red_i[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  for (int j = warp; j < n; j += kWarps) {
    double s = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double v = (double)X[r + (int64_t)j * ld];
      s += v * v;
    }
    s = warp_sum(s);
    if (lane == 0) {
      nu[j] = s;
      nuref[j] = s;
      perm[j] = j;
    }
  }
  __syncthreads();
  int k = 0;
  for (int i = 0; i < kmax; ++i) {
    // pivot: largest nu[j], j >= i, ties to the lowest index
    double bv = -1.0;
    int bi = n;
    for (int j = i + threadIdx.x; j < n; j += kThreads) {
      const double v = nu[j];
      if (v > bv || (v == bv && j < bi)) {
        bv = v;
        bi = j;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = red_v[0];
      int p = red_i[0];
      for (int w = 1; w < kWarps; ++w)
        if (red_v[w] > v || (red_v[w] == v && red_i[w] < p)) {
          v = red_v[w];
          p = red_i[w];
        }
      s_piv = p;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != i) {
      for (int r = threadIdx.x; r < m; r += kThreads) {
        const T a = X[r + (int64_t)i * ld];
        X[r + (int64_t)i * ld] = X[r + (int64_t)p * ld];
        X[r + (int64_t)p * ld] = a;
      }
      if (threadIdx.x == 0) {
        double t = nu[i];
        nu[i] = nu[p];
        nu[p] = t;
        t = nuref[i];
        nuref[i] = nuref[p];
        nuref[p] = t;
        const int q = perm[i];
        perm[i] = perm[p];
        perm[p] = q;
      }
      __syncthreads();
    }
    make_reflector_warp0(X, ld, m, i, &s_tau, &s_beta);
    __syncthreads();
    if (threadIdx.x == 0) {
      const double ab = fabs(s_beta);
      if (i == 0) s_r11 = ab;
      s_stop = (s_beta == 0.0 || ab < eps * s_r11) ? 1 : 0;
    }
    __syncthreads();
    if (s_stop) break;  // column i keeps a spent reflector; only rows < k are ever read
    const T tau = s_tau;
    if (threadIdx.x == 0) taus[i] = tau;
    if (tau != T(0)) apply_reflector_cols(X, ld, m, i, tau, i + 1, n);
    __syncthreads();
    for (int j = i + 1 + threadIdx.x; j < n; j += kThreads) {
      const double x = (double)X[i + (int64_t)j * ld];
      double v = nu[j] - x * x;
      if (v < kRecompute * nuref[j]) {
        v = 0.0;
        for (int r = i + 1; r < m; ++r) {
          const double y = (double)X[r + (int64_t)j * ld];
          v += y * y;
        }
        nuref[j] = v;
      }
      nu[j] = v;
    }
    k = i + 1;
    __syncthreads();
  }
  if (threadIdx.x == 0) d.rank[0] = k;
  if (d.V) {
    for (int64_t e = threadIdx.x; e < (int64_t)m * k; e += kThreads) {
      const int r = (int)(e % m), i = (int)(e / m);
      d.V[e] = r < i ? T(0) : (r == i ? T(1) : X[r + (int64_t)i * ld]);
    }
    for (int i = threadIdx.x; i < k; i += kThreads) d.tau[i] = taus[i];
  }
  // the first k rows of Q^T A in the original column order replace rows
  // 0..k-1 of out, and only when something is dropped (k < m)
  if (d.out && k < m) {
    for (int64_t e = threadIdx.x; e < (int64_t)k * n; e += kThreads) {
      const int i = (int)(e % k), j = (int)(e / k);
      d.out[i + (int64_t)perm[j] * d.ldo] = j < i ? T(0) : X[i + (int64_t)j * ld];
    }
  }
}

// ------------------------------------------------------ reflector applies
template <typename T>
__global__ void __launch_bounds__(kThreads) refl_kernel(const ReflDesc<T>* descs) {
  const ReflDesc<T> d = descs[blockIdx.y];
  const int k = *d.k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vec = blockIdx.x * kWarps + warp;
  if (vec >= d.nvec) return;
  const int len = d.len;
  if (d.mode == 0) {
    // row vector x (elements x[l] = ptr[vec + l*ld]) <- x^T H_1 ... H_k
    T* x = d.ptr + vec;
    if (k < len) {
      for (int i = 0; i < k; ++i) {
        const T* v = d.V + (int64_t)i * len;
        T s = T(0);
        for (int l = i + lane; l < len; l += 32) s += x[(int64_t)l * d.ld] * (l == i ? T(1) : v[l]);
        s = warp_sum(s) * d.tau[i];
        for (int l = i + lane; l < len; l += 32) x[(int64_t)l * d.ld] -= s * (l == i ? T(1) : v[l]);
      }
      for (int l = k + lane; l < len; l += 32) x[(int64_t)l * d.ld] = T(0);
    }
  } else {
    // column vector y (contiguous) <- H_k ... H_1 y
    T* y = d.ptr + (int64_t)vec * d.ld;
    if (k < len) {
      for (int i = 0; i < k; ++i) {
        const T* v = d.V + (int64_t)i * len;
        T s = T(0);
        for (int l = i + lane; l < len; l += 32) s += y[l] * (l == i ? T(1) : v[l]);
        s = warp_sum(s) * d.tau[i];
        for (int l = i + lane; l < len; l += 32) y[l] -= s * (l == i ? T(1) : v[l]);
      }
      for (int l = k + lane; l < len; l += 32) y[l] = T(0);
    }
  }
}

// ---------------------------------------------------------- X <- X R^{-1}
template <typename T>
__global__ void __launch_bounds__(kThreads) trsm_kernel(const TrsmDesc<T>* descs) {
  const TrsmDesc<T> d = descs[blockIdx.y];
  const int r = blockIdx.x * kThreads + threadIdx.x;
  if (r >= d.rows) return;
  T* x = d.ptr + r;
  for (int j = 0; j < d.c; ++j) {
    T s = x[(int64_t)j * d.ld];
    const T* Rj = d.R + (int64_t)j * d.rld;
    for (int i = 0; i < j; ++i) s -= x[(int64_t)i * d.ld] * Rj[i];
    x[(int64_t)j * d.ld] = s / Rj[j];
  }
}

// ----------------------------------------------------- max-norm row rule
template <typename T>
__global__ void __launch_bounds__(kThreads) argmax_kernel(const ArgmaxDesc<T>* descs) {
  const ArgmaxDesc<T> d = descs[blockIdx.y];
  const int r = d.r0 + blockIdx.x * kThreads + threadIdx.x;
  if (r >= d.r1) return;
  double best = -1.0;
  int bl = -1, bid = 0x7fffffff, bt = -1;
  for (int t = 0; t < d.ncl; ++t) {
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
  // dynamic-smem kernels (a few hundred bytes)
  int dev = 0, mx = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return mx - 1024;
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
  static bool init = false;
  if (!init) {
    allow_smem(front_qr_smem_kernel<T>);
    init = true;
  }
  front_qr_smem_kernel<T><<<(unsigned)count, kThreads, (size_t)smem_bytes, st>>>(d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_front_panel(const FrontDesc<T>* d, int count, int j0, int nb, T* Tbuf, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  front_panel_kernel<T><<<(unsigned)count, kThreads, 0, st>>>(d, j0, nb, Tbuf);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_front_trailing(const FrontDesc<T>* d, int count, int j0, int nb, const T* Tbuf, int max_tiles,
                                  cudaStream_t st) {
  if (count <= 0 || max_tiles <= 0) return cudaSuccess;
  front_trailing_kernel<T><<<dim3((unsigned)max_tiles, (unsigned)count), kThreads, 0, st>>>(d, j0, nb, Tbuf);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_front_finish(const FrontDesc<T>* d, int count, int max_c, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  front_finish_kernel<T><<<(unsigned)count, kThreads, (size_t)(((max_c + 31) / 32) * 4 + 16), st>>>(d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_qrcp(const QrcpDesc<T>* d, int count, double eps, int smem_bytes, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  static bool init = false;
  if (!init) {
    allow_smem(qrcp_kernel<T, true>);
    allow_smem(qrcp_kernel<T, false>);
    init = true;
  }
  // smem_bytes > 0: matrices in shared memory; < 0: in the work buffers with |smem_bytes| of scratch.
  if (smem_bytes > 0)
    qrcp_kernel<T, true><<<(unsigned)count, kThreads, (size_t)smem_bytes, st>>>(d, eps);
  else
    qrcp_kernel<T, false><<<(unsigned)count, kThreads, (size_t)(-smem_bytes), st>>>(d, eps);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_refl(const ReflDesc<T>* d, int count, int max_vec, cudaStream_t st) {
  if (count <= 0 || max_vec <= 0) return cudaSuccess;
  refl_kernel<T><<<dim3((unsigned)((max_vec + kWarps - 1) / kWarps), (unsigned)count), kThreads, 0, st>>>(d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_trsm(const TrsmDesc<T>* d, int count, int max_rows, cudaStream_t st) {
  if (count <= 0 || max_rows <= 0) return cudaSuccess;
  trsm_kernel<T><<<dim3((unsigned)((max_rows + kThreads - 1) / kThreads), (unsigned)count), kThreads, 0, st>>>(d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_argmax(const ArgmaxDesc<T>* d, int count, int max_rows, cudaStream_t st) {
  if (count <= 0 || max_rows <= 0) return cudaSuccess;
  argmax_kernel<T><<<dim3((unsigned)((max_rows + kThreads - 1) / kThreads), (unsigned)count), kThreads, 0, st>>>(d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_values(T* base, const int64_t* dest, const T* vals, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  scatter_values_kernel<T><<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(base, dest, vals, n);
  return cudaGetLastError();
}

#define SPAQR_INST(T)                                                                                     \
  template cudaError_t launch_scatter_values<T>(T*, const int64_t*, const T*, int64_t, cudaStream_t);    \
  template cudaError_t launch_copy<T>(const CopyDesc<T>*, const int*, int, int, cudaStream_t);           \
  template cudaError_t launch_identity<T>(const CopyDesc<T>*, int, cudaStream_t);                        \
  template cudaError_t launch_front_qr_smem<T>(const FrontDesc<T>*, int, int, cudaStream_t);             \
  template cudaError_t launch_front_panel<T>(const FrontDesc<T>*, int, int, int, T*, cudaStream_t);      \
  template cudaError_t launch_front_trailing<T>(const FrontDesc<T>*, int, int, int, const T*, int,       \
                                                cudaStream_t);                                           \
  template cudaError_t launch_front_finish<T>(const FrontDesc<T>*, int, int, cudaStream_t);                   \
  template cudaError_t launch_qrcp<T>(const QrcpDesc<T>*, int, double, int, cudaStream_t);               \
  template cudaError_t launch_refl<T>(const ReflDesc<T>*, int, int, cudaStream_t);                       \
  template cudaError_t launch_trsm<T>(const TrsmDesc<T>*, int, int, cudaStream_t);                       \
  template cudaError_t launch_argmax<T>(const ArgmaxDesc<T>*, int, int, cudaStream_t);

SPAQR_INST(double)
SPAQR_INST(float)

}  // namespace spaqr
