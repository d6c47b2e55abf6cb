// Launchers for the device kernels of the factorization and the solve.
// All matrices are column-major.  Every launcher enqueues on `st` and returns
// the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace spaqr {

// One 2D block copy dst[r + c*dld] = src[row(r) + c*sld], row(r) = r or
// rowidx[r]; src == nullptr writes zeros.  Optionally transposed:
// dst[c + r*dld] = src[row(r) + c*sld].
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
// the reflectors go to V (m x k, ld m, unit diagonal) and tau.
template <typename T>
struct QrcpDesc {
  const T* src;
  T* work;
  T* out;
  T* V;
  T* tau;
  int* rank;
  int m, n, ld, ldo;
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
// out[r - r0].
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
// Small fronts: whole front in shared memory (smem_bytes >= m*n*sizeof(T) for every front).
template <typename T> cudaError_t launch_front_qr_smem(const FrontDesc<T>* d, int count, int smem_bytes, cudaStream_t st);
// Large fronts, blocked: panel j0..j0+nb of each front then the trailing update.
template <typename T>
cudaError_t launch_front_panel(const FrontDesc<T>* d, int count, int j0, int nb, T* Tbuf, cudaStream_t st);
template <typename T>
cudaError_t launch_front_trailing(const FrontDesc<T>* d, int count, int j0, int nb, const T* Tbuf, int max_tiles,
                                  cudaStream_t st);
template <typename T>
cudaError_t launch_front_finish(const FrontDesc<T>* d, int count, int max_c, cudaStream_t st);
// smem_bytes > 0: whole matrices in shared memory (qrcp_smem_bytes(m, n, sizeof(T), true));
// smem_bytes < 0: matrices in `work` with -smem_bytes of shared scratch.
template <typename T>
cudaError_t launch_qrcp(const QrcpDesc<T>* d, int count, double eps, int smem_bytes, cudaStream_t st);
inline int qrcp_smem_bytes(int m, int n, int elem, bool whole) {
  const int kmax = m < n ? m : n;
  long long b = ((long long)n * 20 + 15) / 16 * 16 + (long long)(((kmax + 1) & ~1) + 2) * elem;
  if (whole) b += (long long)m * n * elem;
  return (int)(b + 16);
}
inline int front_smem_bytes(int m, int n, int c, int elem) {
  return (int)((long long)m * n * elem + ((c + 31) / 32) * 4 + 16);
}
template <typename T> cudaError_t launch_refl(const ReflDesc<T>* d, int count, int max_vec, cudaStream_t st);
template <typename T> cudaError_t launch_trsm(const TrsmDesc<T>* d, int count, int max_rows, cudaStream_t st);
template <typename T> cudaError_t launch_argmax(const ArgmaxDesc<T>* d, int count, int max_rows, cudaStream_t st);
// Write an identity c x c block at ptr (ld) for each desc (src/transposed unused).
template <typename T> cudaError_t launch_identity(const CopyDesc<T>* d, int count, cudaStream_t st);

// base[dest[e]] = vals[e] for e < n (initial matrix into the group blocks)
template <typename T> cudaError_t launch_scatter_values(T* base, const int64_t* dest, const T* vals, int64_t n, cudaStream_t st);

int max_smem_optin();

}  // namespace spaqr
