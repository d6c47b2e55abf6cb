/*
 * spaqr.h -- C ABI of the GB300 spaQR library: a hierarchical sparse QR
 * preconditioner for sparse least squares  min ||A x - b||_2,  A in R^{M x N},
 * M >= N, rank(A) = N  (problem statement, Section 1 of Gnanasekaran & Darve,
 * "Hierarchical Orthogonal Factorization: Sparse Least Squares problems").
 *
 * The factorization (Algorithm 1, Section 2.7) produces Q^T A W^{-1} ~= I with
 * W a product of sparse upper-triangular and orthogonal factors; the solve is
 * CGLS preconditioned on the right by W (Section 4).
 *
 * Conventions for every entry point:
 *  - Return value: SPAQR_OK (0) or one of the SPAQR_ERR_* codes below; the
 *    message of the last failure on the calling thread is spaqr_last_error().
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the current device.  The library never takes ownership
 *    of caller memory; it copies what it keeps.
 *  - All device work is issued on the stream given in the options (NULL =
 *    legacy default stream) and every entry point returns with that stream
 *    synchronised unless stated otherwise.
 *  - Matrices are column-major; "ld" is the leading dimension in elements.
 *  - There is no CPU fallback: without a CUDA device the compute entry points
 *    fail with SPAQR_ERR_NO_DEVICE.  spaqr_analyze and the analysis queries
 *    are host-only.
 */
#ifndef SPAQR_H
#define SPAQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPAQR_OK 0
#define SPAQR_ERR_INVALID_ARG 1
#define SPAQR_ERR_RANK_DEFICIENT 2 /* a diagonal block lost full column rank (Section 1: rank(A) = N) */
#define SPAQR_ERR_CAPACITY 3       /* a planned size bound was exceeded */
#define SPAQR_ERR_NOT_CONVERGED 4  /* CGLS hit maxit; x and info are still written */
#define SPAQR_ERR_TIMEOUT 5        /* a bounded device wait gave up */
#define SPAQR_ERR_CUDA 6
#define SPAQR_ERR_OOM 7
#define SPAQR_ERR_NO_DEVICE 8

#define SPAQR_PREC_FP64 0  /* every step in FP64 */
#define SPAQR_PREC_MIXED 1 /* factor in FP32, CGLS in FP64 */

#define SPAQR_MODE_SPAQR 0  /* scaling + two-step sparsification (Algorithm 1) */
#define SPAQR_MODE_DIRECT 1 /* no compression: multifrontal QR ("Direct", Section 4) */
#define SPAQR_MODE_DIAG 2   /* no factorization, W = I: the solve is CGLS preconditioned by the column
                               scaling D alone (the "Diag." comparator of Section 4); the analysis is
                               still required and only its n is used */

/* Sparse A in CSR form (host pointers).  Column indices in [0, n) and
 * ascending within a row; no explicit zeros are required to be absent. */
typedef struct {
  int64_t m, n, nnz;
  const int64_t* rowptr; /* m + 1 entries */
  const int32_t* colidx; /* nnz entries */
  const double* vals;    /* nnz entries */
  const int32_t* match;  /* optional (NULL = none), n entries: match[j] = the row matched to column j
                            (Section 2.2's matching step; distinct rows, each with an entry in its
                            column); a matched row belongs to its column's cluster, every other row
                            follows the max-norm rule.  Without it a row with a single entry is
                            matched by that rule anyway.  Invalid matchings fail with INVALID_ARG. */
} spaqr_csr;

/* Geometric ordering of a structured grid (Section 4.1, "regular geometric
 * partitioning"): column j is the vertex (i, j', k) with j = i + nx*(j' + ny*k).
 * depth = number of levels L of the nested-dissection tree (leaves at level L). */
typedef struct {
  int nx, ny, nz;
  int depth;
} spaqr_grid_ordering;

typedef struct {
  double eps;      /* rank tolerance of the sparsification RRQRs (Section 4: |R_ii| >= eps |R_11|) */
  int skip;        /* scaling/sparsification start at stage L - skip (default 2, Section 4.2) */
  int precision;   /* SPAQR_PREC_FP64 or SPAQR_PREC_MIXED */
  int mode;        /* SPAQR_MODE_SPAQR or SPAQR_MODE_DIRECT */
  double tol;      /* CGLS stop: ||A^T (A x - b)|| / ||A^T b|| < tol (default 1e-10) */
  int maxit;       /* CGLS iteration cap (default 500) */
  int use_graphs;  /* capture the per-iteration apply + SpMV sequence in a CUDA graph */
  int verbose;     /* print per-stage statistics to stderr */
  void* stream;    /* cudaStream_t for all device work (NULL = default stream) */
  int row_rule;    /* candidates of the max-norm row rule (Section 2.2): SPAQR_ROWS_TREE (default) =
                      the touched clusters of the deepest nested-dissection node, which keeps every
                      row on one root-to-leaf chain (disjoint subtrees stay disjoint, Section 2.5.2);
                      SPAQR_ROWS_ANY = every touched cluster */
  int apply_persistent; /* 1: each W^{-1} / W^{-T} apply is one cooperative persistent launch over all
                           stored operations (bounded grid barriers between dependent segments);
                           0 (default): one launch per segment and operation form, graph-captured */
  int step1_qr_width; /* a step-1 block (Section 2.5.1) at least this wide and at least 1.1 times taller
                         than wide is first reduced by a Householder QR to its square triangle, whose
                         column-pivoted QR has the same pivots, rank and rows; 0 = never (default 1280) */
} spaqr_options;

#define SPAQR_ROWS_TREE 0
#define SPAQR_ROWS_ANY 1

/* Fill *opt with the defaults: eps 1e-4, skip 2, FP64, spaqr mode, tol 1e-10,
 * maxit 500, graphs on, quiet, default stream, tree row rule, per-segment apply,
 * step-1 QR from width 1280. */
void spaqr_default_options(spaqr_options* opt);

/* ---------------------------------------------------------------- analysis
 * Symbolic phase (host only): geometric nested dissection of the grid, the
 * interfaces of every separator at every stage (modified nested dissection,
 * Section 2.2, Fig. 2-3) and the clustering hierarchy used by the merges
 * (Section 2.6).  Depends only on the grid and the depth, never on values. */
typedef struct spaqr_analysis spaqr_analysis;

/* Errors: INVALID_ARG for non-positive sizes or depth outside [1, 30]. */
int spaqr_analyze(const spaqr_grid_ordering* ord, spaqr_analysis** out);

/* spaqr_analyze_matrix: the same analysis for a matrix without a grid, from
 * the pattern of A alone (host only; values are not read): nested dissection
 * of graph(A^T A) (columns adjacent when a row holds both) to `depth` levels by
 * level structures of breadth-first searches, the interfaces of every
 * separator at every stage from the adjacency of its vertices to the
 * subdomains and interfaces below it, and the merge hierarchy (Section 2.2,
 * Fig. 2-3; Section 2.6).  On a grid with the geometric tree the interfaces
 * are those of spaqr_analyze.  The result is used with spaqr_factor like any
 * analysis (A's n must equal the analysed n).  A is caller-owned host CSR;
 * nothing is kept.  Errors: INVALID_ARG (bad CSR arrays, depth outside [1, 30]). */
int spaqr_analyze_matrix(const spaqr_csr* A, int depth, spaqr_analysis** out);

/* spaqr_match: the row-to-column matching of Section 2.2 for matrices without
 * a natural one: match[j] (n entries, caller-owned host memory) receives the
 * row matched to column j, distinct rows, each with a nonzero in its column,
 * chosen to maximise the sum of log|a_ij| over the matched entries (a
 * maximum-product matching; the paper uses a third-party routine for it).
 * Pass it to spaqr_factor in spaqr_csr.match.  Host only.  Errors: INVALID_ARG
 * (bad CSR arrays, m < n), RANK_DEFICIENT (no column-perfect matching exists:
 * A is structurally rank deficient). */
int spaqr_match(const spaqr_csr* A, int32_t* match);
void spaqr_analysis_destroy(spaqr_analysis* an);

/* Number of clusters alive at stage k (1 <= k <= depth) and the total number
 * of their vertices.  Host only. */
int spaqr_analysis_stage_size(const spaqr_analysis* an, int k, int64_t* nclusters, int64_t* nverts);

/* Copy the clusters of stage k in canonical order (node id, interface key):
 * node[c] = nested-dissection node (heap numbering, root 0), level[c] = its
 * level, vptr[c]..vptr[c+1] index verts[] = the cluster's vertex ids in
 * ascending order.  Arrays are caller-owned host memory sized by
 * spaqr_analysis_stage_size (vptr has nclusters + 1 entries). */
int spaqr_analysis_stage_clusters(const spaqr_analysis* an, int k, int32_t* node, int32_t* level,
                                  int64_t* vptr, int32_t* verts);

/* ---------------------------------------------------------------- factor
 * spaqr_factor: Algorithm 1 on A D (D = column scaling to unit 2-norms,
 * Section 2.7) with the given analysis.  Level by level, leaves to root:
 * block Householder QR of every separator front and reassignment of its extra
 * rows (Section 2.3), scaling of the remaining interfaces (2.4), sparsification
 * step 1 (2.5.1) and step 2 (2.5.2), merge (2.6).  A is read from host memory.
 * The handle owns every device allocation.  The analysis must outlive nothing:
 * the handle keeps what it needs.
 * Errors: INVALID_ARG (shape mismatch, n != grid size, m < n, a bad CSR pattern,
 * a match that is not a matching, unknown options; all checked on the host
 * before any device work), RANK_DEFICIENT, OOM, CUDA, NO_DEVICE, TIMEOUT. */
typedef struct spaqr_handle spaqr_handle;
int spaqr_factor(const spaqr_csr* A, const spaqr_analysis* an, const spaqr_options* opt, spaqr_handle** out);

/* spaqr_factor_batch: spaqr_factor of count matrices with one analysis (for
 * example many problems on one grid), run concurrently: every problem gets its
 * own handle and non-blocking stream, and the host planning of different
 * problems runs on different threads.  opt applies to all (its stream must be
 * NULL).  out[i] receives the handle of A[i]; on an error no handle is created
 * and the message names the problem.  Errors as spaqr_factor. */
int spaqr_factor_batch(int count, const spaqr_csr* const* A, const spaqr_analysis* an, const spaqr_options* opt,
                       spaqr_handle** out);

typedef struct {
  int iters;         /* CGLS iterations taken */
  double rel_resid;  /* final ||A^T (A x - b)|| / ||A^T b|| */
  int converged;     /* rel_resid < tol */
  double seconds;    /* wall time of the solve */
} spaqr_solve_info;

/* spaqr_solve: right-preconditioned CGLS (Section 4) on min ||A D W^{-1} y - b||,
 * x = D W^{-1} y.  b has m entries, x has n; both host pointers when
 * on_device == 0 (copied in / out inside the call) or device pointers when
 * on_device != 0.  Returns NOT_CONVERGED (x and info written) at maxit. */
int spaqr_solve(spaqr_handle* h, const double* b, double* x, int on_device, spaqr_solve_info* info);

/* spaqr_solve_csne: the corrected seminormal equations with iterative
 * refinement (Section 1, after Bjorck: R^T R x = A^T b solved with the factor,
 * then corrected with the residual).  With W^T W ~= (A D)^T (A D), each step is
 *     x~ <- x~ + W^{-1} W^{-T} (A D)^T (b - A D x~),     x = D x~,
 * from x~ = 0, until ||A^T (A x - b)|| / ||A^T b|| < tol (handle options) or
 * maxit steps.  At eps = 0 the first step is exact up to rounding; at eps > 0
 * it is a stationary iteration that converges when W is close enough to the
 * exact factor (no Krylov acceleration, unlike spaqr_solve).  Arguments,
 * return codes and info as spaqr_solve (NOT_CONVERGED with x and info written
 * at maxit; INVALID_ARG for a non-finite b). */
int spaqr_solve_csne(spaqr_handle* h, const double* b, double* x, int on_device, spaqr_solve_info* info);

/* z <- W^{-1} z (transpose = 0) or z <- W^{-T} z (transpose = 1) for a device
 * vector z of n entries in column (slot) order (Section 2.7: W is stored as a
 * sequence of sparse triangular and orthogonal factors). */
int spaqr_apply_Winv(spaqr_handle* h, double* z, int transpose);

/* y <- A D x (forward = 1, x: n, y: m) or y <- (A D)^T x (forward = 0, x: m,
 * y: n); device pointers.  The scaled operator the preconditioner is built for. */
int spaqr_apply_A(spaqr_handle* h, const double* x, double* y, int forward);

/* ------------------------------------------------------------------ adjoint
 * x(A, b) = argmin ||A x - b|| = (A^T A)^{-1} A^T b (Section 1).  For a loss L
 * with g = dL/dx, lambda = (A^T A)^{-1} g and r = b - A x give
 *     dL/db = A lambda,     dL/dA_ij = r_i lambda_j - (A lambda)_i x_j
 * on the nonzeros of A.  The factor is reused for lambda: A^T A =
 * D^{-1} (A D)^T (A D) D^{-1} and (A D)^T (A D) ~= W^T W (Section 2.7). */

/* spaqr_solve_normal: lambda = (A^T A)^{-1} g by conjugate gradients on
 * (A D)^T (A D) nu = D g, lambda = D nu, preconditioned by W^{-1} W^{-T}
 * (a triangular/orthogonal sweep with W^{-T}, then one with W^{-1}).  Stops
 * when ||g - A^T A lambda|| / ||g|| < tol or after the handle's maxit
 * iterations.  g and lambda have n entries; host pointers (on_device = 0,
 * copied inside the call) or device pointers.  Returns NOT_CONVERGED (lambda
 * and info written) at maxit; info may be NULL. */
int spaqr_solve_normal(spaqr_handle* h, const double* g, double* lambda, int on_device, double tol,
                       spaqr_solve_info* info);

/* spaqr_lstsq_grad: from b (m), x (n) and lambda (n), write dL/db (m entries)
 * and dL/dvals (nnz entries, in the CSR order of A) with one fused kernel (one
 * thread per row of A).  Either output may be NULL.  Host or device pointers
 * per on_device. */
int spaqr_lstsq_grad(spaqr_handle* h, const double* b, const double* x, const double* lambda, double* grad_b,
                     double* grad_vals, int on_device);

/* spaqr_update_values: A <- A' with the pattern unchanged; vals holds the nnz
 * values in the CSR order of A (host or device per on_device).
 * refactor = 0: the solves use A' and the factor built for A stays the
 *   preconditioner (the solves still converge to the solution for A': CGLS
 *   stops on the residual of A'); the column scaling D is kept.
 * refactor != 0: the factorization is redone for A' with the handle's
 *   options and the analysis an (required then; D is recomputed).
 * Errors: INVALID_ARG (null vals, or refactor without an analysis). */
int spaqr_update_values(spaqr_handle* h, const spaqr_analysis* an, const double* vals, int on_device,
                        int refactor);

/* Batched solves over `count` independent handles (for example many problems
 * with one pattern): hs[i] with b[i] -> x[i] (CGLS) or g[i] -> lambda[i]
 * (normal equations), each as in the single-problem call.  The iterations of
 * all handles advance side by side, each on its own handle's stream, with one
 * residual read per handle per iteration.  infos (count entries) may be NULL.
 * Returns the first error, else NOT_CONVERGED if some handle did not converge. */
int spaqr_solve_batch(int count, spaqr_handle* const* hs, const double* const* b, double* const* x, int on_device,
                      spaqr_solve_info* infos);
int spaqr_solve_normal_batch(int count, spaqr_handle* const* hs, const double* const* g, double* const* lambda,
                             int on_device, double tol, spaqr_solve_info* infos);

typedef struct {
  double t_analyze;  /* seconds in spaqr_analyze (copied from the analysis) */
  double t_factor;   /* seconds in spaqr_factor */
  double t_solve;    /* seconds in the last spaqr_solve */
  int iters;         /* iterations of the last solve */
  int64_t nnz_W;     /* stored entries of W (Section 3 memory measure) */
  int64_t n_ops;     /* number of stored W operations */
  int64_t n_fronts;  /* eliminated separator fronts */
  int64_t max_front_rows, max_front_cols;
  int64_t top_cols, top_rows; /* size of the root front (Section 4.3 top separator) */
  double flops_front;  /* algorithmic flops of the front QRs (Golub-Van Loan counts; includes the Householder
                          QR that precedes the step-1 pivoted QR of a tall block) */
  double flops_sparsify; /* step-1 and step-2 column-pivoted QRs plus the step-2 two-sided application */
  double t_phase[6];   /* wall seconds: eliminate (incl. row reassignment), prep (column scaling, row
                          owners, initial blocks), scale, step1, step2, merge */
  int64_t launches;    /* kernels launched by the factorization */
  int64_t syncs;       /* device-to-host waits during the factorization */
  /* device time (CUDA events on the library stream) summed per kernel family:
   * [0] block copies, [1] front QR (eliminate, scale, tall step-1 blocks), [2] column-pivoted QR,
   * [3] other factor kernels (argmax, trsm, reflector apply),
   * [4] W^{-1}/W^{-T} apply in the last solve, [5] SpMV + vector kernels in
   * the last solve.  Seconds. */
  double t_kernel[6];
  int64_t n_kernel[6]; /* launches counted in each family */
  double bytes_apply;  /* algorithmic bytes of one W^{-1} plus one W^{-T} apply */
  double flops_qrcp;   /* algorithmic flops of the column-pivoted QRs alone, 4mnk - 2k^2(m+n) + 4k^3/3 each */
  double bytes_qrcp;   /* algorithmic bytes of the same QRs: one read of the unpivoted trailing block per
                          pivot step, elem * (kmn - k^2(m+n)/2 + k^3/3), plus reading and writing m x n once */
} spaqr_stats;

int spaqr_get_stats(const spaqr_handle* h, spaqr_stats* st);

/* ------------------------------------------------------------ W inspection
 * The stored operations in factorization order (for tests and diagnostics).
 * kind: 0 = R_s (elimination, Section 2.3), 1 = R_p (scaling, 2.4),
 * 2 = Q_p (step-2 reflectors, 2.5.2).  For op i: stage, c (slots of s or p),
 * w (R_s: columns of R_sn; Q_p: number of reflectors k). */
int spaqr_num_ops(const spaqr_handle* h, int64_t* count);
int spaqr_op_info(const spaqr_handle* h, int64_t i, int* kind, int* stage, int* c, int* w);
/* Copy op i to host memory: slots (c ints), nslots (w ints, R_s only),
 * R (c x c column-major; R_s/R_p) or V (c x w reflectors, Q_p), Rn (c x w,
 * R_s only), taus (w, Q_p only).  Unused outputs may be NULL. */
int spaqr_op_copy(const spaqr_handle* h, int64_t i, int32_t* slots, int32_t* nslots, double* R, double* Rn,
                  double* taus);

const char* spaqr_last_error(void);
void spaqr_destroy(spaqr_handle* h);

/* Device and pinned host blocks that the library freed (a factorization's
 * working pools, upload arena, W store and operator) are kept in a
 * process-wide cache and handed out again to later factorizations of the
 * same or smaller sizes; the cache waits for the device before it takes a
 * block back, as cudaFree does.  spaqr_release_cached_memory returns every
 * cached block to the driver (after cudaDeviceSynchronize on the current
 * device); spaqr_cached_bytes reports their total size.  Blocks owned by live
 * handles are not affected.  Thread-safe; host only. */
void spaqr_release_cached_memory(void);
size_t spaqr_cached_bytes(void);

/* ---------------------------------------------------------------- autotuning
 * spaqr_autotune: times, for every size class of the column-pivoted QRs
 * (m and n in powers of two, 128..max_m rows, 64..max_n columns, at most 4M
 * entries), each launch shape -- a cluster of 1, 2, 4, 8 or 16 CTAs with the
 * column slabs in shared memory, or 16 CTAs over a global work copy -- on
 * synthetic full-rank matrices that fill the GPU, and installs the fastest per
 * class for every later factorization of this process in that precision
 * (SPAQR_PREC_FP64: FP64 kernels, SPAQR_PREC_MIXED: FP32 kernels).  Writes the
 * table (with the timings as comments) to path when path != NULL; *seconds
 * (may be NULL) receives the tuning time.  Untuned classes keep the built-in
 * rule.  Errors: INVALID_ARG, NO_DEVICE, OOM, CUDA.
 * spaqr_load_tuning: installs a table written by spaqr_autotune (path = NULL
 * removes the table).  Errors: INVALID_ARG (unreadable or malformed file). */
int spaqr_autotune(int precision, int max_m, int max_n, const char* path, double* seconds);
int spaqr_load_tuning(const char* path);

/* ----------------------------------------------------- batched dense kernels
 * The dense building blocks of the factorization, exposed for testing.  Each
 * takes `count` problems described by host arrays; A[i] are device pointers
 * to column-major matrices; stream as in spaqr_options.
 *
 * spaqr_dense_front_qr: Householder QR (Section 2.3) of the first c[i]
 * columns of the m[i] x n[i] matrix A[i], every reflector applied to the
 * remaining columns; afterwards rows 0..c-1 hold R (diag >= 0, zeros below
 * the diagonal in the first c columns) and rows c.. the transformed rows.
 * Requires c[i] <= m[i]. */
int spaqr_dense_front_qr(int count, double* const* A, const int* m, const int* n, const int* c, const int* ld,
                         void* stream);

/* spaqr_dense_front_qr_f32: the same Householder QR on FP32 matrices, as the
 * mixed-precision factorization runs it: fronts too large for shared memory
 * take the blocked path with the trailing updates C <- C - V T^T V^T C on the
 * tensor cores (tcgen05, 3xTF32 with FP32 accumulation).  Errors as
 * spaqr_dense_front_qr, plus TIMEOUT if a tensor-core completion wait gave up. */
int spaqr_dense_front_qr_f32(int count, float* const* A, const int* m, const int* n, const int* c, const int* ld,
                             void* stream);

/* spaqr_dense_tc_gemm: C <- C - A B for FP32 column-major device matrices
 * (A m x k, lda; B k x n, ldb; C m x n, ldc) on the tensor cores in 3xTF32 --
 * the product that the FP32 trailing updates use, exposed for testing.
 * Errors: INVALID_ARG (negative sizes, short leading dimensions), TIMEOUT. */
int spaqr_dense_tc_gemm(int m, int n, int k, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                        void* stream);

/* spaqr_dense_qrcp: column-pivoted Householder QR stopped at the rank
 * k = max r with |R_ii| >= eps |R_11| and R_ii != 0 (Section 4).  On return
 * rank[i] (host) = k; A[i] rows 0..k-1 hold the first k rows of Q^T A[i] in the
 * ORIGINAL column order; columns 0..k-1 of V[i] (device, m[i] x min(m,n),
 * ld = m[i]) hold the reflectors (unit diagonal) and taus[i] (device) their
 * scalars, so that Q = H_1 ... H_k. */
int spaqr_dense_qrcp(int count, double* const* A, const int* m, const int* n, const int* ld, double eps,
                     double* const* V, double* const* taus, int* rank, void* stream);

/* spaqr_dense_qrcp_route: spaqr_dense_qrcp with the launch form chosen by
 * route: SPAQR_QRCP_CLUSTER = one thread-block cluster of at most 16 CTAs per
 * matrix, column slabs in shared memory or, when they do not fit, a global
 * work copy with delayed updates (what spaqr_dense_qrcp runs);
 * SPAQR_QRCP_AUTO = as the factorization runs it: matrices whose slabs need
 * more than 16 CTAs take a group of up to one CTA per SM, exchanging pivots and
 * reflectors through global memory (cooperative launch; bounded waits end in
 * SPAQR_ERR_TIMEOUT); SPAQR_QRCP_GRID = every matrix above the one-warp size
 * takes such a CTA group, over a global work copy when even the shared memory
 * of every SM cannot hold it (for testing the group forms).
 * Results agree with spaqr_dense_qrcp up to rounding. */
#define SPAQR_QRCP_AUTO 0
#define SPAQR_QRCP_CLUSTER 1
#define SPAQR_QRCP_GRID 2
int spaqr_dense_qrcp_route(int count, double* const* A, const int* m, const int* n, const int* ld, double eps,
                           double* const* V, double* const* taus, int* rank, int route, void* stream);
/* spaqr_dense_qrcp_f32: spaqr_dense_qrcp_route in FP32 (the arithmetic of the
 * mixed-precision factorization's pivoted QRs: FP32 data and updates, partial
 * column norms for the pivot order in FP32, R_ii and the eps rank test to FP64
 * accuracy in double-float arithmetic),
 * exposed for testing. */
int spaqr_dense_qrcp_f32(int count, float* const* A, const int* m, const int* n, const int* ld, double eps,
                         float* const* V, float* const* taus, int* rank, int route, void* stream);

/* spaqr_debug_set_qrcp_wait: failure-detection hook for tests.  The CTA
 * groups of the column-pivoted QR (the SPAQR_QRCP_GRID / AUTO forms above and
 * the factorization's large matrices) exchange pivots through arrival
 * counters in global memory; every wait on a counter gives up after `cycles`
 * SM clock cycles (<= 0 restores the default, about 2 s at the maximum SM
 * clock), writes rank -1 for its matrix and returns, and the host then
 * reports SPAQR_ERR_TIMEOUT.  missing_arrivals > 0 makes every wait expect
 * that many arrivals more than there are CTAs, so that it expires without
 * fail (the CUDA context stays usable); 0 restores normal operation.
 * Process-wide; affects launches issued after the call.  Host only; always
 * returns SPAQR_OK. */
int spaqr_debug_set_qrcp_wait(long long cycles, int missing_arrivals);

/* spaqr_dense_qrcp_static: the same batched column-pivoted QR as
 * spaqr_dense_qrcp (same arguments, same results), for callers that cannot
 * allocate device memory: code that runs under a memory manager which owns
 * all device memory (a framework's caching allocator, a fixed per-process
 * budget), or latency-critical code that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree may cause.  The paper has no
 * counterpart.  It calls no cudaMalloc, cudaFree or allocating library routine: the
 * descriptor array, the rank slots and the work copies of matrices too wide
 * for shared memory live in one static device array of 4 MiB
 * (4,194,304 bytes), reserved on every GPU that loads the library until the
 * process exits.  A batch whose scratch exceeds it fails with
 * SPAQR_ERR_CAPACITY and a message giving both sizes.  The first call on a
 * device looks up the array's device address (with that device current);
 * make that first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents; nothing in it needs to start at
 * zero.  Calls that overlap on the GPU (other streams, other host threads)
 * race on the array: serialise them.  Returns with `stream` synchronised.
 * Host exceptions (a failed host allocation) come back as SPAQR_ERR_OOM. */
int spaqr_dense_qrcp_static(int count, double* const* A, const int* m, const int* n, const int* ld, double eps,
                            double* const* V, double* const* taus, int* rank, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SPAQR_H */
