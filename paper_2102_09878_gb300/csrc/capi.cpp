// C ABI of the library (declared in include/spaqr.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <exception>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "kernels.h"
#include "parallel.h"

struct spaqr_analysis {
  std::unique_ptr<spaqr::Analysis> an;
};
struct spaqr_handle {
  std::unique_ptr<spaqr::Handle> h;
};

namespace {
thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

using spaqr::guarded;

int need_device() {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return fail(SPAQR_ERR_NO_DEVICE, "no CUDA device");
  }
  return SPAQR_OK;
}

double secs_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// successive sections of handle construction, printed in verbose mode
struct Tick {
  bool on;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  explicit Tick(int verbose) : on(verbose != 0) {}
  void operator()(const char* what) {
    if (!on) return;
    std::fprintf(stderr, "[spaqr] handle: %-28s %8.3f ms\n", what, 1e3 * secs_since(t));
    t = std::chrono::steady_clock::now();
  }
};

// The pattern of A^T in CSR form (column pointers, row indices) and, per
// transposed entry, its position in A; the entries of a column keep the row
// order.  Serial: it runs on a helper thread beside the factorization.
void transpose_pattern(const spaqr_csr& A, std::vector<int64_t>& trp, std::vector<int32_t>& tci,
                       std::vector<int64_t>& tperm) {
  for (int64_t q = 0; q < A.nnz; ++q) trp[(size_t)A.colidx[q] + 1]++;
  for (int64_t j = 0; j < A.n; ++j) trp[(size_t)j + 1] += trp[(size_t)j];
  std::vector<int64_t> pos(trp.begin(), trp.end() - 1);
  for (int64_t r = 0; r < A.m; ++r)
    for (int64_t q = A.rowptr[r]; q < A.rowptr[r + 1]; ++q) {
      const int64_t t = pos[(size_t)A.colidx[q]]++;
      tci[(size_t)t] = (int32_t)r;
      tperm[(size_t)t] = q;
    }
}

// Column scaling D (Section 2.7): D_j = 1 / ||A e_j||, each squared norm summed
// over the column's entries in row order.  Threads own disjoint column ranges
// and each scans all of A, so the result does not depend on the thread count.
void column_scaling(const spaqr_csr& A, std::vector<double>& D) {
  const int64_t n = A.n;
  D.assign((size_t)n, 0.0);
  const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(spaqr::ThreadPool::get().workers(), n / 4096));
  spaqr::parallel_for(parts, [&](int64_t b, int64_t e, int) {
    for (int64_t p = b; p < e; ++p) {
      const int64_t c0 = n * p / parts, c1 = n * (p + 1) / parts;
      const uint32_t w = (uint32_t)(c1 - c0);
      for (int64_t q = 0; q < A.nnz; ++q) {
        const uint32_t d = (uint32_t)(A.colidx[q] - c0);
        if (d < w) D[(size_t)A.colidx[q]] += A.vals[q] * A.vals[q];
      }
    }
  }, 1);
  for (int64_t j = 0; j < n; ++j) {
    if (!(D[(size_t)j] > 0.0)) throw spaqr::Error(SPAQR_ERR_RANK_DEFICIENT, "zero column " + std::to_string(j));
    D[(size_t)j] = 1.0 / std::sqrt(D[(size_t)j]);
  }
}

// The scaled operator A~ = A D (FP64) and its transpose on the device, built
// and uploaded on a stream of its own (the host copies are kept until the
// uploads are done).
void upload_operator(spaqr::Handle& h, const spaqr_csr& A, cudaStream_t st) {
  std::vector<int64_t> trp((size_t)A.n + 1, 0);
  std::vector<int32_t> tci((size_t)A.nnz);
  std::vector<int64_t> tperm((size_t)A.nnz);
  transpose_pattern(A, trp, tci, tperm);
  std::vector<double> v((size_t)A.nnz), tv((size_t)A.nnz);
  for (int64_t q = 0; q < A.nnz; ++q) v[(size_t)q] = A.vals[q] * h.D[(size_t)A.colidx[q]];
  for (int64_t q = 0; q < A.nnz; ++q) tv[(size_t)q] = v[(size_t)tperm[(size_t)q]];
  SPAQR_CUDA(spaqr::dmalloc(&h.d_rowptr, (size_t)(A.m + 1) * sizeof(int64_t)));
  SPAQR_CUDA(spaqr::dmalloc(&h.d_colidx, (size_t)std::max<int64_t>(A.nnz, 1) * sizeof(int32_t)));
  SPAQR_CUDA(spaqr::dmalloc(&h.d_vals, (size_t)std::max<int64_t>(A.nnz, 1) * sizeof(double)));
  SPAQR_CUDA(spaqr::dmalloc(&h.d_trowptr, (size_t)(A.n + 1) * sizeof(int64_t)));
  SPAQR_CUDA(spaqr::dmalloc(&h.d_tcolidx, (size_t)std::max<int64_t>(A.nnz, 1) * sizeof(int32_t)));
  SPAQR_CUDA(spaqr::dmalloc(&h.d_tvals, (size_t)std::max<int64_t>(A.nnz, 1) * sizeof(double)));
  SPAQR_CUDA(spaqr::dmalloc(&h.d_D, (size_t)A.n * sizeof(double)));
  SPAQR_CUDA(spaqr::dmalloc(&h.d_tperm, (size_t)std::max<int64_t>(A.nnz, 1) * sizeof(int64_t)));
  SPAQR_CUDA(cudaMemcpyAsync(h.d_rowptr, A.rowptr, (size_t)(A.m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  SPAQR_CUDA(cudaMemcpyAsync(h.d_trowptr, trp.data(), trp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  SPAQR_CUDA(cudaMemcpyAsync(h.d_D, h.D.data(), h.D.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  if (A.nnz) {
    SPAQR_CUDA(cudaMemcpyAsync(h.d_colidx, A.colidx, (size_t)A.nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    SPAQR_CUDA(cudaMemcpyAsync(h.d_vals, v.data(), (size_t)A.nnz * sizeof(double), cudaMemcpyHostToDevice, st));
    SPAQR_CUDA(cudaMemcpyAsync(h.d_tcolidx, tci.data(), tci.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    SPAQR_CUDA(cudaMemcpyAsync(h.d_tvals, tv.data(), tv.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    SPAQR_CUDA(cudaMemcpyAsync(h.d_tperm, tperm.data(), tperm.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  }
  SPAQR_CUDA(cudaStreamSynchronize(st));
}
}  // namespace

namespace spaqr {
void set_last_error(const std::string& msg) { g_last_error = msg; }

void Handle::wait_caller() {
  if (!ev) SPAQR_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  SPAQR_CUDA(cudaEventRecord(ev, user_st));
  SPAQR_CUDA(cudaStreamWaitEvent(st, ev, 0));
}

Handle::~Handle() {
  free_apply_plan(*this);
  if (ev) cudaEventDestroy(ev);
  dfree(d_rowptr);
  dfree(d_colidx);
  dfree(d_vals);
  dfree(d_trowptr);
  dfree(d_tcolidx);
  dfree(d_tvals);
  dfree(d_D);
  dfree(d_tperm);
  cudaFree(d_work);
  cudaFree(d_flag);
  if (own_stream && st) cudaStreamDestroy(st);
}
}  // namespace spaqr

namespace {
// The CSR arrays of A are well formed (sizes, monotone rowptr, column indices in range).
void check_csr(const spaqr_csr* A) {
  if (A->m < 0 || A->n <= 0 || A->nnz < 0) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "bad sizes");
  if (!A->rowptr || !A->colidx || !A->vals) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "null CSR array");
  if (A->rowptr[0] != 0 || A->rowptr[A->m] != A->nnz) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "bad rowptr");
  for (int64_t r = 0; r < A->m; ++r)
    if (A->rowptr[r + 1] < A->rowptr[r]) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "rowptr not monotone");
  for (int64_t e = 0; e < A->nnz; ++e)
    if (A->colidx[e] < 0 || A->colidx[e] >= A->n) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "column index out of range");
}

// Host-side checks of a matrix and options (before any device work, so that
// they also answer without a GPU).
void check_input(const spaqr_csr* A, const spaqr::Analysis& a, const spaqr_options& opt) {
  if (A->n != a.n) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "A has n != nx*ny*nz columns");
  if (A->m < A->n) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "A must have m >= n");
  check_csr(A);
  if (A->match) {
    std::vector<char> used((size_t)A->m, 0);
    for (int64_t j = 0; j < A->n; ++j) {
      const int64_t r = A->match[j];
      if (r < 0 || r >= A->m || used[(size_t)r]) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "match is not a matching");
      used[(size_t)r] = 1;
      bool has = false;
      for (int64_t e = A->rowptr[r]; e < A->rowptr[r + 1] && !has; ++e) has = A->colidx[e] == j;
      if (!has) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "matched row " + std::to_string(r) + " has no entry in column " +
                                                              std::to_string(j));
    }
  }
  if (opt.skip < 0) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "skip must be >= 0");
  if (opt.row_rule != SPAQR_ROWS_TREE && opt.row_rule != SPAQR_ROWS_ANY)
    throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "unknown row rule");
  if (!(opt.eps >= 0.0)) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "eps must be >= 0");
  if (opt.precision != SPAQR_PREC_FP64 && opt.precision != SPAQR_PREC_MIXED)
    throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "unknown precision");
  if (opt.mode != SPAQR_MODE_SPAQR && opt.mode != SPAQR_MODE_DIRECT && opt.mode != SPAQR_MODE_DIAG)
    throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "unknown mode");
  if (opt.step1_qr_width < 0) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "step1_qr_width must be >= 0");
}

// Checks A, factors it and builds the solve-side state (spaqr_factor and the
// refactorization of spaqr_update_values).
std::unique_ptr<spaqr::Handle> build_handle(const spaqr_csr* A, const spaqr::Analysis& a, const spaqr_options& opt) {
  auto t0 = std::chrono::steady_clock::now();
  check_input(A, a, opt);
  auto hd = std::make_unique<spaqr::Handle>();
  spaqr::Handle& h = *hd;
  h.opt = opt;
  // all library work runs on a non-blocking stream of its own unless the
  // caller gives one (the legacy default stream cannot be graph-captured)
  h.user_st = static_cast<cudaStream_t>(h.opt.stream);
  if (h.user_st) {
    h.st = h.user_st;
  } else {
    SPAQR_CUDA(cudaStreamCreateWithFlags(&h.st, cudaStreamNonBlocking));
    h.own_stream = true;
  }
  h.precision = h.opt.precision;
  h.m = A->m;
  h.n = A->n;
  h.nnz = A->nnz;
  h.depth = a.depth;
  h.t_analyze = a.seconds;
  Tick tick(h.opt.verbose);
  column_scaling(*A, h.D);
  tick("column scaling");
  // the scaled operator and its transpose are built and uploaded by a helper
  // thread on a stream of its own while this thread runs the factorization
  int dev = 0;
  SPAQR_CUDA(cudaGetDevice(&dev));
  cudaStream_t up_st = nullptr;
  SPAQR_CUDA(cudaStreamCreateWithFlags(&up_st, cudaStreamNonBlocking));
  std::exception_ptr up_err;
  std::thread up_thread([&] {
    try {
      SPAQR_CUDA(cudaSetDevice(dev));
      upload_operator(h, *A, up_st);
    } catch (...) {
      up_err = std::current_exception();
    }
  });
  struct Finish {  // the helper joined and its stream released however this scope is left
    std::thread& t;
    cudaStream_t s;
    ~Finish() {
      if (t.joinable()) t.join();
      if (s) cudaStreamDestroy(s);
    }
  } finish{up_thread, up_st};
  // Diag. comparator (Section 4): no factorization, W = I
  if (h.opt.mode != SPAQR_MODE_DIAG) spaqr::run_factor(h, *A, a);
  tick("factor");
  up_thread.join();
  if (up_err) std::rethrow_exception(up_err);
  tick("operator upload (wait)");
  h.rowptr.assign(A->rowptr, A->rowptr + A->m + 1);
  h.colidx.assign(A->colidx, A->colidx + A->nnz);
  if (A->match) h.match.assign(A->match, A->match + A->n);
  spaqr::build_apply_plan(h);
  tick("apply plan");
  SPAQR_CUDA(cudaStreamSynchronize(h.st));
  tick("final wait");
  int64_t nnzW = 0;
  for (auto& op : h.ops) {
    const int64_t c = op.c;
    if (op.kind == 0)
      nnzW += c * (c + 1) / 2 + c * op.w;
    else if (op.kind == 1)
      nnzW += c * (c + 1) / 2;
    else
      nnzW += c * op.k;
  }
  h.stats.nnz_W = nnzW;
  h.stats.n_ops = (int64_t)h.ops.size();
  h.stats.t_analyze = h.t_analyze;
  h.stats.t_factor = secs_since(t0);
  return hd;
}

}  // namespace

namespace {
template <typename T>
int dense_qrcp_route_t(int count, T* const* A, const int* m, const int* n, const int* ld, double eps, T* const* V,
                       T* const* taus, int* rank, int route, void* stream) {
  if (count < 0 || (count > 0 && (!A || !m || !n || !ld || !rank)) ||
      (route != SPAQR_QRCP_AUTO && route != SPAQR_QRCP_CLUSTER && route != SPAQR_QRCP_GRID))
    return fail(SPAQR_ERR_INVALID_ARG, "bad arguments");
  if (int rc = need_device()) return rc;
  return guarded([&] {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int lim = spaqr::max_smem_optin();
    std::vector<spaqr::QrcpDesc<T>> qs;
    std::vector<int> ms, ns;
    std::vector<void*> bufs;
    struct Free {
      std::vector<void*>& b;
      ~Free() {
        for (void* p : b) cudaFree(p);
      }
    } free_all{bufs};
    auto dev_alloc = [&](size_t bytes) {
      void* p = nullptr;
      SPAQR_CUDA(cudaMalloc(&p, std::max<size_t>(bytes, 1)));
      bufs.push_back(p);
      return p;
    };
    int* d_rank = static_cast<int*>(dev_alloc(std::max(count, 1) * sizeof(int)));
    for (int i = 0; i < count; ++i) {
      if (m[i] < 0 || n[i] < 0 || ld[i] < std::max(1, m[i])) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "bad shape");
      qs.push_back(spaqr::QrcpDesc<T>{A[i], nullptr, A[i], V ? V[i] : nullptr, taus ? taus[i] : nullptr,
                                           d_rank + i, m[i], n[i], ld[i], ld[i]});
      ms.push_back(m[i]);
      ns.push_back(n[i]);
    }
    const int gctas = route == SPAQR_QRCP_CLUSTER ? 0 : spaqr::qrcp_grid_capacity(lim, (int)sizeof(T));
    std::vector<spaqr::QrcpGroup> groups;
    std::vector<char> need_work;
    if (!spaqr::plan_qrcp(ms, ns, (int)sizeof(T), lim, groups, need_work, gctas, route == SPAQR_QRCP_GRID))
      throw spaqr::Error(SPAQR_ERR_CAPACITY, "too many columns");
    for (int i = 0; i < count; ++i)
      if (need_work[(size_t)i])
        qs[(size_t)i].work =
            static_cast<T*>(dev_alloc((size_t)std::max(1, m[i]) * std::max(1, n[i]) * sizeof(T)));
    auto* d = static_cast<spaqr::QrcpDesc<T>*>(dev_alloc(std::max<size_t>(qs.size(), 1) * sizeof(qs[0])));
    size_t off = 0;
    for (auto& g : groups) {
      std::vector<spaqr::QrcpDesc<T>> part;
      for (int i : g.idx) part.push_back(qs[(size_t)i]);
      SPAQR_CUDA(cudaMemcpyAsync(d + off, part.data(), part.size() * sizeof(part[0]), cudaMemcpyHostToDevice, st));
      if (g.grid) {
        size_t bytes = 0;
        for (int c : g.ctas) bytes += spaqr::qrcp_grid_xchg_bytes(c, g.m_max, (int)sizeof(T));
        unsigned char* x = static_cast<unsigned char*>(dev_alloc(bytes));
        SPAQR_CUDA(cudaMemsetAsync(x, 0, bytes, st));
        std::vector<spaqr::QrcpGridDesc> gd;
        const int cta0 = spaqr::qrcp_grid_descs(g.ctas, g.m_max, (int)sizeof(T), x, gd);
        auto* dgd = static_cast<spaqr::QrcpGridDesc*>(dev_alloc(gd.size() * sizeof(gd[0])));
        SPAQR_CUDA(cudaMemcpyAsync(dgd, gd.data(), gd.size() * sizeof(gd[0]), cudaMemcpyHostToDevice, st));
        SPAQR_CUDA(spaqr::launch_qrcp_grid<T>(d + off, dgd, (int)part.size(), cta0, eps, g.nl_max, g.m_max, g.slab, st));
      } else {
        SPAQR_CUDA(spaqr::launch_qrcp<T>(d + off, (int)part.size(), eps, g.cs, g.nl_max, g.m_max, g.slab, st, g.nb));
      }
      off += part.size();
    }
    SPAQR_CUDA(cudaMemcpyAsync(rank, d_rank, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, st));
    SPAQR_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < count; ++i)  // only an expired exchange wait writes a negative rank
      if (rank[i] < 0)
        return fail(SPAQR_ERR_TIMEOUT, "column-pivoted QR exchange wait timed out (matrix " + std::to_string(i) + ")");
    return SPAQR_OK;
  });
}

// spaqr_solve (CGLS, Section 4) and spaqr_solve_csne (corrected seminormal
// equations, Section 1) with host or device b and x.
int solve_any(spaqr_handle* hh, const double* b, double* x, int on_device, spaqr_solve_info* info, bool csne) {
  if (!hh || !b || !x) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    spaqr::Handle& h = *hh->h;
    const double* bd = b;
    double* xd = x;
    double* tmp = nullptr;
    if (on_device) h.wait_caller();
    if (!on_device) {
      SPAQR_CUDA(cudaMalloc(&tmp, (size_t)(h.m + h.n) * sizeof(double)));
      SPAQR_CUDA(cudaMemcpyAsync(tmp, b, (size_t)h.m * sizeof(double), cudaMemcpyHostToDevice, h.st));
      bd = tmp;
      xd = tmp + h.m;
    }
    spaqr_solve_info inf{};
    try {
      if (csne)
        spaqr::csne(h, bd, xd, &inf);
      else
        spaqr::cgls(h, bd, xd, &inf);
    } catch (...) {
      cudaStreamSynchronize(h.st);
      cudaFree(tmp);
      throw;
    }
    if (!on_device) {
      SPAQR_CUDA(cudaMemcpyAsync(x, xd, (size_t)h.n * sizeof(double), cudaMemcpyDeviceToHost, h.st));
      SPAQR_CUDA(cudaStreamSynchronize(h.st));
      cudaFree(tmp);
    }
    if (info) *info = inf;
    return inf.converged ? SPAQR_OK
                         : fail(SPAQR_ERR_NOT_CONVERGED, csne ? "CSNE refinement reached maxit" : "CGLS reached maxit");
  });
}

}  // namespace

extern "C" {

void spaqr_default_options(spaqr_options* o) {
  if (!o) return;
  o->eps = 1e-4;
  o->skip = 2;
  o->precision = SPAQR_PREC_FP64;
  o->mode = SPAQR_MODE_SPAQR;
  o->tol = 1e-10;
  o->maxit = 500;
  o->use_graphs = 1;
  o->verbose = 0;
  o->stream = nullptr;
  o->row_rule = SPAQR_ROWS_TREE;
  o->apply_persistent = 0;
  o->step1_qr_width = 1280;
}

const char* spaqr_last_error(void) { return g_last_error.c_str(); }

int spaqr_analyze(const spaqr_grid_ordering* ord, spaqr_analysis** out) {
  if (!ord || !out) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    auto* a = new spaqr_analysis();
    a->an.reset(spaqr::build_analysis(ord->nx, ord->ny, ord->nz, ord->depth));
    *out = a;
    return SPAQR_OK;
  });
}

int spaqr_analyze_matrix(const spaqr_csr* A, int depth, spaqr_analysis** out) {
  if (!A || !out) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    check_csr(A);
    auto* a = new spaqr_analysis();
    a->an.reset(spaqr::build_analysis_matrix(A->m, A->n, A->rowptr, A->colidx, depth));
    *out = a;
    return SPAQR_OK;
  });
}

int spaqr_match(const spaqr_csr* A, int32_t* match) {
  if (!A || !match) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    check_csr(A);
    if (A->m < A->n) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "A must have m >= n");
    if (!spaqr::max_weight_matching(A->m, A->n, A->rowptr, A->colidx, A->vals, match))
      throw spaqr::Error(SPAQR_ERR_RANK_DEFICIENT, "A has no matching of every column to a distinct row (structurally "
                                                   "rank deficient)");
    return SPAQR_OK;
  });
}

void spaqr_analysis_destroy(spaqr_analysis* an) { delete an; }

int spaqr_analysis_stage_size(const spaqr_analysis* an, int k, int64_t* nclusters, int64_t* nverts) {
  if (!an || !nclusters || !nverts) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  if (k < 1 || k > an->an->depth) return fail(SPAQR_ERR_INVALID_ARG, "stage out of range");
  const auto& st = an->an->stages[(size_t)k];
  *nclusters = (int64_t)st.node.size();
  *nverts = (int64_t)st.verts.size();
  return SPAQR_OK;
}

int spaqr_analysis_stage_clusters(const spaqr_analysis* an, int k, int32_t* node, int32_t* level, int64_t* vptr,
                                  int32_t* verts) {
  if (!an || !node || !level || !vptr || !verts) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  if (k < 1 || k > an->an->depth) return fail(SPAQR_ERR_INVALID_ARG, "stage out of range");
  const auto& st = an->an->stages[(size_t)k];
  std::copy(st.node.begin(), st.node.end(), node);
  std::copy(st.level.begin(), st.level.end(), level);
  std::copy(st.vptr.begin(), st.vptr.end(), vptr);
  std::copy(st.verts.begin(), st.verts.end(), verts);
  return SPAQR_OK;
}

int spaqr_factor(const spaqr_csr* A, const spaqr_analysis* an, const spaqr_options* opt, spaqr_handle** out) {
  if (!A || !an || !out) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  spaqr_options o;
  if (opt)
    o = *opt;
  else
    spaqr_default_options(&o);
  if (int rc = guarded([&] {
        check_input(A, *an->an, o);
        return SPAQR_OK;
      }))
    return rc;
  if (int rc = need_device()) return rc;
  return guarded([&] {
    auto hd = build_handle(A, *an->an, o);
    auto* out_h = new spaqr_handle();
    out_h->h = std::move(hd);
    *out = out_h;
    return SPAQR_OK;
  });
}

int spaqr_factor_batch(int count, const spaqr_csr* const* A, const spaqr_analysis* an, const spaqr_options* opt,
                       spaqr_handle** out) {
  if (count < 0 || (count > 0 && (!A || !an || !out))) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  for (int i = 0; i < count; ++i)
    if (!A[i]) return fail(SPAQR_ERR_INVALID_ARG, "null matrix");
  if (opt && opt->stream) return fail(SPAQR_ERR_INVALID_ARG, "a batch gives every handle its own stream");
  if (count == 0) return SPAQR_OK;
  if (int rc = need_device()) return rc;
  spaqr_options o;
  if (opt)
    o = *opt;
  else
    spaqr_default_options(&o);
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<std::unique_ptr<spaqr::Handle>> hs((size_t)count);
  std::vector<int> codes((size_t)count, SPAQR_OK);
  std::vector<std::string> msgs((size_t)count);
  const int nt = std::max(1, std::min({count, (int)std::thread::hardware_concurrency(), 16}));
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      cudaSetDevice(dev);
      for (int i = t; i < count; i += nt) {
        try {
          hs[(size_t)i] = build_handle(A[i], *an->an, o);
        } catch (const spaqr::Error& e) {
          codes[(size_t)i] = e.code;
          msgs[(size_t)i] = e.what();
        } catch (const std::bad_alloc&) {
          codes[(size_t)i] = SPAQR_ERR_OOM;
          msgs[(size_t)i] = "host allocation failed";
        } catch (const std::exception& e) {
          codes[(size_t)i] = SPAQR_ERR_CUDA;
          msgs[(size_t)i] = e.what();
        }
      }
    });
  for (auto& t : th) t.join();
  for (int i = 0; i < count; ++i)
    if (codes[(size_t)i] != SPAQR_OK) return fail(codes[(size_t)i], "problem " + std::to_string(i) + ": " + msgs[(size_t)i]);
  for (int i = 0; i < count; ++i) {
    auto* h = new spaqr_handle();
    h->h = std::move(hs[(size_t)i]);
    out[i] = h;
  }
  return SPAQR_OK;
}

void spaqr_destroy(spaqr_handle* h) { delete h; }

void spaqr_release_cached_memory(void) { spaqr::release_cached_memory(); }

size_t spaqr_cached_bytes(void) { return spaqr::cached_bytes(); }

int spaqr_solve(spaqr_handle* hh, const double* b, double* x, int on_device, spaqr_solve_info* info) {
  return solve_any(hh, b, x, on_device, info, false);
}

int spaqr_solve_csne(spaqr_handle* hh, const double* b, double* x, int on_device, spaqr_solve_info* info) {
  return solve_any(hh, b, x, on_device, info, true);
}

int spaqr_apply_Winv(spaqr_handle* hh, double* z, int transpose) {
  if (!hh || !z) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    hh->h->wait_caller();
    spaqr::apply_Winv(*hh->h, z, transpose ? 1 : 0);
    SPAQR_CUDA(cudaStreamSynchronize(hh->h->st));
    return SPAQR_OK;
  });
}

int spaqr_apply_A(spaqr_handle* hh, const double* x, double* y, int forward) {
  if (!hh || !x || !y) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    hh->h->wait_caller();
    spaqr::apply_A(*hh->h, x, y, forward ? 1 : 0);
    SPAQR_CUDA(cudaStreamSynchronize(hh->h->st));
    return SPAQR_OK;
  });
}

namespace {
// Device staging of host vectors for the calls that take on_device = 0.
struct Staged {
  double* base = nullptr;
  ~Staged() {
    if (base) cudaFree(base);
  }
};

// Runs IterSolve on several handles; in/out are host or device vectors.  CGLS
// (kind 0) stops at each handle's own tolerance, PCG (kind 1) at tol.
int run_batch(int count, spaqr_handle* const* hs, const double* const* in, double* const* out, int on_device,
              int kind, double tol, spaqr_solve_info* infos) {
  if (count < 0 || (count > 0 && (!hs || !in || !out))) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  for (int i = 0; i < count; ++i)
    if (!hs[i] || !in[i] || !out[i]) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  if (kind == 1 && !(tol > 0.0)) return fail(SPAQR_ERR_INVALID_ARG, "tol must be > 0");
  return guarded([&] {
    std::vector<Staged> stage((size_t)count);
    std::vector<spaqr::IterSolve> S((size_t)count);
    for (int i = 0; i < count; ++i) {
      spaqr::Handle& h = *hs[i]->h;
      const int64_t nin = kind == 0 ? h.m : h.n;
      spaqr::IterSolve& s = S[(size_t)i];
      s.h = &h;
      s.kind = kind;
      s.tol = kind == 0 ? h.opt.tol : tol;
      s.maxit = h.opt.maxit;
      if (on_device) {
        h.wait_caller();
        s.rhs = in[i];
        s.out = out[i];
      } else {
        SPAQR_CUDA(cudaMalloc(&stage[(size_t)i].base, (size_t)(nin + h.n) * sizeof(double)));
        SPAQR_CUDA(cudaMemcpyAsync(stage[(size_t)i].base, in[i], (size_t)nin * sizeof(double), cudaMemcpyHostToDevice,
                                   h.st));
        s.rhs = stage[(size_t)i].base;
        s.out = stage[(size_t)i].base + nin;
      }
    }
    spaqr::run_iterative(S);
    bool all = true;
    for (int i = 0; i < count; ++i) {
      spaqr::Handle& h = *hs[i]->h;
      if (!on_device) {
        SPAQR_CUDA(cudaMemcpyAsync(out[i], S[(size_t)i].out, (size_t)h.n * sizeof(double), cudaMemcpyDeviceToHost, h.st));
        SPAQR_CUDA(cudaStreamSynchronize(h.st));
      }
      spaqr_solve_info inf{};
      S[(size_t)i].report(&inf);
      if (infos) infos[i] = inf;
      all = all && inf.converged;
    }
    return all ? SPAQR_OK : fail(SPAQR_ERR_NOT_CONVERGED, kind == 0 ? "CGLS reached maxit" : "PCG reached maxit");
  });
}
}  // namespace

int spaqr_solve_batch(int count, spaqr_handle* const* hs, const double* const* b, double* const* x, int on_device,
                      spaqr_solve_info* infos) {
  if (count == 0) return SPAQR_OK;
  return run_batch(count, hs, b, x, on_device, 0, 0.0, infos);
}

int spaqr_solve_normal_batch(int count, spaqr_handle* const* hs, const double* const* g, double* const* lambda,
                             int on_device, double tol, spaqr_solve_info* infos) {
  if (count == 0) return SPAQR_OK;
  return run_batch(count, hs, g, lambda, on_device, 1, tol, infos);
}

int spaqr_solve_normal(spaqr_handle* hh, const double* g, double* lambda, int on_device, double tol,
                       spaqr_solve_info* info) {
  if (!hh || !g || !lambda) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  spaqr_handle* hs[1] = {hh};
  const double* in[1] = {g};
  double* out[1] = {lambda};
  return run_batch(1, hs, in, out, on_device, 1, tol, info);
}

int spaqr_lstsq_grad(spaqr_handle* hh, const double* b, const double* x, const double* lambda, double* grad_b,
                     double* grad_vals, int on_device) {
  if (!hh || !b || !x || !lambda) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    spaqr::Handle& h = *hh->h;
    if (on_device) {
      h.wait_caller();
      spaqr::lstsq_grad(h, b, x, lambda, grad_b, grad_vals);
      SPAQR_CUDA(cudaStreamSynchronize(h.st));
      return SPAQR_OK;
    }
    Staged st;
    const size_t m = (size_t)h.m, n = (size_t)h.n, nnz = (size_t)h.nnz;
    SPAQR_CUDA(cudaMalloc(&st.base, (2 * m + 2 * n + nnz) * sizeof(double)));
    double* db = st.base;
    double* dx = db + m;
    double* dl = dx + n;
    double* dgb = dl + n;
    double* dgv = dgb + m;
    SPAQR_CUDA(cudaMemcpyAsync(db, b, m * sizeof(double), cudaMemcpyHostToDevice, h.st));
    SPAQR_CUDA(cudaMemcpyAsync(dx, x, n * sizeof(double), cudaMemcpyHostToDevice, h.st));
    SPAQR_CUDA(cudaMemcpyAsync(dl, lambda, n * sizeof(double), cudaMemcpyHostToDevice, h.st));
    spaqr::lstsq_grad(h, db, dx, dl, grad_b ? dgb : nullptr, grad_vals ? dgv : nullptr);
    if (grad_b) SPAQR_CUDA(cudaMemcpyAsync(grad_b, dgb, m * sizeof(double), cudaMemcpyDeviceToHost, h.st));
    if (grad_vals) SPAQR_CUDA(cudaMemcpyAsync(grad_vals, dgv, nnz * sizeof(double), cudaMemcpyDeviceToHost, h.st));
    SPAQR_CUDA(cudaStreamSynchronize(h.st));
    return SPAQR_OK;
  });
}

int spaqr_update_values(spaqr_handle* hh, const spaqr_analysis* an, const double* vals, int on_device, int refactor) {
  if (!hh || !vals) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  if (refactor && !an) return fail(SPAQR_ERR_INVALID_ARG, "a refactorization needs the analysis");
  return guarded([&] {
    spaqr::Handle& h = *hh->h;
    const size_t nnz = (size_t)h.nnz;
    if (refactor) {
      std::vector<double> v(nnz);
      if (on_device) {
        h.wait_caller();
        SPAQR_CUDA(cudaMemcpyAsync(v.data(), vals, nnz * sizeof(double), cudaMemcpyDeviceToHost, h.st));
        SPAQR_CUDA(cudaStreamSynchronize(h.st));
      } else {
        std::copy(vals, vals + nnz, v.begin());
      }
      spaqr_csr A{h.m, h.n, h.nnz, h.rowptr.data(), h.colidx.data(), v.data(), h.match.empty() ? nullptr : h.match.data()};
      spaqr_options o = h.opt;
      auto fresh = build_handle(&A, *an->an, o);
      hh->h = std::move(fresh);
      return SPAQR_OK;
    }
    Staged st;
    const double* dv = vals;
    if (on_device) {
      h.wait_caller();
    } else {
      SPAQR_CUDA(cudaMalloc(&st.base, std::max<size_t>(nnz, 1) * sizeof(double)));
      SPAQR_CUDA(cudaMemcpyAsync(st.base, vals, nnz * sizeof(double), cudaMemcpyHostToDevice, h.st));
      dv = st.base;
    }
    spaqr::set_values(h, dv);
    SPAQR_CUDA(cudaStreamSynchronize(h.st));
    return SPAQR_OK;
  });
}

int spaqr_get_stats(const spaqr_handle* hh, spaqr_stats* st) {
  if (!hh || !st) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  *st = hh->h->stats;
  return SPAQR_OK;
}

int spaqr_num_ops(const spaqr_handle* hh, int64_t* count) {
  if (!hh || !count) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  *count = (int64_t)hh->h->ops.size();
  return SPAQR_OK;
}

int spaqr_op_info(const spaqr_handle* hh, int64_t i, int* kind, int* stage, int* c, int* w) {
  if (!hh) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  const auto& ops = hh->h->ops;
  if (i < 0 || i >= (int64_t)ops.size()) return fail(SPAQR_ERR_INVALID_ARG, "op index out of range");
  const auto& op = ops[(size_t)i];
  if (kind) *kind = op.kind;
  if (stage) *stage = op.stage;
  if (c) *c = op.c;
  if (w) *w = op.kind == 2 ? op.k : op.w;
  return SPAQR_OK;
}

int spaqr_op_copy(const spaqr_handle* hh, int64_t i, int32_t* slots, int32_t* nslots, double* R, double* Rn,
                  double* taus) {
  if (!hh) return fail(SPAQR_ERR_INVALID_ARG, "null argument");
  return guarded([&] {
    const spaqr::Handle& h = *hh->h;
    if (i < 0 || i >= (int64_t)h.ops.size()) throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "op index out of range");
    const auto& op = h.ops[(size_t)i];
    const bool f32 = h.precision == SPAQR_PREC_MIXED;
    const size_t es = f32 ? 4 : 8;
    auto fetch = [&](const void* src, size_t count, double* dst) {
      if (!dst || count == 0) return;
      std::vector<char> buf(count * es);
      SPAQR_CUDA(cudaMemcpy(buf.data(), src, count * es, cudaMemcpyDeviceToHost));
      for (size_t t = 0; t < count; ++t)
        dst[t] = f32 ? (double)reinterpret_cast<float*>(buf.data())[t] : reinterpret_cast<double*>(buf.data())[t];
    };
    if (slots) std::copy(op.slots.begin(), op.slots.end(), slots);
    if (nslots && op.kind == 0) std::copy(op.nslots.begin(), op.nslots.end(), nslots);
    const size_t c = (size_t)op.c;
    if (op.kind == 0) {
      fetch(op.R, c * c, R);
      if (Rn && op.w) fetch(static_cast<const char*>(op.R) + c * c * es, c * (size_t)op.w, Rn);
    } else if (op.kind == 1) {
      fetch(op.R, c * c, R);
    } else {
      fetch(op.V, c * (size_t)op.k, R);
      fetch(op.tau, (size_t)op.k, taus);
    }
    return SPAQR_OK;
  });
}

extern "C++" {
namespace {
template <typename T>
int dense_front_qr_t(int count, T* const* A, const int* m, const int* n, const int* c, const int* ld, void* stream) {
  if (count < 0 || (count > 0 && (!A || !m || !n || !c || !ld))) return fail(SPAQR_ERR_INVALID_ARG, "bad arguments");
  if (int rc = need_device()) return rc;
  return guarded([&] {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int lim = spaqr::max_smem_optin();
    std::vector<int> ms, ns, cs;
    for (int i = 0; i < count; ++i) {
      if (c[i] < 0 || c[i] > m[i] || n[i] < c[i] || ld[i] < std::max(1, m[i]))
        throw spaqr::Error(SPAQR_ERR_INVALID_ARG, "front " + std::to_string(i) + ": bad shape");
      ms.push_back(m[i]);
      ns.push_back(n[i]);
      cs.push_back(c[i]);
    }
    const auto groups = spaqr::plan_fronts(ms, ns, cs, (int)sizeof(T), lim);
    std::vector<std::vector<spaqr::FrontDesc<T>>> host(groups.size());
    std::vector<const spaqr::FrontDesc<T>*> dev(groups.size());
    std::vector<void*> frees;
    T* Tbuf = nullptr;
    for (size_t g = 0; g < groups.size(); ++g) {
      for (int i : groups[g].idx) host[g].push_back(spaqr::FrontDesc<T>{A[i], m[i], n[i], c[i], ld[i]});
      spaqr::FrontDesc<T>* d = nullptr;
      SPAQR_CUDA(cudaMalloc(&d, host[g].size() * sizeof(host[g][0])));
      frees.push_back(d);
      SPAQR_CUDA(cudaMemcpyAsync(d, host[g].data(), host[g].size() * sizeof(host[g][0]), cudaMemcpyHostToDevice, st));
      dev[g] = d;
      if (groups[g].kind == 2) {  // per front: a 32 x 32 T factor, later the sign mask of diag(R)
        int maxc = 0;
        for (auto& f : host[g]) maxc = std::max(maxc, f.c);
        const size_t per = std::max<size_t>(32 * 32 * sizeof(T), (size_t)((maxc + 31) / 32) * sizeof(unsigned));
        SPAQR_CUDA(cudaMalloc(&Tbuf, host[g].size() * per));
        frees.push_back(Tbuf);
      }
    }
    void* tc = nullptr;
    const size_t tcb = spaqr::front_groups_tc_bytes<T>(groups, host);
    if (tcb) {
      SPAQR_CUDA(cudaMalloc(&tc, tcb));
      frees.push_back(tc);
    }
    int* flag = nullptr;  // this call's tensor-core timeout flag
    SPAQR_CUDA(cudaMalloc(&flag, sizeof(int)));
    frees.push_back(flag);
    SPAQR_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    int64_t launches = 0;
    SPAQR_CUDA(spaqr::launch_front_groups<T>(groups, dev, host, Tbuf, st, &launches, tc, flag));
    int late = 0;
    SPAQR_CUDA(cudaMemcpyAsync(&late, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SPAQR_CUDA(cudaStreamSynchronize(st));
    for (void* p : frees) cudaFree(p);
    if (late) return fail(SPAQR_ERR_TIMEOUT, "tensor-core MMA completion wait timed out");
    return SPAQR_OK;
  });
}
}  // namespace
}

int spaqr_dense_front_qr(int count, double* const* A, const int* m, const int* n, const int* c, const int* ld,
                         void* stream) {
  return dense_front_qr_t<double>(count, A, m, n, c, ld, stream);
}

int spaqr_dense_front_qr_f32(int count, float* const* A, const int* m, const int* n, const int* c, const int* ld,
                             void* stream) {
  return dense_front_qr_t<float>(count, A, m, n, c, ld, stream);
}

int spaqr_dense_tc_gemm(int m, int n, int k, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                        void* stream) {
  if (m < 0 || n < 0 || k < 0 || (m * n * k > 0 && (!A || !B || !C)) || lda < std::max(1, m) ||
      ldb < std::max(1, k) || ldc < std::max(1, m))
    return fail(SPAQR_ERR_INVALID_ARG, "bad arguments");
  if (int rc = need_device()) return rc;
  return guarded([&] {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* flag = nullptr;  // this call's tensor-core timeout flag
    SPAQR_CUDA(cudaMalloc(&flag, sizeof(int)));
    int late = 0;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = spaqr::launch_tc_gemm(m, n, k, A, lda, B, ldb, C, ldc, flag, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&late, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(flag);
    SPAQR_CUDA(e);
    if (late) return fail(SPAQR_ERR_TIMEOUT, "tensor-core MMA completion wait timed out");
    return SPAQR_OK;
  });
}

int spaqr_debug_set_qrcp_wait(long long cycles, int missing_arrivals) {
  spaqr::qrcp_grid_set_wait(cycles, missing_arrivals);
  return SPAQR_OK;
}

int spaqr_dense_qrcp(int count, double* const* A, const int* m, const int* n, const int* ld, double eps,
                     double* const* V, double* const* taus, int* rank, void* stream) {
  return spaqr_dense_qrcp_route(count, A, m, n, ld, eps, V, taus, rank, SPAQR_QRCP_CLUSTER, stream);
}

int spaqr_dense_qrcp_route(int count, double* const* A, const int* m, const int* n, const int* ld, double eps,
                           double* const* V, double* const* taus, int* rank, int route, void* stream) {
  return dense_qrcp_route_t<double>(count, A, m, n, ld, eps, V, taus, rank, route, stream);
}

int spaqr_dense_qrcp_f32(int count, float* const* A, const int* m, const int* n, const int* ld, double eps,
                         float* const* V, float* const* taus, int* rank, int route, void* stream) {
  return dense_qrcp_route_t<float>(count, A, m, n, ld, eps, V, taus, rank, route, stream);
}

}  // extern "C"
