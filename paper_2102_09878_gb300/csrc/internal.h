// Internal types shared by the factorization, the solve and the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <chrono>
#include <vector>

#include "../../include/spaqr.h"
#include "symbolic.h"

namespace spaqr {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& msg) : std::runtime_error(msg), code(c) {}
};

#define SPAQR_CUDA(x)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (x);                                                                          \
    if (e_ != cudaSuccess)                                                                         \
      throw ::spaqr::Error(e_ == cudaErrorMemoryAllocation ? SPAQR_ERR_OOM : SPAQR_ERR_CUDA,       \
                           std::string(#x) + ": " + cudaGetErrorString(e_) + " at " + __FILE__ + ":" + \
                               std::to_string(__LINE__));                                          \
  } while (0)

// Size-class sub-allocator over large cudaMalloc chunks.  All work of one
// handle runs on one stream, so a block released on the host after its last
// use was enqueued may be handed out again at once (stream order protects it).
class DevicePool {
 public:
  explicit DevicePool(size_t chunk_bytes = size_t(256) << 20) : chunk_(chunk_bytes) {}
  ~DevicePool();
  DevicePool(const DevicePool&) = delete;
  DevicePool& operator=(const DevicePool&) = delete;
  void* alloc(size_t bytes);
  void release(void* p);
  // true when [p, p + bytes) lies inside one live block (host-side bounds check)
  bool contains(const void* p, size_t bytes) const;
  size_t in_use() const { return in_use_; }
  size_t peak() const { return peak_; }
  size_t reserved() const { return reserved_; }

 private:
  struct Chunk {
    char* base;
    size_t size, used;
  };
  size_t chunk_;
  std::vector<Chunk> chunks_;
  std::vector<std::vector<void*>> free_;  // by size class
  std::unordered_map<const void*, int> live_;  // live block -> size class
  size_t in_use_ = 0, peak_ = 0, reserved_ = 0;
};

// Bump allocator for the W store: blocks are carved from large cudaMalloc
// chunks and released only when the arena is destroyed.
class Arena {
 public:
  explicit Arena(size_t chunk_bytes = size_t(64) << 20) : chunk_(chunk_bytes) {}
  ~Arena();
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  void* alloc(size_t bytes);
  bool contains(const void* p, size_t bytes) const;
  size_t used() const { return used_; }

 private:
  struct Chunk {
    char* base;
    size_t size, used;
  };
  size_t chunk_;
  std::vector<Chunk> chunks_;
  size_t used_ = 0;
};

// Pinned staging + device arena for small descriptor arrays.  put() copies a
// host array into pinned memory and enqueues the H2D copy; the device pointer
// stays valid until reset(), which the owner calls right after a stream
// synchronisation.  When a block fills up a larger one is started; retired
// blocks are released at the next reset(), so no pointer handed out since the
// last reset is ever reused early.
class Uploader {
 public:
  Uploader() = default;
  ~Uploader();
  void init(cudaStream_t st, size_t bytes);
  template <typename X>
  X* put(const std::vector<X>& v) {
    return static_cast<X*>(put_bytes(v.data(), v.size() * sizeof(X)));
  }
  void* put_bytes(const void* src, size_t bytes);
  void* scratch(size_t bytes);  // device-only space, same lifetime
  void reset();
  int64_t syncs = 0;

 private:
  struct Block {
    char* host = nullptr;
    char* dev = nullptr;
    size_t cap = 0;
  };
  cudaStream_t st_ = nullptr;
  Block cur_;
  std::vector<Block> retired_;
  size_t off_ = 0;
  void* take(size_t bytes, const void* src);
  static void free_block(Block& b);
};

// Device-time accounting by kernel family with CUDA events on one stream.
// begin()/end() bracket the launches of a family; drain() (after a stream
// synchronisation) adds the elapsed times into the totals.
class EventTimer {
 public:
  ~EventTimer();
  void begin(cudaStream_t st, int family);
  void end(cudaStream_t st);
  void drain(double* totals, int64_t* counts);

 private:
  struct Pair {
    cudaEvent_t a, b;
    int fam;
  };
  std::vector<cudaEvent_t> free_;
  std::vector<Pair> pending_;
  Pair open_{nullptr, nullptr, -1};
  cudaEvent_t get();
};

// One stored factor of W (Section 2.7): kind 0 = R_s = [R_ss R_sn], kind 1 =
// R_pp, kind 2 = Q_pp as k Householder reflectors.
struct WOp {
  int kind = 0, stage = 0, round = 0;
  int c = 0, w = 0;                 // slots of s/p; R_sn columns or reflector capacity
  int k = 0;                        // Q_p: number of reflectors (known after the sync)
  std::vector<int32_t> slots, nslots;
  void* R = nullptr;                // c x (c + w) (kind 0), c x c (kind 1); ld = c
  void* V = nullptr;                // c x w, ld c (kind 2)
  void* tau = nullptr;              // w (kind 2)
  int* kdev = nullptr;              // device rank (kind 2)
  void* G = nullptr;                // dense operator of a large op, formed once for the apply (solve.cu)
};

struct Handle {
  spaqr_options opt{};
  cudaStream_t st = nullptr;       // stream of all library work
  cudaStream_t user_st = nullptr;  // caller's stream (NULL = legacy default stream)
  bool own_stream = false;
  cudaEvent_t ev = nullptr;
  // make st wait for the work the caller enqueued on its stream so far
  void wait_caller();
  int precision = SPAQR_PREC_FP64;
  int64_t m = 0, n = 0, nnz = 0;
  double t_analyze = 0.0;
  // scaled operator A~ = A D (FP64, device) and its transpose, CSR
  int64_t* d_rowptr = nullptr;
  int32_t* d_colidx = nullptr;
  double* d_vals = nullptr;
  int64_t* d_trowptr = nullptr;
  int32_t* d_tcolidx = nullptr;
  double* d_tvals = nullptr;
  int64_t* d_tperm = nullptr;  // transposed position -> row-major position
  double* d_D = nullptr;  // column scaling
  std::vector<int64_t> rowptr;  // host copy of the pattern (for a refactorization)
  std::vector<int32_t> colidx;
  std::vector<int32_t> match;   // the caller's row matching, if any
  std::vector<double> D;
  // W store
  Arena wpool{size_t(64) << 20};
  std::vector<WOp> ops;
  int depth = 0;
  // device-side apply plan (built after the factorization)
  struct ApplyPlan* plan = nullptr;
  spaqr_stats stats{};
  // device int raised by a tensor-core kernel whose MMA completion wait gave up
  int* d_flag = nullptr;
  // solve workspace
  double* d_work = nullptr;
  size_t work_elems = 0;
  ~Handle();
};

// Message returned by spaqr_last_error() on this thread (capi.cpp).
void set_last_error(const std::string& msg);

// Process-wide block cache (memcache.cpp): cudaMalloc / cudaFree and
// cudaMallocHost / cudaFreeHost with freed blocks kept for reuse (a free waits
// for the device, as cudaFree does); release_cached_memory() hands them back.
cudaError_t dmalloc(void** p, size_t bytes);
void dfree(void* p);
cudaError_t hmalloc(void** p, size_t bytes);
void hfree(void* p);
void release_cached_memory();
size_t cached_bytes();
template <typename X>
cudaError_t dmalloc(X** p, size_t bytes) {
  return dmalloc(reinterpret_cast<void**>(p), bytes);
}
template <typename X>
cudaError_t hmalloc(X** p, size_t bytes) {
  return hmalloc(reinterpret_cast<void**>(p), bytes);
}

// Runs the body of a C entry point and maps every host exception to a return
// code, so that none crosses the extern "C" boundary: library errors keep
// their code, a failed host allocation is SPAQR_ERR_OOM, anything else
// SPAQR_ERR_CUDA (INVALID_ARG for std::invalid_argument).
template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return SPAQR_ERR_OOM;
  } catch (const std::invalid_argument& e) {
    set_last_error(e.what());
    return SPAQR_ERR_INVALID_ARG;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return SPAQR_ERR_CUDA;
  }
}

// Factorization entry (factor.cpp): fills h.ops, h.stats, device CSR.
void run_factor(Handle& h, const spaqr_csr& A, const Analysis& an);
// Apply / solve (solve.cu)
void build_apply_plan(Handle& h);
void free_apply_plan(Handle& h);
void apply_Winv(Handle& h, double* z, int transpose);
void apply_A(Handle& h, const double* x, double* y, int forward);
void cgls(Handle& h, const double* b_dev, double* x_dev, spaqr_solve_info* info);
// Corrected seminormal equations with refinement: x <- x + W^{-1} W^{-T} A~^T (b - A~ x).
void csne(Handle& h, const double* b_dev, double* x_dev, spaqr_solve_info* info);
// Adjoint pieces: g_b = A lambda, g_A = r lambda^T - (A lambda) x^T on the pattern.
void lstsq_grad(Handle& h, const double* b, const double* x, const double* lam, double* gb, double* gv);
// New values of A (same pattern, device array in the caller's CSR order).
void set_values(Handle& h, const double* a_dev);

// One iterative solve on one handle: kind 0 = CGLS for min ||A x - b|| (rhs b,
// out x), kind 1 = PCG for (A^T A) lambda = g (rhs g, out lambda), kind 2 =
// corrected seminormal equations for min ||A x - b|| (rhs b, out x), all with
// the factor W.  run_iterative() advances several of them
// side by side, one iteration per handle per round.
struct IterSolve {
  Handle* h = nullptr;
  int kind = 0;
  const double* rhs = nullptr;
  double* out = nullptr;
  double tol = 1e-10;
  int maxit = 500;
  int it = 0;
  bool done = false;
  double norm0 = 0.0, rel = 0.0;
  std::chrono::steady_clock::time_point t0;
  void begin();
  void begun();
  void step();
  void stepped();
  void finish();
  void report(spaqr_solve_info* info);
};
void run_iterative(std::vector<IterSolve>& S);

}  // namespace spaqr
