// Tensor-core (tcgen05, sm_103a) GEMMs of the mixed-precision blocked
// Householder QR: the trailing update C <- C - V T^T V^T C of a panel of b <= 32
// reflectors (Section 2.3 front QR and Section 2.4 scaling, FP32 factor).
//
// Both products run on the 5th-generation tensor cores in 3xTF32: every FP32
// operand x is split into x_hi = tf32(x) and x_lo = x - x_hi, and
// a.b ~= a_hi.b_hi + a_hi.b_lo + a_lo.b_hi is accumulated in FP32 in tensor
// memory (TMEM).  One elected thread issues tcgen05.mma with shared-memory
// descriptors (K-major, no swizzle: 8-row x 16-byte core matrices, LBO = 128 B
// between core matrices along K, SBO between 8-row groups), completion is
// tracked by tcgen05.commit on an mbarrier (bounded wait), and the epilogue
// reads the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31).
//
//   tc_project_kernel:      P_s = C_s^T V_s for a slice s of the rows (split
//                           K), M = 128 trailing columns, N = 32 reflectors;
//   tc_reduce_kernel:       W' = T^T (sum_s P_s)^T, b x ncols;
//   tc_panel_update_kernel: C <- C - V W', M = 128 rows, N = 128 columns,
//                           K = b <= 32 (V unit lower trapezoidal).
// Every launch covers the same panel step of all fronts of a batch (grid z).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace spaqr {
namespace {

constexpr int kTcThreads = 128;  // one warpgroup: the four TMEM lane quarters
constexpr long long kWaitLimit = 1LL << 28;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// K-major, no swizzle: element (r, k) of an R x K operand (4-byte elements)
// sits at (r / 8) * SBO + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4 bytes,
// SBO = K / 4 * 128.  Returns the offset in floats.
__device__ __forceinline__ int kmajor_off(int r, int k, int K) {
  return (r >> 3) * (K * 8) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // tcgen05 descriptor version; base offset 0, no swizzle
  return d;
}

// Instruction descriptor, kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the phase `parity` of the mbarrier; on expiry it raises the
// launch's timeout flag (owned by the caller, read after the launch).
__device__ __forceinline__ void mbar_wait(uint64_t* mbar, uint32_t parity, int* flag) {
  const uint32_t a = smem_u32(mbar);
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return;
  }
  if (flag) atomicExch(flag, 1);
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* out) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(r[j]);
}

// split x into its TF32 head and FP32 remainder at one operand position
__device__ __forceinline__ void put_split(float* hi, float* lo, int off, float x) {
  const float h = tf32_hi(x);
  hi[off] = h;
  lo[off] = x - h;
}

// Issue the 3xTF32 MMAs of one K = 32 stage (4 K-steps of 8): D (+)= A B.
__device__ __forceinline__ void issue_stage(uint32_t tmem, const float* Ahi, const float* Alo, const float* Bhi,
                                            const float* Blo, int Ka, int Kb, uint32_t idesc, bool first) {
  const uint32_t sbo_a = (uint32_t)Ka * 32, sbo_b = (uint32_t)Kb * 32;  // bytes between 8-row groups
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const uint64_t ah = smem_desc(Ahi + s * 64, 128, sbo_a), al = smem_desc(Alo + s * 64, 128, sbo_a);
    const uint64_t bh = smem_desc(Bhi + s * 64, 128, sbo_b), bl = smem_desc(Blo + s * 64, 128, sbo_b);
    mma_tf32(tmem, ah, bh, idesc, (first && s == 0) ? 0u : 1u);
    mma_tf32(tmem, ah, bl, idesc, 1u);
    mma_tf32(tmem, al, bh, idesc, 1u);
  }
}

// C[0:m, 0:n] -= A[0:m, 0:k] B[0:k, 0:n] (column-major) for the 128 x 128 tile
// (row0, col0).  UNIT: A is unit lower trapezoidal (zero above the diagonal,
// one on it, stored below).  K in stages of 32.
template <bool UNIT>
__device__ __forceinline__ void tc_update_tile(int m, int n, int k, const float* A, int lda, const float* B, int ldb,
                                               float* C, int ldc, int row0, int col0, int* flag) {
  extern __shared__ __align__(1024) float tsm[];
  float* Ahi = tsm;           // 128 x 32, K-major
  float* Alo = Ahi + 4096;
  float* Bhi = Alo + 4096;    // 128 (n) x 32 (k), K-major
  float* Blo = Bhi + 4096;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_base, 128);
  if (tid == 0) mbar_init(&mbar, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_tf32(128, 128);
  uint32_t phase = 0;
  for (int k0 = 0; k0 < k; k0 += 32) {
    for (int e = tid; e < 128 * 32; e += kTcThreads) {
      const int mm = e & 127, kk = e >> 7;  // consecutive threads: consecutive rows of A
      const int r = row0 + mm, t = k0 + kk;
      float a = 0.f;
      if (r < m && t < k) {
        if (UNIT)
          a = r < t ? 0.f : (r == t ? 1.f : A[r + (int64_t)t * lda]);
        else
          a = A[r + (int64_t)t * lda];
      }
      put_split(Ahi, Alo, kmajor_off(mm, kk, 32), a);
    }
    for (int e = tid; e < 128 * 32; e += kTcThreads) {
      const int kk = e & 31, nn = e >> 5;  // consecutive threads: consecutive rows of B
      const int t = k0 + kk, cc = col0 + nn;
      const float b = (t < k && cc < n) ? B[t + (int64_t)cc * ldb] : 0.f;
      put_split(Bhi, Blo, kmajor_off(nn, kk, 32), b);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      issue_stage(tmem, Ahi, Alo, Bhi, Blo, 32, 32, idesc, k0 == 0);
      mma_commit(&mbar);
    }
    mbar_wait(&mbar, phase, flag);
    phase ^= 1u;
    fence_after_sync();
  }
  const int mm = warp * 32 + lane;
  const int r = row0 + mm;
  for (int c0 = 0; c0 < 128; c0 += 16) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (r < m && k > 0)
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int cc = col0 + c0 + j;
        if (cc < n) C[r + (int64_t)cc * ldc] -= v[j];
      }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(int m, int n, int k, const float* A, int lda,
                                                                 const float* B, int ldb, float* C, int ldc,
                                                                 int* flag) {
  tc_update_tile<false>(m, n, k, A, lda, B, ldb, C, ldc, blockIdx.x * 128, blockIdx.y * 128, flag);
}

// P[s][c][t] = sum over rows r in slice s of C[r, c] V[r, t]  (V unit lower
// trapezoidal, b <= 32 columns).  Grid (column tiles of 128, slices, fronts);
// M = 128 columns of C, N = 32, K = 32 rows per stage.
__global__ void __launch_bounds__(kTcThreads, 1) tc_project_kernel(const TcPanel* panels) {
  const TcPanel f = panels[blockIdx.z];
  const int col0 = blockIdx.x * 128;
  const int r_begin = blockIdx.y * f.rps, r_end = min(f.mr, r_begin + f.rps);
  if (col0 >= f.ncols || blockIdx.y >= (unsigned)f.nsl) return;  // before any TMEM allocation
  extern __shared__ __align__(1024) float tsm[];
  float* Ahi = tsm;          // 128 (columns of C) x 32 (rows), K-major
  float* Alo = Ahi + 4096;
  float* Bhi = Alo + 4096;   // 32 (reflectors) x 32 (rows), K-major
  float* Blo = Bhi + 1024;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* V = f.X + f.j0 + (int64_t)f.j0 * f.ld;
  const float* C = V + (int64_t)f.b * f.ld;
  if (warp == 0) tmem_alloc(&tmem_base, 32);
  if (tid == 0) mbar_init(&mbar, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_tf32(128, 32);
  uint32_t phase = 0;
  bool first = true;
  for (int k0 = r_begin; k0 < r_end; k0 += 32) {
    for (int e = tid; e < 128 * 32; e += kTcThreads) {
      const int kk = e & 31, mm = e >> 5;  // consecutive threads: consecutive rows of a column of C
      const int r = k0 + kk, cc = col0 + mm;
      const float a = (r < r_end && cc < f.ncols) ? C[r + (int64_t)cc * f.ld] : 0.f;
      put_split(Ahi, Alo, kmajor_off(mm, kk, 32), a);
    }
    for (int e = tid; e < 32 * 32; e += kTcThreads) {
      const int kk = e & 31, nn = e >> 5;
      const int r = k0 + kk;
      float v = 0.f;
      if (r < r_end && nn < f.b) v = r < nn ? 0.f : (r == nn ? 1.f : V[r + (int64_t)nn * f.ld]);
      put_split(Bhi, Blo, kmajor_off(nn, kk, 32), v);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      issue_stage(tmem, Ahi, Alo, Bhi, Blo, 32, 32, idesc, first);
      mma_commit(&mbar);
    }
    mbar_wait(&mbar, phase, f.flag);
    phase ^= 1u;
    fence_after_sync();
    first = false;
  }
  const int mm = warp * 32 + lane;
  const int cc = col0 + mm;
  for (int c0 = 0; c0 < 32; c0 += 16) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (cc < f.ncols) {
      float* out = f.P + ((int64_t)blockIdx.y * f.ncols + cc) * 32 + c0;
#pragma unroll
      for (int j = 0; j < 16; ++j) out[j] = first ? 0.f : v[j];
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

// W'[0:b, c] = T^T (sum_s P[s][c][0:b])  (T upper, ld 32); one thread per column.
__global__ void __launch_bounds__(256) tc_reduce_kernel(const TcPanel* panels) {
  const TcPanel f = panels[blockIdx.y];
  __shared__ float Ts[32 * 32];
  for (int e = threadIdx.x; e < 32 * 32; e += 256) Ts[e] = f.Tm[e];
  __syncthreads();
  const int c = blockIdx.x * 256 + threadIdx.x;
  if (c >= f.ncols) return;
  float w[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) w[t] = 0.f;
  for (int s = 0; s < f.nsl; ++s) {
    const float* p = f.P + ((int64_t)s * f.ncols + c) * 32;
#pragma unroll
    for (int t = 0; t < 32; ++t) w[t] += p[t];
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float acc = 0.f;
#pragma unroll
    for (int l = 0; l < 32; ++l)
      if (l <= i && i < f.b) acc += Ts[l + i * 32] * w[l];
    f.Wp[i + (int64_t)c * 32] = i < f.b ? acc : 0.f;
  }
}

// C <- C - V W' for every panel (grid: row tiles, column tiles, fronts)
__global__ void __launch_bounds__(kTcThreads, 1) tc_panel_update_kernel(const TcPanel* panels);

__global__ void __launch_bounds__(kTcThreads, 1) tc_panel_update_kernel(const TcPanel* panels) {
  const TcPanel f = panels[blockIdx.z];
  const int row0 = blockIdx.x * 128, col0 = blockIdx.y * 128;
  if (row0 >= f.mr || col0 >= f.ncols) return;  // before any TMEM allocation
  const float* V = f.X + f.j0 + (int64_t)f.j0 * f.ld;
  float* C = f.X + f.j0 + (int64_t)(f.j0 + f.b) * f.ld;
  tc_update_tile<true>(f.mr, f.ncols, f.b, V, f.ld, f.Wp, 32, C, f.ld, row0, col0, f.flag);
}

constexpr int kUpdateSmem = 4 * 4096 * (int)sizeof(float);
constexpr int kProjectSmem = (2 * 4096 + 2 * 1024) * (int)sizeof(float);

void tc_setup() {
  static std::once_flag done;  // attributes set once, whichever host thread launches first
  std::call_once(done, [] {
    cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kUpdateSmem);
    cudaFuncSetAttribute(tc_panel_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kUpdateSmem);
    cudaFuncSetAttribute(tc_project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kProjectSmem);
  });
}

}  // namespace

cudaError_t launch_tc_gemm(int m, int n, int k, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                           int* flag, cudaStream_t st) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  tc_setup();
  tc_gemm_kernel<<<dim3((unsigned)((m + 127) / 128), (unsigned)((n + 127) / 128)), kTcThreads, kUpdateSmem, st>>>(
      m, n, k, A, lda, B, ldb, C, ldc, flag);
  return cudaGetLastError();
}

void tc_plan_panel(TcPanel& f) {
  const int tiles = (f.ncols + 127) / 128;
  int s = (304 + tiles - 1) / tiles;                 // about two CTAs per SM
  s = std::max(1, std::min(s, (f.mr + 255) / 256));  // at least 256 rows per slice
  int rps = (f.mr + s - 1) / s;
  rps = (rps + 31) / 32 * 32;
  f.rps = std::max(rps, 32);
  f.nsl = std::max(1, (f.mr + f.rps - 1) / f.rps);
}

size_t tc_panel_scratch(const TcPanel& f) { return (size_t)f.nsl * f.ncols * 32 + (size_t)f.ncols * 32; }

cudaError_t launch_tc_panels(const TcPanel* d_panels, const std::vector<TcPanel>& host, cudaStream_t st) {
  if (host.empty()) return cudaSuccess;
  tc_setup();
  int ct = 0, sl = 0, rt = 0;
  for (const auto& f : host) {
    ct = std::max(ct, (f.ncols + 127) / 128);
    sl = std::max(sl, f.nsl);
    rt = std::max(rt, (f.mr + 127) / 128);
  }
  if (ct == 0) return cudaSuccess;
  const unsigned nf = (unsigned)host.size();
  tc_project_kernel<<<dim3((unsigned)ct, (unsigned)sl, nf), kTcThreads, kProjectSmem, st>>>(d_panels);
  tc_reduce_kernel<<<dim3((unsigned)((ct * 128 + 255) / 256), nf), 256, 0, st>>>(d_panels);
  tc_panel_update_kernel<<<dim3((unsigned)rt, (unsigned)ct, nf), kTcThreads, kUpdateSmem, st>>>(d_panels);
  return cudaGetLastError();
}

}  // namespace spaqr
