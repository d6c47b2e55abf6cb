// spaqr_dense_qrcp_static: the batched column-pivoted QR of spaqr_dense_qrcp,
// with every piece of device scratch it needs (descriptor array, rank slots,
// work copies of matrices too large for shared memory) taken from one
// file-scope device array instead of cudaMalloc.  For callers that cannot
// allocate device memory themselves (see include/spaqr.h).
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;  // 4 MiB per device, held until exit
__device__ __align__(256) unsigned char g_qrcp_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

int fail(int code, const std::string& m) {
  spaqr::set_last_error(m);
  return code;
}

// Device address of the static array on the current device (set up once per
// device, with that device current).  Host code must never hand the symbol
// itself to a kernel: on the host it names a shadow, not device memory.
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(SPAQR_ERR_NO_DEVICE, "no usable CUDA device");
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_qrcp_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(SPAQR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SPAQR_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int run_static(int count, double* const* A, const int* m, const int* n, const int* ld, double eps,
               double* const* V, double* const* taus, int* rank, void* stream, unsigned char* base);

}  // namespace

extern "C" int spaqr_dense_qrcp_static(int count, double* const* A, const int* m, const int* n, const int* ld,
                                       double eps, double* const* V, double* const* taus, int* rank,
                                       void* stream) {
  if (count < 0 || (count > 0 && (!A || !m || !n || !ld || !rank))) return fail(SPAQR_ERR_INVALID_ARG, "bad arguments");
  if (count == 0) return SPAQR_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return fail(SPAQR_ERR_NO_DEVICE, "no CUDA device");
  }
  unsigned char* base = nullptr;
  if (int rc = scratch_for_current_device(&base)) return rc;
  return spaqr::guarded([&]() -> int { return run_static(count, A, m, n, ld, eps, V, taus, rank, stream, base); });
}

namespace {
int run_static(int count, double* const* A, const int* m, const int* n, const int* ld, double eps,
               double* const* V, double* const* taus, int* rank, void* stream, unsigned char* base) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int lim = spaqr::max_smem_optin();
  std::vector<int> ms, ns;
  for (int i = 0; i < count; ++i) {
    if (m[i] < 0 || n[i] < 0 || ld[i] < (m[i] > 1 ? m[i] : 1)) return fail(SPAQR_ERR_INVALID_ARG, "bad shape");
    ms.push_back(m[i]);
    ns.push_back(n[i]);
  }
  std::vector<spaqr::QrcpGroup> groups;
  std::vector<char> need_work;
  if (!spaqr::plan_qrcp(ms, ns, 8, lim, groups, need_work)) return fail(SPAQR_ERR_CAPACITY, "too many columns");
  // carve the static array: descriptors, rank slots, work copies
  size_t off = 0;
  const size_t desc_off = off;
  off += align256((size_t)count * sizeof(spaqr::QrcpDesc<double>));
  const size_t rank_off = off;
  off += align256((size_t)count * sizeof(int));
  std::vector<size_t> work_off((size_t)count, 0);
  for (int i = 0; i < count; ++i)
    if (need_work[(size_t)i]) {
      work_off[(size_t)i] = off;
      off += align256((size_t)(m[i] > 1 ? m[i] : 1) * (n[i] > 1 ? n[i] : 1) * sizeof(double));
    }
  if (off > kStaticScratchBytes)
    return fail(SPAQR_ERR_CAPACITY, "batch needs " + std::to_string(off) + " bytes of scratch; the static array holds " +
                                        std::to_string(kStaticScratchBytes));
  int* d_rank = reinterpret_cast<int*>(base + rank_off);
  std::vector<spaqr::QrcpDesc<double>> ordered;
  for (auto& g : groups)
    for (int i : g.idx) {
      spaqr::QrcpDesc<double> q{A[i], need_work[(size_t)i] ? reinterpret_cast<double*>(base + work_off[(size_t)i]) : nullptr,
                                A[i], V ? V[i] : nullptr, taus ? taus[i] : nullptr, d_rank + i, m[i], n[i], ld[i], ld[i]};
      ordered.push_back(q);
    }
  auto* d_desc = reinterpret_cast<spaqr::QrcpDesc<double>*>(base + desc_off);
  cudaError_t e = cudaMemcpyAsync(d_desc, ordered.data(), ordered.size() * sizeof(ordered[0]),
                                  cudaMemcpyHostToDevice, st);
  size_t pos = 0;
  for (auto& g : groups) {
    if (e != cudaSuccess) break;
    e = spaqr::launch_qrcp<double>(d_desc + pos, (int)g.idx.size(), eps, g.cs, g.nl_max, g.m_max, g.slab, st, g.nb);
    pos += g.idx.size();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(rank, d_rank, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(SPAQR_ERR_CUDA, cudaGetErrorString(e));
  return SPAQR_OK;
}
}  // namespace
