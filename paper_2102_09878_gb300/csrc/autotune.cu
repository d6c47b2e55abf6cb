// Autotuner of the column-pivoted QR launch shape (sparsification steps 1
// and 2, Section 2.5).  For every size class (rows m and columns n in powers of
// two) it times, on synthetic full-rank matrices filling the GPU, each
// feasible choice -- a thread-block cluster of 1, 2, 4, 8 or 16 CTAs with the
// column slabs in shared memory, or 16 CTAs over a global work copy with
// delayed updates -- and keeps the fastest.  plan_qrcp() consults the table
// (qrcp_tuned_choice) for every matrix of a batch; classes that were not tuned
// keep the built-in rule (smallest cluster that fits shared memory).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"
#include "kernels.h"

namespace spaqr {
namespace {

std::mutex g_mu;
std::map<std::tuple<int, int, int>, int> g_table;  // (element bytes, m class, n class) -> choice

int cls_of(int x) {
  int c = 0;
  while ((1 << c) < x) ++c;
  return c;
}

template <typename T>
__global__ void fill_kernel(T* a, int64_t n, uint32_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    a[i] = (T)((double)(h & 0xFFFFFF) / 8388608.0 - 1.0);
  }
}

struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      throw Error(SPAQR_ERR_OOM, "autotune: device allocation failed");
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

// milliseconds of one launch of `count` m x n QRCPs with the given choice
template <typename T>
float time_choice(int m, int n, int count, int choice, cudaStream_t st) {
  const int limit = max_smem_optin();
  const bool slab = choice <= 16;
  const int cs = slab ? choice : 16;
  const int nl = (n + cs - 1) / cs;
  Scratch sc;
  T* A = sc.get<T>((size_t)count * m * n);
  T* W = slab ? nullptr : sc.get<T>((size_t)count * m * n);
  T* V = sc.get<T>((size_t)count * m * std::min(m, n));
  T* tau = sc.get<T>((size_t)count * std::min(m, n));
  int* rank = sc.get<int>((size_t)count);
  fill_kernel<T><<<1024, 256, 0, st>>>(A, (int64_t)count * m * n, 12345u + (uint32_t)m * 7u + (uint32_t)n);
  std::vector<QrcpDesc<T>> h((size_t)count);
  for (int i = 0; i < count; ++i) {
    const size_t off = (size_t)i * m * n;
    h[(size_t)i] = QrcpDesc<T>{A + off, slab ? nullptr : W + off, nullptr, V + (size_t)i * m * std::min(m, n),
                               tau + (size_t)i * std::min(m, n), rank + i, m, n, m, m};
  }
  QrcpDesc<T>* d = sc.get<QrcpDesc<T>>((size_t)count);
  SPAQR_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice, st));
  const int nb = slab ? kQrcpNB : qrcp_panel_depth(m, nl, (int)sizeof(T), limit);
  if (slab ? qrcp_smem_bytes(m, nl, (int)sizeof(T), true) > limit : nb == 0) return -1.f;
  cudaEvent_t e0, e1;
  SPAQR_CUDA(cudaEventCreate(&e0));
  SPAQR_CUDA(cudaEventCreate(&e1));
  float best = -1.f;
  for (int rep = 0; rep < 3; ++rep) {
    SPAQR_CUDA(cudaEventRecord(e0, st));
    SPAQR_CUDA(launch_qrcp<T>(d, count, 0.0, cs, nl, m, slab, st, nb));
    SPAQR_CUDA(cudaEventRecord(e1, st));
    SPAQR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SPAQR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && (best < 0.f || ms < best)) best = ms;  // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

template <typename T>
int tune_t(int max_m, int max_n, std::vector<std::string>& log) {
  const int limit = max_smem_optin();
  cudaStream_t st;
  SPAQR_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  int tuned = 0;
  for (int mc = 7; mc <= std::min(cls_of(max_m), 11); ++mc) {
    for (int nc = 6; nc <= std::min(cls_of(max_n), 12); ++nc) {
      const int m = (1 << mc) - (1 << (mc - 2)), n = (1 << nc) - (1 << (nc - 2));  // 3/4 of the class top
      if ((long long)m * n > (4LL << 20)) continue;
      int cmin = 1;
      while (cmin < 16 && qrcp_smem_bytes(m, (n + cmin - 1) / cmin, (int)sizeof(T), true) > limit) cmin *= 2;
      const bool fits = qrcp_smem_bytes(m, (n + cmin - 1) / cmin, (int)sizeof(T), true) <= limit;
      const int lead = fits ? cmin : 16;
      int count = (int)std::max<long long>(1, (304 + lead - 1) / lead);
      count = (int)std::min<long long>(count, std::max<long long>(1, (256LL << 20) / ((long long)m * n)));
      std::vector<int> cand;
      if (fits)
        for (int c = cmin; c <= 16; c *= 2)
          if (n / c >= 32 || c == cmin) cand.push_back(c);
      cand.push_back(32);
      int best = 0;
      float tbest = 0.f;
      std::string line = "m " + std::to_string(m) + " n " + std::to_string(n) + " x" + std::to_string(count) + ":";
      for (int ch : cand) {
        const float t = time_choice<T>(m, n, count, ch, st);
        if (t < 0.f) continue;
        char buf[64];
        std::snprintf(buf, sizeof(buf), " %s%d %.3f ms", ch == 32 ? "global" : "cs", ch == 32 ? 16 : ch, t);
        line += buf;
        if (best == 0 || t < tbest) {
          best = ch;
          tbest = t;
        }
      }
      if (best) {
        std::lock_guard<std::mutex> lock(g_mu);
        g_table[std::make_tuple((int)sizeof(T), mc, nc)] = best;
        ++tuned;
      }
      log.push_back(line);
    }
  }
  cudaStreamDestroy(st);
  return tuned;
}

}  // namespace

int qrcp_tuned_choice(int elem, int m, int n) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_table.empty()) return 0;
  auto it = g_table.find(std::make_tuple(elem, cls_of(std::max(m, 1)), cls_of(std::max(n, 1))));
  return it == g_table.end() ? 0 : it->second;
}

}  // namespace spaqr

extern "C" int spaqr_autotune(int precision, int max_m, int max_n, const char* path, double* seconds) {
  if ((precision != SPAQR_PREC_FP64 && precision != SPAQR_PREC_MIXED) || max_m < 1 || max_n < 1) {
    spaqr::set_last_error("bad arguments");
    return SPAQR_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    spaqr::set_last_error("no CUDA device");
    return SPAQR_ERR_NO_DEVICE;
  }
  try {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<std::string> log;
    if (precision == SPAQR_PREC_MIXED)
      spaqr::tune_t<float>(max_m, max_n, log);
    else
      spaqr::tune_t<double>(max_m, max_n, log);
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (path) {
      FILE* f = std::fopen(path, "w");
      if (!f) {
        spaqr::set_last_error(std::string("cannot write ") + path);
        return SPAQR_ERR_INVALID_ARG;
      }
      std::fprintf(f, "# spaqr QRCP launch-shape table: element-bytes m-class n-class choice (1..16 CTAs in shared "
                      "memory, 32 = 16 CTAs over global memory)\n");
      for (const auto& l : log) std::fprintf(f, "# %s\n", l.c_str());
      std::lock_guard<std::mutex> lock(spaqr::g_mu);
      for (const auto& kv : spaqr::g_table)
        std::fprintf(f, "%d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                     kv.second);
      std::fclose(f);
    }
    return SPAQR_OK;
  } catch (const spaqr::Error& e) {
    spaqr::set_last_error(e.what());
    return e.code;
  }
}

extern "C" int spaqr_load_tuning(const char* path) {
  if (!path) {
    std::lock_guard<std::mutex> lock(spaqr::g_mu);
    spaqr::g_table.clear();
    return SPAQR_OK;
  }
  FILE* f = std::fopen(path, "r");
  if (!f) {
    spaqr::set_last_error(std::string("cannot read ") + path);
    return SPAQR_ERR_INVALID_ARG;
  }
  std::map<std::tuple<int, int, int>, int> t;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    int e, mc, nc, ch;
    if (std::sscanf(line, "%d %d %d %d", &e, &mc, &nc, &ch) == 4) {
      if ((e != 4 && e != 8) || mc < 0 || mc > 30 || nc < 0 || nc > 30 ||
          !(ch == 1 || ch == 2 || ch == 4 || ch == 8 || ch == 16 || ch == 32)) {
        std::fclose(f);
        spaqr::set_last_error("malformed tuning table");
        return SPAQR_ERR_INVALID_ARG;
      }
      t[std::make_tuple(e, mc, nc)] = ch;
    }
  }
  std::fclose(f);
  std::lock_guard<std::mutex> lock(spaqr::g_mu);
  spaqr::g_table.swap(t);
  return SPAQR_OK;
}
