// Host driver of the spaQR factorization (Algorithm 1, Section 2.7) on one GPU.
//
// The evolving matrix is a set of row groups: rows that share an owner cluster
// and a column support; a group keeps one dense column-major block over its
// support clusters (in ascending cluster id).  The host plans every phase from
// the symbolic structure, the device does every floating-point step:
//
//   stage k = L..1:
//     eliminate   rounds of independent level-k separators; per round one
//                 batched front QR (Section 2.3), the max-norm destinations of
//                 the extra rows (Section 2.2 rule), one device->host wait
//     scale       batched QR of every remaining A_pp, X <- X R_pp^{-1} on every
//                 block column (Section 2.4)
//     step 1      batched column-pivoted QR of every p2 block (Section 2.5.1)
//     step 2      colour by colour: M_p = [A_np^T A_p1n], column-pivoted QR,
//                 reflectors applied to block column p and block row p1
//                 (Section 2.5.2); one wait for the ranks
//     merge       relayout of the groups onto the merged clusters (Section 2.6)
//
// Readings of the paper (identical to the ones the CPU oracle implements):
//   column scaling to unit norms, rows of the caller's matching to their
//   column's cluster, the max-norm row rule on A D for every other row with
//   ties to the deeper then lower-id cluster; front rows = own groups (by creation
//   number) then the other owners' groups touching s (by owner, number);
//   rows at positions >= r_s return to their owners, positions c_s..r_s-1 are
//   reassigned; same-level separators run in rounds of a greedy maximal set of
//   separators with disjoint fronts; step 2 by a greedy colouring of
//   "q in support(p1 of p)"; scaling and sparsification at stages k <= L - skip.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>

#include "internal.h"
#include "kernels.h"
#include "parallel.h"

namespace spaqr {

// ------------------------------------------------------------- DevicePool
DevicePool::~DevicePool() {
  for (auto& c : chunks_) dfree(c.base);
}

void* DevicePool::alloc(size_t bytes) {
  if (bytes == 0) bytes = 1;
  int cls = 0;
  while ((size_t(256) << cls) < bytes) ++cls;
  const size_t sz = size_t(256) << cls;
  if ((int)free_.size() <= cls) free_.resize((size_t)cls + 1);
  void* p = nullptr;
  if (!free_[(size_t)cls].empty()) {
    p = free_[(size_t)cls].back();
    free_[(size_t)cls].pop_back();
  } else {
    Chunk* ch = chunks_.empty() ? nullptr : &chunks_.back();
    if (!ch || ch->used + sz > ch->size) {
      // keep the tail of the old chunk usable by smaller classes
      if (ch) {
        while (ch->size - ch->used >= 256) {
          int c2 = 0;
          while ((size_t(256) << (c2 + 1)) <= ch->size - ch->used) ++c2;
          const size_t s2 = size_t(256) << c2;
          if ((int)free_.size() <= c2) free_.resize((size_t)c2 + 1);
          void* q = ch->base + ch->used;
          free_[(size_t)c2].push_back(q);
          ch->used += s2;
        }
      }
      const size_t csz = std::max(chunk_, sz);
      char* base = nullptr;
      SPAQR_CUDA(dmalloc(&base, csz));
      chunks_.push_back(Chunk{base, csz, 0});
      reserved_ += csz;
      ch = &chunks_.back();
    }
    p = ch->base + ch->used;
    ch->used += sz;
  }
  live_[p] = cls;
  in_use_ += sz;
  peak_ = std::max(peak_, in_use_);
  return p;
}

bool DevicePool::contains(const void* p, size_t bytes) const {
  // a block starts at a multiple of 256 bytes inside a chunk: walk down to it
  const char* q = static_cast<const char*>(p);
  for (const auto& c : chunks_) {
    if (q < c.base || q >= c.base + c.size) continue;
    size_t off = (size_t)(q - c.base) & ~size_t(255);
    while (true) {
      auto it = live_.find(c.base + off);
      if (it != live_.end()) {
        const size_t sz = size_t(256) << it->second;
        return q + bytes <= c.base + off + sz;
      }
      if (off == 0) return false;
      off -= 256;
    }
  }
  return false;
}

void DevicePool::release(void* p) {
  if (!p) return;
  auto it = live_.find(p);
  if (it == live_.end()) return;
  const int cls = it->second;
  live_.erase(it);
  free_[(size_t)cls].push_back(p);
  in_use_ -= size_t(256) << cls;
}

// ------------------------------------------------------------------ Arena
Arena::~Arena() {
  for (auto& c : chunks_) dfree(c.base);
}

void* Arena::alloc(size_t bytes) {
  const size_t need = (std::max<size_t>(bytes, 1) + 255) & ~size_t(255);
  if (chunks_.empty() || chunks_.back().used + need > chunks_.back().size) {
    const size_t csz = std::max(chunk_, need);
    char* base = nullptr;
    SPAQR_CUDA(dmalloc(&base, csz));
    chunks_.push_back(Chunk{base, csz, 0});
  }
  Chunk& c = chunks_.back();
  void* p = c.base + c.used;
  c.used += need;
  used_ += need;
  return p;
}

bool Arena::contains(const void* p, size_t bytes) const {
  const char* q = static_cast<const char*>(p);
  for (const auto& c : chunks_)
    if (q >= c.base && q + bytes <= c.base + c.used) return true;
  return false;
}

// --------------------------------------------------------------- Uploader
void Uploader::free_block(Block& b) {
  if (b.host) hfree(b.host);
  if (b.dev) dfree(b.dev);
  b = Block();
}

Uploader::~Uploader() {
  for (auto& b : retired_) free_block(b);
  free_block(cur_);
}

void Uploader::init(cudaStream_t st, size_t bytes) {
  st_ = st;
  if (cur_.cap < bytes) {
    free_block(cur_);
    cur_.cap = bytes;
    SPAQR_CUDA(hmalloc(&cur_.host, cur_.cap));
    SPAQR_CUDA(dmalloc(&cur_.dev, cur_.cap));
  }
  off_ = 0;
}

void Uploader::reset() {
  // called after a stream synchronisation: nothing handed out is in use
  for (auto& b : retired_) free_block(b);
  retired_.clear();
  off_ = 0;
}

void* Uploader::take(size_t bytes, const void* src) {
  const size_t need = (bytes + 255) & ~size_t(255);
  if (off_ + need > cur_.cap) {
    retired_.push_back(cur_);
    cur_ = Block();
    cur_.cap = std::max(need, 2 * retired_.back().cap);
    SPAQR_CUDA(hmalloc(&cur_.host, cur_.cap));
    SPAQR_CUDA(dmalloc(&cur_.dev, cur_.cap));
    off_ = 0;
  }
  char* d = cur_.dev + off_;
  if (src && bytes) {
    char* h = cur_.host + off_;
    std::memcpy(h, src, bytes);
    SPAQR_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st_));
  }
  off_ += need;
  return d;
}

void* Uploader::put_bytes(const void* src, size_t bytes) { return take(bytes, src); }
void* Uploader::scratch(size_t bytes) { return take(bytes, nullptr); }

// ------------------------------------------------------------- EventTimer
EventTimer::~EventTimer() {
  for (auto e : free_) cudaEventDestroy(e);
  for (auto& p : pending_) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
}

cudaEvent_t EventTimer::get() {
  if (!free_.empty()) {
    cudaEvent_t e = free_.back();
    free_.pop_back();
    return e;
  }
  cudaEvent_t e;
  SPAQR_CUDA(cudaEventCreate(&e));
  return e;
}

void EventTimer::begin(cudaStream_t st, int family) {
  open_.a = get();
  open_.fam = family;
  SPAQR_CUDA(cudaEventRecord(open_.a, st));
}

void EventTimer::end(cudaStream_t st) {
  open_.b = get();
  SPAQR_CUDA(cudaEventRecord(open_.b, st));
  pending_.push_back(open_);
  open_ = Pair{nullptr, nullptr, -1};
}

void EventTimer::drain(double* totals, int64_t* counts) {
  for (auto& p : pending_) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      totals[p.fam] += ms * 1e-3;
      counts[p.fam] += 1;
    } else {
      cudaGetLastError();
    }
    free_.push_back(p.a);
    free_.push_back(p.b);
  }
  pending_.clear();
}

namespace {

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// A short int list stored inline up to kInline entries (most row-group
// supports), on the heap beyond: groups are created and dropped by the hundred
// thousand per stage, in parallel, and this keeps the allocator out of it.
class SmallInts {
 public:
  static constexpr int kInline = 8;
  SmallInts() = default;
  SmallInts(const SmallInts& o) { assign(o.begin(), o.end()); }
  SmallInts(SmallInts&& o) noexcept { take(o); }
  SmallInts& operator=(const SmallInts& o) {
    if (this != &o) assign(o.begin(), o.end());
    return *this;
  }
  SmallInts& operator=(SmallInts&& o) noexcept {
    if (this != &o) {
      clear_free();
      take(o);
    }
    return *this;
  }
  ~SmallInts() { clear_free(); }
  void assign(const int* b, const int* e) {
    const size_t n = (size_t)(e - b);
    reserve_exact(n);
    std::copy(b, e, data());
    n_ = (int)n;
  }
  void resize(size_t n) {
    if (n > (size_t)cap()) {
      SmallInts t;
      t.reserve_exact(n);
      std::copy(begin(), end(), t.data());
      t.n_ = n_;
      *this = std::move(t);
    }
    n_ = (int)n;
  }
  void clear_free() {
    if (heap_) delete[] heap_;
    heap_ = nullptr;
    hcap_ = 0;
    n_ = 0;
  }
  void swap(SmallInts& o) noexcept {
    SmallInts t(std::move(o));
    o = std::move(*this);
    *this = std::move(t);
  }
  size_t size() const { return (size_t)n_; }
  bool empty() const { return n_ == 0; }
  int* data() { return heap_ ? heap_ : in_; }
  const int* data() const { return heap_ ? heap_ : in_; }
  int* begin() { return data(); }
  int* end() { return data() + n_; }
  const int* begin() const { return data(); }
  const int* end() const { return data() + n_; }
  int& operator[](size_t i) { return data()[i]; }
  int operator[](size_t i) const { return data()[i]; }

 private:
  int cap() const { return heap_ ? hcap_ : kInline; }
  // room for n entries; the contents are not kept
  void reserve_exact(size_t n) {
    if (n <= (size_t)cap()) return;
    clear_free();
    if (n > (size_t)kInline) {
      heap_ = new int[n];
      hcap_ = (int)n;
    }
  }
  void take(SmallInts& o) {
    n_ = o.n_;
    if (o.heap_) {
      heap_ = o.heap_;
      hcap_ = o.hcap_;
      o.heap_ = nullptr;
      o.hcap_ = 0;
    } else {
      std::copy(o.in_, o.in_ + o.n_, in_);
    }
    o.n_ = 0;
  }
  int* heap_ = nullptr;
  int hcap_ = 0, n_ = 0;
  int in_[kInline];
};

// Group ids per cluster in CSR form (ascending ids per cluster): index_groups()
// builds one for the groups each cluster owns and one for the groups of other
// owners that touch it.
struct IdRange {
  const int* b;
  const int* e;
  const int* begin() const { return b; }
  const int* end() const { return e; }
  size_t size() const { return (size_t)(e - b); }
  operator std::vector<int>() const { return std::vector<int>(b, e); }
};
struct GroupIndex {
  std::vector<int64_t> ptr;
  std::vector<int> ids;
  IdRange operator[](size_t c) const { return IdRange{ids.data() + ptr[c], ids.data() + ptr[c + 1]}; }
};

template <typename T>
class Factorizer {
 public:
  Factorizer(Handle& h, const Analysis& an) : h_(h), an_(an), st_(h.st) {}
  ~Factorizer() {
    for (auto& x : aux_)
      if (x.st) {
        cudaStreamDestroy(x.st);
        cudaEventDestroy(x.done);
      }
    if (fork_) cudaEventDestroy(fork_);
  }
  void run(const spaqr_csr& A);

 private:
  struct Group {
    int owner = -1;
    int rows = 0, ld = 0, width = 0;
    SmallInts sup, off;  // support clusters (ascending) and their first column in the block
    T* ptr = nullptr;
    int buf = -1;
    bool alive = false;
  };
  struct Buf {
    void* p;
    int refs;
  };

  Handle& h_;
  const Analysis& an_;
  cudaStream_t st_;
  // side streams for independent launches of one phase (forked from and joined back into st_)
  struct Aux {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
  };
  Aux aux_[3];
  cudaEvent_t fork_ = nullptr;
  DevicePool pool_;
  Uploader up_;
  EventTimer tm_;
  int L_ = 0, k_ = 0;
  const StageClusters* sc_ = nullptr;
  std::vector<int> ccols_;
  std::vector<std::vector<int32_t>> slots_;
  std::vector<char> calive_;
  std::vector<Group> G_;
  std::vector<int> live_;  // ids of live groups (dead ones dropped lazily)
  std::vector<Buf> bufs_;
  std::vector<int> p1_of_, p2_of_;
  std::vector<int> own_head_;  // scratch
  int smem_max_ = 0;
  int grid_ctas_ = 0;  // CTAs of one grid-mode QRCP launch (all resident)
  int64_t launches_ = 0;
  struct StageLog {
    int fronts = 0, rounds = 0, max_m = 0, max_n = 0, max_c = 0;
    int scaled = 0, max_rp = 0, s1 = 0, s1_max_m = 0, s1_max_n = 0, s2 = 0, colours = 0, s2_max_c = 0, s2_max_w = 0;
    int64_t sum_c = 0, sum_k = 0;
    double front_flops = 0;
  } slog_;

  // ----------------------------------------------------------- helpers
  int level(int c) const { return sc_->level[(size_t)c]; }
  void check(cudaError_t e, const char* what) {
    ++launches_;
    if (e != cudaSuccess) throw Error(SPAQR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
  // host-side section timers (verbose output): 0 waits in sync, 1 index_groups,
  // 2 eliminate planning, 3 eliminate new groups, 4 scale planning, 5 step2 planning, 6 merge planning
  double ht_[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  struct HT {
    double& acc;
    double t0;
    explicit HT(double& a) : acc(a), t0(now_s()) {}
    ~HT() { acc += now_s() - t0; }
    static double now_s() {
      return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
    }
  };
  // named host timers (printed in verbose mode, largest first)
  std::vector<std::pair<std::string, double>> nt_;
  const char* phase_ = "start";
  void nt_add(const std::string& n, double dt) {
    for (auto& e : nt_)
      if (e.first == n) {
        e.second += dt;
        return;
      }
    nt_.emplace_back(n, dt);
  }
  // successive sections of one function: lap("x") charges the time since the previous lap to "x"
  struct Lap {
    Factorizer* f;
    double t;
    explicit Lap(Factorizer* ff) : f(ff), t(HT::now_s()) {}
    void operator()(const char* name) {
      const double now = HT::now_s();
      f->nt_add(name, now - t);
      t = now;
    }
  };
  struct NT {
    Factorizer* f;
    const char* name;
    double t0;
    NT(Factorizer* ff, const char* n) : f(ff), name(n), t0(HT::now_s()) {}
    ~NT() { f->nt_add(name, HT::now_s() - t0); }
  };
  // reset = false keeps the upload arena (and every scratch pointer taken from
  // it) alive until the caller's own up_.reset()
  void sync(bool reset = true) {
    HT w(ht_[0]);
    const double t0 = HT::now_s();
    SPAQR_CUDA(cudaStreamSynchronize(st_));
    nt_add(std::string("wait in ") + phase_, HT::now_s() - t0);
    ++up_.syncs;
    if (reset) up_.reset();
    tm_.drain(h_.stats.t_kernel, h_.stats.n_kernel);
  }
  // wait for the stream, copy n elements of dev (upload-arena scratch) to host,
  // then recycle the arena: the arena may have grown since dev was taken, and a
  // reset releases the retired blocks
  template <typename X>
  void sync_read(X* host, const X* dev, size_t n) {
    sync(false);
    if (n) SPAQR_CUDA(cudaMemcpy(host, dev, n * sizeof(X), cudaMemcpyDeviceToHost));
    up_.reset();
  }
  void make_group(Group& g, int owner, int rows, const int* sb, const int* se) const {
    g.owner = owner;
    g.rows = rows;
    g.ld = std::max(rows, 1);
    g.sup.assign(sb, se);
    g.off.resize(g.sup.size());
    int w = 0;
    for (size_t t = 0; t < g.sup.size(); ++t) {
      g.off[t] = w;
      w += ccols_[(size_t)g.sup[t]];
    }
    g.width = w;
    g.alive = true;
  }
  // n new (empty) groups with consecutive ids, appended to the live list; returns the first id
  int add_groups(size_t n) {
    const int base = (int)G_.size();
    G_.resize(G_.size() + n);
    for (size_t i = 0; i < n; ++i) live_.push_back(base + (int)i);
    return base;
  }
  // live group ids in ascending order (compacts the list)
  const std::vector<int>& live() {
    size_t w = 0;
    for (size_t i = 0; i < live_.size(); ++i)
      if (G_[(size_t)live_[i]].alive) live_[w++] = live_[i];
    live_.resize(w);
    return live_;
  }
  // one buffer for a list of new groups (zero-initialised when zero = true)
  void assign_buffer(const std::vector<int>& ids, bool zero) {
    size_t total = 0;
    for (int id : ids) total += (size_t)G_[(size_t)id].ld * G_[(size_t)id].width;
    if (total == 0) {
      for (int id : ids) G_[(size_t)id].ptr = nullptr;
      return;
    }
    T* base = static_cast<T*>(pool_.alloc(total * sizeof(T)));
    if (zero) SPAQR_CUDA(cudaMemsetAsync(base, 0, total * sizeof(T), st_));
    bufs_.push_back(Buf{base, 0});
    const int b = (int)bufs_.size() - 1;
    size_t o = 0;
    for (int id : ids) {
      Group& g = G_[(size_t)id];
      const size_t sz = (size_t)g.ld * g.width;
      g.ptr = sz ? base + o : nullptr;
      g.buf = sz ? b : -1;
      if (sz) bufs_[(size_t)b].refs++;
      o += sz;
    }
    if (bufs_[(size_t)b].refs == 0) {
      pool_.release(base);
      bufs_[(size_t)b].p = nullptr;
    }
  }
  void drop_data(Group& g) {
    if (g.buf >= 0) {
      Buf& b = bufs_[(size_t)g.buf];
      if (--b.refs == 0) {
        pool_.release(b.p);
        b.p = nullptr;
      }
    }
    g.buf = -1;
    g.ptr = nullptr;
  }
  // kill a list of groups in parallel: buffer references drop atomically, the
  // buffers that lose their last reference go back to the pool afterwards (in
  // ascending buffer number)
  void kill_many(const std::vector<int>& ids) {
    std::vector<std::vector<int>> freed((size_t)ThreadPool::get().workers());
    parallel_for((int64_t)ids.size(), [&](int64_t b, int64_t e, int w) {
      // groups of one buffer tend to be neighbours: one atomic per run of equal buffers
      int run_buf = -1, run = 0;
      auto flush = [&]() {
        if (run_buf >= 0 && __atomic_sub_fetch(&bufs_[(size_t)run_buf].refs, run, __ATOMIC_ACQ_REL) == 0)
          freed[(size_t)w].push_back(run_buf);
        run_buf = -1;
        run = 0;
      };
      for (int64_t i = b; i < e; ++i) {
        Group& g = G_[(size_t)ids[(size_t)i]];
        if (g.buf >= 0) {
          if (g.buf != run_buf) {
            flush();
            run_buf = g.buf;
          }
          ++run;
        }
        g.buf = -1;
        g.ptr = nullptr;
        g.alive = false;
        g.sup.clear_free();
        g.off.clear_free();
      }
      flush();
    }, 4096);
    std::vector<int> all;
    for (auto& v : freed) all.insert(all.end(), v.begin(), v.end());
    std::sort(all.begin(), all.end());
    for (int b : all) {
      pool_.release(bufs_[(size_t)b].p);
      bufs_[(size_t)b].p = nullptr;
    }
  }
  void kill(int id) {
    Group& g = G_[(size_t)id];
    drop_data(g);
    g.alive = false;
    g.sup.clear_free();
    g.off.clear_free();
  }
  int col_off(const Group& g, int c) const {
    auto it = std::lower_bound(g.sup.begin(), g.sup.end(), c);
    if (it == g.sup.end() || *it != c) return -1;
    return g.off[(size_t)(it - g.sup.begin())];
  }
  T* wstore(size_t elems) { return static_cast<T*>(h_.wpool.alloc(std::max<size_t>(elems, 1) * sizeof(T))); }
  // (descriptor, first unit) work items covering `units(i)` units per descriptor in steps of `per`
  template <typename F>
  std::vector<int2> items_for(size_t count, int per, F units) const {
    std::vector<int2> it;
    for (size_t i = 0; i < count; ++i)
      for (int u = 0; u < units(i); u += per) it.push_back(make_int2((int)i, u));
    return it;
  }

  // ---- optional host-side bounds checks of every descriptor (SPAQR_CHECK=1)
  bool checking_ = false;
  void in_bounds(const void* p, int64_t rows, int64_t cols, int64_t ld, int64_t esz, const char* what) const {
    if (rows <= 0 || cols <= 0) return;
    if (!p) throw Error(SPAQR_ERR_CAPACITY, std::string("check: null pointer in ") + what);
    if (ld < rows) throw Error(SPAQR_ERR_CAPACITY, std::string("check: ld < rows in ") + what);
    const size_t bytes = (size_t)((rows - 1) + (cols - 1) * ld + 1) * (size_t)esz;
    if (!pool_.contains(p, bytes) && !h_.wpool.contains(p, bytes))
      throw Error(SPAQR_ERR_CAPACITY, std::string("check: out-of-bounds ") + what + " rows " + std::to_string(rows) +
                                          " cols " + std::to_string(cols) + " ld " + std::to_string(ld) + " at stage " +
                                          std::to_string(k_));
  }
  void check_copies(const std::vector<CopyDesc<T>>& v, const std::vector<std::vector<int>>* rowsets = nullptr) const {
    (void)rowsets;
    for (auto& d : v) {
      if (d.src) in_bounds(d.src, d.rowidx ? 1 : d.rows, d.cols, d.rowidx ? std::max(d.sld, 1) : d.sld, sizeof(T), "copy src");
      if (d.transpose)
        in_bounds(d.dst, d.cols, d.rows, d.dld, sizeof(T), "copy dst (transposed)");
      else
        in_bounds(d.dst, d.rows, d.cols, d.dld, sizeof(T), "copy dst");
    }
  }

  // batched front QR of fronts (ptr,m,n,c,ld) in device memory
  void front_qr(std::vector<FrontDesc<T>>& fr);
  // batched QRCP
  void qrcp(std::vector<QrcpDesc<T>>& qs, std::vector<T*>& work_bufs);
  void copies(const std::vector<CopyDesc<T>>& cps);

  void init_stage(const spaqr_csr& A);
  void eliminate();
  void eliminate_round(const std::vector<std::pair<int, std::vector<int>>>& batch, int round);
  void scale();
  void step1();
  void step2();
  void merge();
  bool sparsify_here() const {
    return h_.opt.mode == SPAQR_MODE_SPAQR && k_ <= L_ - h_.opt.skip && k_ >= 2;
  }
  void index_groups(GroupIndex& own, GroupIndex& touch);
  // step 2's structure (colours, and per interface the groups touching it and
  // its neighbour clusters) depends only on the groups, not on the step-1
  // ranks: it is prepared while step 1 runs on the device
  struct S2Member {
    std::vector<int> nb, ncols;  // touching groups (by owner, id), neighbour clusters of p1
    int cn = 0;                  // columns of the neighbour clusters
  };
  struct S2Plan {
    bool ready = false;
    std::vector<int> ps;
    int ncol = 0;
    std::vector<std::vector<int>> members;      // by colour
    std::vector<std::vector<S2Member>> pre;     // parallel to members
  } s2_;
  void prepare_step2();
};

template <typename T>
void Factorizer<T>::copies(const std::vector<CopyDesc<T>>& cps) {
  NT nt_f(this, "copies (plan+launch)");
  if (cps.empty()) return;
  std::vector<int> start(cps.size() + 1, 0);
  int64_t tot = 0;
  for (size_t i = 0; i < cps.size(); ++i) {
    start[i] = (int)tot;
    tot += copy_ctas(cps[i].rows, cps[i].cols, cps[i].transpose);
    if (tot > INT32_MAX / 2) throw Error(SPAQR_ERR_CAPACITY, "block copies larger than one launch covers");
  }
  start[cps.size()] = (int)tot;
  if (checking_) check_copies(cps);
  auto* d = up_.put(cps);
  int* ds = up_.put(start);
  tm_.begin(st_, 0);
  check(launch_copy<T>(d, ds, (int)cps.size(), (int)tot, st_), "copy");
  tm_.end(st_);
}

template <typename T>
void Factorizer<T>::front_qr(std::vector<FrontDesc<T>>& fr) {
  NT nt_f(this, "front_qr (plan+launch)");
  if (fr.empty()) return;
  std::vector<int> ms, ns, cs;
  for (auto& f : fr) {
    if (checking_ && f.c > 0) in_bounds(f.ptr, f.m, f.n, f.ld, sizeof(T), "front");
    ms.push_back(f.m);
    ns.push_back(f.n);
    cs.push_back(f.c);
  }
  const auto groups = plan_fronts(ms, ns, cs, (int)sizeof(T), smem_max_);
  if (groups.empty()) return;
  std::vector<std::vector<FrontDesc<T>>> host(groups.size());
  std::vector<const FrontDesc<T>*> dev(groups.size());
  T* Tbuf = nullptr;
  for (size_t g = 0; g < groups.size(); ++g) {
    for (int i : groups[g].idx) host[g].push_back(fr[(size_t)i]);
    dev[g] = up_.put(host[g]);
    if (groups[g].kind == 2) {  // per front: a 32 x 32 T factor, later the sign mask of diag(R)
      int maxc = 0;
      for (auto& f : host[g]) maxc = std::max(maxc, f.c);
      const size_t per = std::max<size_t>(32 * 32 * sizeof(T), (size_t)((maxc + 31) / 32) * sizeof(unsigned));
      Tbuf = static_cast<T*>(up_.scratch(host[g].size() * per));
    }
  }
  // FP32 factor: blocked fronts take the tensor-core trailing updates
  const size_t tc_bytes = front_groups_tc_bytes<T>(groups, host);
  void* tc_scratch = tc_bytes ? up_.scratch(tc_bytes) : nullptr;
  tm_.begin(st_, 1);
  check(launch_front_groups<T>(groups, dev, host, Tbuf, st_, &launches_, tc_scratch, h_.d_flag), "front_qr");
  tm_.end(st_);
}

template <typename T>
void Factorizer<T>::qrcp(std::vector<QrcpDesc<T>>& qs, std::vector<T*>& work_bufs) {
  NT nt_f(this, "qrcp (plan+launch)");
  if (qs.empty()) return;
  std::vector<int> ms, ns;
  for (auto& q : qs) {
    if (checking_) {
      in_bounds(q.src, q.m, q.n, q.ld, sizeof(T), "qrcp src");
      if (q.out) in_bounds(q.out, q.m, q.n, q.ldo, sizeof(T), "qrcp out");
      if (q.V) in_bounds(q.V, q.m, std::min(q.m, q.n), q.m, sizeof(T), "qrcp V");
      if (q.tau) in_bounds(q.tau, 1, std::min(q.m, q.n), 1, sizeof(T), "qrcp tau");
    }
    ms.push_back(q.m);
    ns.push_back(q.n);
  }
  std::vector<QrcpGroup> groups;
  std::vector<char> need_work;
  if (!plan_qrcp(ms, ns, (int)sizeof(T), smem_max_, groups, need_work, grid_ctas_))
    throw Error(SPAQR_ERR_CAPACITY, "column-pivoted QR with too many columns for 16 CTAs");
  for (size_t i = 0; i < qs.size(); ++i)
    if (need_work[i]) {
      T* w = static_cast<T*>(pool_.alloc((size_t)std::max(1, qs[i].m) * std::max(1, qs[i].n) * sizeof(T)));
      work_bufs.push_back(w);
      qs[i].work = w;
    }
  const double eps = h_.opt.mode == SPAQR_MODE_SPAQR ? h_.opt.eps : 0.0;
  std::vector<QrcpDesc<T>*> dg;
  for (auto& g : groups) {
    std::vector<QrcpDesc<T>> part;
    for (int i : g.idx) part.push_back(qs[(size_t)i]);
    dg.push_back(up_.put(part));
  }
  // grid-mode groups: exchange areas (tags zeroed) and CTA ranges
  std::vector<QrcpGridDesc*> dgd(groups.size(), nullptr);
  std::vector<int> gtot(groups.size(), 0);
  for (size_t t = 0; t < groups.size(); ++t) {
    const auto& g = groups[t];
    if (!g.grid) continue;
    size_t bytes = 0;
    for (int c : g.ctas) bytes += qrcp_grid_xchg_bytes(c, g.m_max, (int)sizeof(T));
    unsigned char* x = static_cast<unsigned char*>(pool_.alloc(bytes));
    work_bufs.push_back(reinterpret_cast<T*>(x));
    SPAQR_CUDA(cudaMemsetAsync(x, 0, bytes, st_));
    std::vector<QrcpGridDesc> gd;
    gtot[t] = qrcp_grid_descs(g.ctas, g.m_max, (int)sizeof(T), x, gd);
    dgd[t] = up_.put(gd);
  }
  tm_.begin(st_, 2);
  // the shared-memory and warp groups are independent launches: they run side by side on st_ and
  // the side streams (forked after the uploads above, joined before anything that follows); the
  // cooperative CTA-group launches run alone on st_ afterwards
  std::vector<size_t> plain;
  for (size_t t = 0; t < groups.size(); ++t)
    if (!groups[t].grid) plain.push_back(t);
  const size_t nside = std::min<size_t>(plain.size() > 0 ? plain.size() - 1 : 0, 3);
  if (nside) {
    if (!fork_) SPAQR_CUDA(cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming));
    SPAQR_CUDA(cudaEventRecord(fork_, st_));
    for (size_t a = 0; a < nside; ++a) {
      if (!aux_[a].st) {
        SPAQR_CUDA(cudaStreamCreateWithFlags(&aux_[a].st, cudaStreamNonBlocking));
        SPAQR_CUDA(cudaEventCreateWithFlags(&aux_[a].done, cudaEventDisableTiming));
      }
      SPAQR_CUDA(cudaStreamWaitEvent(aux_[a].st, fork_, 0));
    }
  }
  for (size_t q = 0; q < plain.size(); ++q) {
    const size_t t = plain[q];
    const auto& g = groups[t];
    cudaStream_t s = (q == 0 || nside == 0) ? st_ : aux_[(q - 1) % nside].st;
    check(launch_qrcp<T>(dg[t], (int)g.idx.size(), eps, g.cs, g.nl_max, g.m_max, g.slab, s, g.nb), "qrcp");
  }
  for (size_t a = 0; a < nside; ++a) {
    SPAQR_CUDA(cudaEventRecord(aux_[a].done, aux_[a].st));
    SPAQR_CUDA(cudaStreamWaitEvent(st_, aux_[a].done, 0));
  }
  for (size_t t = 0; t < groups.size(); ++t) {
    const auto& g = groups[t];
    if (g.grid)
      check(launch_qrcp_grid<T>(dg[t], dgd[t], (int)g.idx.size(), gtot[t], eps, g.nl_max, g.m_max, g.slab, st_), "qrcp grid");
  }
  tm_.end(st_);
}

template <typename T>
void Factorizer<T>::index_groups(GroupIndex& own, GroupIndex& touch) {
  HT ht(ht_[1]);
  const size_t nc = ccols_.size();
  const std::vector<int>& lv = live();  // ascending ids
  own.ptr.assign(nc + 1, 0);
  touch.ptr.assign(nc + 1, 0);
  for (int id : lv) {
    const Group& g = G_[(size_t)id];
    own.ptr[(size_t)g.owner + 1]++;
    for (int c : g.sup)
      if (c != g.owner) touch.ptr[(size_t)c + 1]++;
  }
  for (size_t c = 0; c < nc; ++c) {
    own.ptr[c + 1] += own.ptr[c];
    touch.ptr[c + 1] += touch.ptr[c];
  }
  own.ids.resize((size_t)own.ptr[nc]);
  touch.ids.resize((size_t)touch.ptr[nc]);
  std::vector<int64_t> po(own.ptr.begin(), own.ptr.end() - 1), pt(touch.ptr.begin(), touch.ptr.end() - 1);
  for (int id : lv) {
    const Group& g = G_[(size_t)id];
    own.ids[(size_t)po[(size_t)g.owner]++] = id;
    for (int c : g.sup)
      if (c != g.owner) touch.ids[(size_t)pt[(size_t)c]++] = id;
  }
}

// ------------------------------------------------------------ init (a0)
template <typename T>
void Factorizer<T>::init_stage(const spaqr_csr& A) {
  NT nt_f(this, "init_stage");
  phase_ = "init_stage";
  Lap lap(this);
  const StageClusters& st = an_.stages[(size_t)L_];
  sc_ = &st;
  const size_t nc = st.node.size();
  ccols_.assign(nc, 0);
  slots_.assign(nc, {});
  calive_.assign(nc, 1);
  std::vector<int32_t> cl_of((size_t)h_.n, -1), pos_of((size_t)h_.n, 0);
  parallel_for((int64_t)nc, [&](int64_t b0, int64_t b1, int) {
    for (int64_t cc = b0; cc < b1; ++cc) {
      const size_t c = (size_t)cc;
      const int64_t b = st.vptr[c], e = st.vptr[c + 1];
      ccols_[c] = (int)(e - b);
      slots_[c].assign(st.verts.begin() + b, st.verts.begin() + e);
      for (int64_t t = b; t < e; ++t) {  // clusters hold disjoint vertex sets
        cl_of[(size_t)st.verts[(size_t)t]] = (int)c;
        pos_of[(size_t)st.verts[(size_t)t]] = (int)(t - b);
      }
    }
  }, 256);
  lap("init: cluster maps");
  // column scaling D (Section 2.7), computed by the caller
  if ((int64_t)h_.D.size() != h_.n) throw Error(SPAQR_ERR_CUDA, "internal: column scaling missing");
  lap("init: column norms");
  // row owners by the max-norm rule on A D (R2), grouped by (owner, support);
  // rows are independent: two parallel passes (support sizes, then contents)
  const int64_t M = A.m;
  std::vector<int32_t> owner((size_t)M);
  std::vector<int64_t> sptr((size_t)M + 1, 0);
  std::vector<int32_t> sups;
  const bool tree = h_.opt.row_rule == SPAQR_ROWS_TREE;
  auto row_support = [&](int64_t r, std::vector<int>& tmp, std::vector<double>& sc) -> int {
    tmp.clear();
    for (int64_t e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) tmp.push_back(cl_of[(size_t)A.colidx[e]]);
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    if (tmp.empty()) return -1;
    sc.assign(tmp.size(), 0.0);
    for (int64_t e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) {
      const int32_t j = A.colidx[e];
      const double v = A.vals[e] * h_.D[(size_t)j];
      const size_t t = (size_t)(std::lower_bound(tmp.begin(), tmp.end(), cl_of[(size_t)j]) - tmp.begin());
      sc[t] += v * v;
    }
    // candidates: every touched cluster, or (tree rule) those of the deepest level
    int deep = 0;
    for (int c : tmp) deep = std::max(deep, level(c));
    int best = -1;
    for (size_t t = 0; t < tmp.size(); ++t) {
      const int a = tmp[t];
      if (tree && level(a) != deep) continue;
      if (best < 0) {
        best = (int)t;
        continue;
      }
      const int b = tmp[(size_t)best];
      if (sc[t] > sc[(size_t)best] ||
          (sc[t] == sc[(size_t)best] && (level(a) > level(b) || (level(a) == level(b) && a < b))))
        best = (int)t;
    }
    return tmp[(size_t)best];
  };
  // a row matched to column j (the caller's matching) belongs to j's cluster
  std::vector<int32_t> matched;
  if (A.match) {
    matched.assign((size_t)M, -1);
    for (int64_t j = 0; j < h_.n; ++j) matched[(size_t)A.match[j]] = cl_of[(size_t)j];
  }
  std::atomic<int64_t> empty_row{-1};
  parallel_for(M, [&](int64_t b, int64_t e, int) {
    std::vector<int> tmp;
    std::vector<double> sc;
    for (int64_t r = b; r < e; ++r) {
      int o = row_support(r, tmp, sc);
      if (o < 0) {
        empty_row.store(r);
        continue;
      }
      if (!matched.empty() && matched[(size_t)r] >= 0) o = matched[(size_t)r];
      owner[(size_t)r] = o;
      sptr[(size_t)r + 1] = (int64_t)tmp.size();
    }
  });
  lap("init: row owners");
  if (empty_row.load() >= 0) throw Error(SPAQR_ERR_INVALID_ARG, "empty row " + std::to_string(empty_row.load()));
  {  // prefix sums of the support sizes: chunk totals, their prefix, then each chunk
    const int parts = ThreadPool::get().workers();
    std::vector<int64_t> base((size_t)parts + 1, 0);
    parallel_for(parts, [&](int64_t b, int64_t e, int) {
      for (int64_t p = b; p < e; ++p)
        for (int64_t r = M * p / parts; r < M * (p + 1) / parts; ++r) base[(size_t)p + 1] += sptr[(size_t)r + 1];
    }, 1);
    for (int p = 0; p < parts; ++p) base[(size_t)p + 1] += base[(size_t)p];
    parallel_for(parts, [&](int64_t b, int64_t e, int) {
      for (int64_t p = b; p < e; ++p) {
        int64_t acc = base[(size_t)p];
        for (int64_t r = M * p / parts; r < M * (p + 1) / parts; ++r) sptr[(size_t)r + 1] = acc += sptr[(size_t)r + 1];
      }
    }, 1);
  }
  sups.resize((size_t)sptr[(size_t)M]);
  parallel_for(M, [&](int64_t b, int64_t e, int) {
    std::vector<int> tmp;
    for (int64_t r = b; r < e; ++r) {
      tmp.clear();
      for (int64_t q = A.rowptr[r]; q < A.rowptr[r + 1]; ++q) tmp.push_back(cl_of[(size_t)A.colidx[q]]);
      std::sort(tmp.begin(), tmp.end());
      tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
      std::copy(tmp.begin(), tmp.end(), sups.begin() + sptr[(size_t)r]);
    }
  });
  lap("init: row supports");
  // bucket the rows by owner (in parallel; the order inside a bucket does not
  // matter: every bucket is then sorted by (support, row))
  std::vector<int64_t> cnt(nc + 1, 0);
  parallel_for(M, [&](int64_t b, int64_t e, int) {
    for (int64_t r = b; r < e; ++r) __atomic_fetch_add(&cnt[(size_t)owner[(size_t)r] + 1], 1, __ATOMIC_RELAXED);
  });
  for (size_t c = 0; c < nc; ++c) cnt[c + 1] += cnt[c];
  std::vector<int64_t> order((size_t)M);
  {
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    parallel_for(M, [&](int64_t b, int64_t e, int) {
      for (int64_t r = b; r < e; ++r)
        order[(size_t)__atomic_fetch_add(&pos[(size_t)owner[(size_t)r]], 1, __ATOMIC_RELAXED)] = r;
    });
  }
  auto sup_less = [&](int64_t a, int64_t b) {
    const int32_t *pa = &sups[(size_t)sptr[(size_t)a]], *pb = &sups[(size_t)sptr[(size_t)b]];
    const int64_t la = sptr[(size_t)a + 1] - sptr[(size_t)a], lb = sptr[(size_t)b + 1] - sptr[(size_t)b];
    if (std::lexicographical_compare(pa, pa + la, pb, pb + lb)) return true;
    if (std::lexicographical_compare(pb, pb + lb, pa, pa + la)) return false;
    return a < b;
  };
  // a support of at most two clusters packs into one integer key that orders
  // like the lists themselves ([a] < [a, b]); owners whose rows all have such
  // supports sort (key, row) pairs, the others compare the lists
  parallel_for((int64_t)nc, [&](int64_t b, int64_t e, int) {
    std::vector<std::pair<uint64_t, int64_t>> kv;
    for (int64_t c = b; c < e; ++c) {
      const int64_t i0 = cnt[(size_t)c], i1 = cnt[(size_t)c + 1];
      bool packed = true;
      for (int64_t i = i0; i < i1 && packed; ++i) packed = sptr[(size_t)order[(size_t)i] + 1] - sptr[(size_t)order[(size_t)i]] <= 2;
      if (!packed) {
        std::sort(order.begin() + i0, order.begin() + i1, sup_less);
        continue;
      }
      kv.resize((size_t)(i1 - i0));
      for (int64_t i = i0; i < i1; ++i) {
        const int64_t r = order[(size_t)i];
        const int32_t* sp = &sups[(size_t)sptr[(size_t)r]];
        const int64_t len = sptr[(size_t)r + 1] - sptr[(size_t)r];
        const uint64_t key = ((uint64_t)(uint32_t)sp[0] << 32) | (len == 2 ? (uint64_t)(uint32_t)sp[1] + 1 : 0);
        kv[(size_t)(i - i0)] = {key, r};
      }
      std::sort(kv.begin(), kv.end());
      for (int64_t i = i0; i < i1; ++i) order[(size_t)i] = kv[(size_t)(i - i0)].second;
    }
  }, 256);
  lap("init: sort rows");
  // groups: runs of equal (owner, support) in the sorted order, built in parallel
  std::vector<int32_t> grp_of_row((size_t)M), rowpos((size_t)M);
  auto same = [&](int64_t a, int64_t b) {
    if (owner[(size_t)a] != owner[(size_t)b]) return false;
    const int64_t la = sptr[(size_t)a + 1] - sptr[(size_t)a], lb = sptr[(size_t)b + 1] - sptr[(size_t)b];
    return la == lb && std::equal(&sups[(size_t)sptr[(size_t)a]], &sups[(size_t)sptr[(size_t)a]] + la,
                                  &sups[(size_t)sptr[(size_t)b]]);
  };
  std::vector<char> starts_here((size_t)M, 0);
  parallel_for(M, [&](int64_t b, int64_t e, int) {
    for (int64_t t = b; t < e; ++t) starts_here[(size_t)t] = t == 0 || !same(order[(size_t)t], order[(size_t)t - 1]);
  });
  // the group starts, in order: per-chunk counts, then each chunk writes its own
  std::vector<int64_t> starts;
  {
    const int parts = ThreadPool::get().workers();
    std::vector<int64_t> pc((size_t)parts + 1, 0);
    parallel_for(parts, [&](int64_t b, int64_t e, int) {
      for (int64_t p = b; p < e; ++p)
        for (int64_t t = M * p / parts; t < M * (p + 1) / parts; ++t) pc[(size_t)p + 1] += starts_here[(size_t)t];
    }, 1);
    for (int p = 0; p < parts; ++p) pc[(size_t)p + 1] += pc[(size_t)p];
    starts.resize((size_t)pc[(size_t)parts] + 1);
    parallel_for(parts, [&](int64_t b, int64_t e, int) {
      for (int64_t p = b; p < e; ++p) {
        int64_t q = pc[(size_t)p];
        for (int64_t t = M * p / parts; t < M * (p + 1) / parts; ++t)
          if (starts_here[(size_t)t]) starts[(size_t)q++] = t;
      }
    }, 1);
    starts.back() = M;
  }
  const size_t ngroups = starts.size() - 1;
  G_.reserve(3 * ngroups + 1024);  // group ids only grow; avoid moving every group on growth
  const int gbase = add_groups(ngroups);
  std::vector<int> ids(ngroups);
  parallel_for((int64_t)ngroups, [&](int64_t b, int64_t e, int) {
    for (int64_t q = b; q < e; ++q) {
      const int64_t i = starts[(size_t)q], j = starts[(size_t)q + 1];
      const int64_t r0 = order[(size_t)i];
      const int id = gbase + (int)q;
      ids[(size_t)q] = id;
      make_group(G_[(size_t)id], owner[(size_t)r0], (int)(j - i), &sups[(size_t)sptr[(size_t)r0]],
                 &sups[(size_t)sptr[(size_t)r0]] + (sptr[(size_t)r0 + 1] - sptr[(size_t)r0]));
      for (int64_t t = i; t < j; ++t) {
        grp_of_row[(size_t)order[(size_t)t]] = id;
        rowpos[(size_t)order[(size_t)t]] = (int32_t)(t - i);
      }
    }
  }, 1024);
  lap("init: groups");
  assign_buffer(ids, true);
  // scatter the scaled values into the group blocks
  T* base = G_[(size_t)ids.front()].ptr;  // all initial groups share one buffer, in id order
  std::vector<int64_t> dest((size_t)A.nnz);
  std::vector<T> vals((size_t)A.nnz);
  parallel_for(M, [&](int64_t b, int64_t e0, int) {
    for (int64_t r = b; r < e0; ++r) {
      const Group& g = G_[(size_t)grp_of_row[(size_t)r]];
      const int64_t gbase = g.ptr - base;
      for (int64_t e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) {
        const int32_t jcol = A.colidx[e];
        const int co = col_off(g, cl_of[(size_t)jcol]) + pos_of[(size_t)jcol];
        dest[(size_t)e] = gbase + rowpos[(size_t)r] + (int64_t)co * g.ld;
        vals[(size_t)e] = (T)(A.vals[e] * h_.D[(size_t)jcol]);
      }
    }
  });
  lap("init: scatter plan");
  int64_t* d_dest = static_cast<int64_t*>(pool_.alloc(dest.size() * sizeof(int64_t)));
  T* d_vals = static_cast<T*>(pool_.alloc(vals.size() * sizeof(T)));
  SPAQR_CUDA(cudaMemcpyAsync(d_dest, dest.data(), dest.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st_));
  SPAQR_CUDA(cudaMemcpyAsync(d_vals, vals.data(), vals.size() * sizeof(T), cudaMemcpyHostToDevice, st_));
  check(launch_scatter_values<T>(base, d_dest, d_vals, A.nnz, st_), "scatter_values");
  sync();
  lap("init: upload+scatter");
  pool_.release(d_dest);
  pool_.release(d_vals);
}

// ------------------------------------------------------------ eliminate
template <typename T>
void Factorizer<T>::eliminate() {
  NT nt_f(this, "eliminate");
  phase_ = "eliminate";
  std::vector<int> todo;
  for (size_t c = 0; c < ccols_.size(); ++c)
    if (calive_[c] && level((int)c) == k_) todo.push_back((int)c);
  GroupIndex own, touch;
  std::vector<int64_t> stamp(G_.size() + 1, -1);
  int round = 0;
  while (!todo.empty()) {
    index_groups(own, touch);
    if (stamp.size() < G_.size()) stamp.resize(G_.size(), -1);
    std::vector<std::pair<int, std::vector<int>>> batch;
    std::vector<int> rest;
    for (int s : todo) {
      std::vector<int> fg = own[(size_t)s];
      std::vector<int> oth = touch[(size_t)s];
      std::sort(oth.begin(), oth.end(), [&](int a, int b) {
        const int oa = G_[(size_t)a].owner, ob = G_[(size_t)b].owner;
        return oa != ob ? oa < ob : a < b;
      });
      fg.insert(fg.end(), oth.begin(), oth.end());
      bool clash = false;
      for (int g : fg)
        if (stamp[(size_t)g] == round) {
          clash = true;
          break;
        }
      if (clash) {
        rest.push_back(s);
        continue;
      }
      for (int g : fg) stamp[(size_t)g] = round;
      batch.emplace_back(s, std::move(fg));
    }
    eliminate_round(batch, round);
    todo.swap(rest);
    ++round;
    slog_.rounds = round;
  }
}

template <typename T>
void Factorizer<T>::eliminate_round(const std::vector<std::pair<int, std::vector<int>>>& batch, int round) {
  struct FrontInfo {
    int s, m, n, c, rs;
    std::vector<int> cols, coff;  // clusters (s first), column offsets (size cols+1)
    size_t foff;                  // offset in the workspace (elements)
    int nextra;
    size_t dest_off;
  };
  std::vector<FrontInfo> fi(batch.size());
  size_t ws = 0, ndest = 0;
  std::vector<CopyDesc<T>> gat;
  double plan_t0 = HT::now_s();
  Lap lap(this);
  // fronts are independent: their column lists and sizes in parallel, then the
  // workspace and destination offsets in front order
  std::vector<size_t> gfirst(batch.size() + 1, 0);
  parallel_for((int64_t)batch.size(), [&](int64_t b0, int64_t b1, int) {
    std::vector<int> u;
    for (int64_t bb = b0; bb < b1; ++bb) {
      const size_t b = (size_t)bb;
      const int s = batch[b].first;
      const auto& fg = batch[b].second;
      FrontInfo& f = fi[b];
      f.s = s;
      f.c = ccols_[(size_t)s];
      f.rs = 0;
      f.m = 0;
      u.clear();
      size_t ng = 0;
      for (int g : fg) {
        const Group& gg = G_[(size_t)g];
        if (gg.owner == s) f.rs += gg.rows;
        f.m += gg.rows;
        u.insert(u.end(), gg.sup.begin(), gg.sup.end());
        if (gg.rows)
          for (int c : gg.sup) ng += ccols_[(size_t)c] ? 1 : 0;
      }
      std::sort(u.begin(), u.end());
      u.erase(std::unique(u.begin(), u.end()), u.end());
      f.cols.clear();
      f.cols.push_back(s);
      for (int c : u)
        if (c != s) f.cols.push_back(c);
      f.coff.assign(f.cols.size() + 1, 0);
      for (size_t t = 0; t < f.cols.size(); ++t) f.coff[t + 1] = f.coff[t] + ccols_[(size_t)f.cols[t]];
      f.n = f.coff.back();
      f.nextra = (f.cols.size() > 1 && f.rs > f.c) ? f.rs - f.c : 0;
      gfirst[b + 1] = ng;
    }
  }, 64);
  for (size_t b = 0; b < batch.size(); ++b) {
    FrontInfo& f = fi[b];
    if (f.rs < f.c)
      throw Error(SPAQR_ERR_RANK_DEFICIENT,
                  "cluster " + std::to_string(f.s) + " at stage " + std::to_string(k_) + ": " + std::to_string(f.rs) +
                      " rows < " + std::to_string(f.c) + " columns");
    f.foff = ws;
    ws += (size_t)f.m * f.n;
    f.dest_off = ndest;
    ndest += (size_t)f.nextra;
    gfirst[b + 1] += gfirst[b];
  }
  T* W = static_cast<T*>(pool_.alloc(std::max<size_t>(ws, 1) * sizeof(T)));
  SPAQR_CUDA(cudaMemsetAsync(W, 0, std::max<size_t>(ws, 1) * sizeof(T), st_));
  lap("elim: front info");
  std::vector<FrontDesc<T>> fr(batch.size());
  gat.resize(gfirst.back());
  parallel_for((int64_t)batch.size(), [&](int64_t b0, int64_t b1, int) {
    for (int64_t bb = b0; bb < b1; ++bb) {
      const size_t b = (size_t)bb;
      const FrontInfo& f = fi[b];
      T* F = W + f.foff;
      int row = 0;
      size_t q = gfirst[b];
      for (int g : batch[b].second) {
        const Group& gg = G_[(size_t)g];
        for (size_t t = 0; t < gg.sup.size(); ++t) {
          const int c = gg.sup[t];
          if (gg.rows == 0 || ccols_[(size_t)c] == 0) continue;
          // f.cols = s, then the other clusters ascending
          const size_t ci = c == f.s ? 0
                                     : (size_t)(std::lower_bound(f.cols.begin() + 1, f.cols.end(), c) - f.cols.begin());
          gat[q++] = CopyDesc<T>{gg.ptr + (size_t)gg.off[t] * gg.ld, F + row + (size_t)f.coff[ci] * f.m, nullptr,
                                 gg.ld, f.m, gg.rows, ccols_[(size_t)c], 0, 0};
        }
        row += gg.rows;
      }
      fr[b] = FrontDesc<T>{F, f.m, f.n, f.c, f.m};
    }
  }, 64);
  ht_[2] += HT::now_s() - plan_t0;
  lap("elim: gather plan");
  copies(gat);
  front_qr(fr);
  lap("elim: gather+front launch");
  // extra-row destinations (max-norm rule over the remaining front clusters)
  std::vector<ArgmaxDesc<T>> am;
  std::vector<int> pack;  // per front: coff (ncl + 1), lvl (ncl), cid (ncl)
  std::vector<size_t> pack_off;
  int* d_dest = ndest ? static_cast<int*>(up_.scratch(ndest * sizeof(int))) : nullptr;
  int max_extra = 0;
  for (auto& f : fi) {
    if (!f.nextra) continue;
    const int ncl = (int)f.cols.size() - 1;
    pack_off.push_back(pack.size());
    // candidate clusters: all of them, or (tree rule) those of the deepest level; a
    // non-candidate gets level -1, which the kernel skips
    int deep = 0;
    for (int t = 0; t < ncl; ++t) deep = std::max(deep, level(f.cols[(size_t)t + 1]));
    for (int t = 0; t <= ncl; ++t) pack.push_back(f.coff[(size_t)t + 1]);
    for (int t = 0; t < ncl; ++t) {
      const int lv = level(f.cols[(size_t)t + 1]);
      pack.push_back(h_.opt.row_rule == SPAQR_ROWS_TREE && lv != deep ? -1 : lv);
    }
    for (int t = 0; t < ncl; ++t) pack.push_back(f.cols[(size_t)t + 1]);
  }
  if (!pack_off.empty()) {
    int* dp0 = up_.put(pack);
    size_t q = 0;
    for (auto& f : fi) {
      if (!f.nextra) continue;
      const int ncl = (int)f.cols.size() - 1;
      int* dp = dp0 + pack_off[q++];
      am.push_back(ArgmaxDesc<T>{W + f.foff, f.m, f.c, f.rs, ncl, dp, dp + ncl + 1, dp + 2 * ncl + 1,
                                 d_dest + f.dest_off});
      max_extra = std::max(max_extra, f.nextra);
    }
    if (checking_)
      for (auto& a : am) in_bounds(a.F, a.r1, 1, a.ld, sizeof(T), "argmax rows");
    auto* d = up_.put(am);
    auto its = items_for(am.size(), kRowsPerItem, [&](size_t i) { return am[i].r1 - am[i].r0; });
    int2* di = up_.put(its);
    tm_.begin(st_, 3);
    check(launch_argmax<T>(d, di, (int)its.size(), st_), "argmax");
    tm_.end(st_);
  }
  // R_s = [R_ss R_sn] into the W store
  lap("elim: argmax plan+launch");
  std::vector<CopyDesc<T>> rc;
  std::vector<WOp> nops(fi.size());
  parallel_for((int64_t)fi.size(), [&](int64_t b0, int64_t b1, int) {
    for (int64_t bb = b0; bb < b1; ++bb) {
      const FrontInfo& f = fi[(size_t)bb];
      WOp& op = nops[(size_t)bb];
      op.kind = 0;
      op.stage = k_;
      op.round = round;
      op.c = f.c;
      op.w = f.n - f.c;
      if (f.c <= 0) continue;
      op.slots = slots_[(size_t)f.s];
      size_t nsl = 0;
      for (size_t t = 1; t < f.cols.size(); ++t) nsl += slots_[(size_t)f.cols[t]].size();
      op.nslots.reserve(nsl);
      for (size_t t = 1; t < f.cols.size(); ++t)
        op.nslots.insert(op.nslots.end(), slots_[(size_t)f.cols[t]].begin(), slots_[(size_t)f.cols[t]].end());
    }
  }, 256);
  h_.ops.reserve(h_.ops.size() + fi.size());
  for (size_t b = 0; b < fi.size(); ++b) {
    const FrontInfo& f = fi[b];
    WOp& op = nops[b];
    if (f.c > 0) {
      T* R = wstore((size_t)f.c * f.n);
      op.R = R;
      rc.push_back(CopyDesc<T>{W + f.foff, R, nullptr, f.m, f.c, f.c, f.n, 0, 0});
    }
    h_.stats.n_fronts++;
    slog_.fronts++;
    slog_.max_m = std::max(slog_.max_m, f.m);
    slog_.max_n = std::max(slog_.max_n, f.n);
    slog_.max_c = std::max(slog_.max_c, f.c);
    h_.stats.max_front_rows = std::max<int64_t>(h_.stats.max_front_rows, f.m);
    h_.stats.max_front_cols = std::max<int64_t>(h_.stats.max_front_cols, f.n);
    if (k_ == 1) {
      h_.stats.top_rows = f.m;
      h_.stats.top_cols = f.c;
    }
    const double m = f.m, c = f.c, t = f.n - f.c;
    h_.stats.flops_front += 2.0 * c * c * (m - c / 3.0) + (4.0 * m * c - 2.0 * c * c) * t;
    if (f.c > 0) h_.ops.push_back(std::move(op));
  }
  copies(rc);
  std::vector<int> dest(ndest);
  lap("elim: W ops");
  sync_read(dest.data(), d_dest, ndest);
  // new groups: returned rows per owner, then extra rows per destination
  HT ht_new(ht_[3]);
  lap("elim: readback");
  // the new groups of every front in front order (ids assigned in that order):
  // first the returned rows, one group per other owner (contiguous rows from
  // position r_s on), then the extra rows c_s..r_s-1, one group per destination
  // cluster (rows listed in rowlist, by destination, ascending); every new
  // group of a front spans the front's remaining clusters
  struct Pending {
    int id;
    int front;
    int r0, cnt;  // contiguous rows (returned)
    int64_t roff; // first entry in rowlist (extra rows), -1 for returned rows
    int owner;
  };
  std::vector<size_t> pfirst(batch.size() + 1, 0);
  std::vector<int32_t> rowlist(ndest);
  std::atomic<int> bad_dest{0};
  parallel_for((int64_t)batch.size(), [&](int64_t b0, int64_t b1, int) {
    std::vector<int> cnt;
    for (int64_t bb = b0; bb < b1; ++bb) {
      const size_t b = (size_t)bb;
      const FrontInfo& f = fi[b];
      const size_t nrest = f.cols.size() - 1;
      const auto& fg = batch[b].second;
      size_t np = 0;
      if (nrest) {
        size_t q = 0;
        while (q < fg.size() && G_[(size_t)fg[q]].owner == f.s) ++q;
        while (q < fg.size()) {
          const int o = G_[(size_t)fg[q]].owner;
          while (q < fg.size() && G_[(size_t)fg[q]].owner == o) ++q;
          ++np;
        }
      }
      if (f.nextra) {
        cnt.assign(nrest + 1, 0);
        bool ok = true;
        for (int i = 0; i < f.nextra; ++i) {
          const int t = dest[f.dest_off + (size_t)i];
          if (t < 0 || t >= (int)nrest) {
            ok = false;
            break;
          }
          cnt[(size_t)t + 1]++;
        }
        if (!ok) {
          bad_dest.store(1);
          continue;
        }
        for (size_t t = 0; t < nrest; ++t) {
          np += cnt[t + 1] ? 1 : 0;
          cnt[t + 1] += cnt[t];
        }
        for (int i = 0; i < f.nextra; ++i) {
          const int t = dest[f.dest_off + (size_t)i];
          rowlist[f.dest_off + (size_t)cnt[(size_t)t]++] = f.c + i;
        }
      }
      pfirst[b + 1] = np;
    }
  }, 64);
  if (bad_dest.load()) throw Error(SPAQR_ERR_RANK_DEFICIENT, "non-finite values in a front at stage " + std::to_string(k_));
  for (size_t b = 0; b < batch.size(); ++b) pfirst[b + 1] += pfirst[b];
  std::vector<Pending> pend(pfirst.back());
  const int base = add_groups(pend.size());
  parallel_for((int64_t)batch.size(), [&](int64_t b0, int64_t b1, int) {
    for (int64_t bb = b0; bb < b1; ++bb) {
      const size_t b = (size_t)bb;
      const FrontInfo& f = fi[b];
      const size_t nrest = f.cols.size() - 1;
      const auto& fg = batch[b].second;
      size_t p = pfirst[b];
      if (nrest) {
        int pos = f.rs;
        size_t q = 0;
        while (q < fg.size() && G_[(size_t)fg[q]].owner == f.s) ++q;
        while (q < fg.size()) {
          const int o = G_[(size_t)fg[q]].owner;
          int c = 0;
          while (q < fg.size() && G_[(size_t)fg[q]].owner == o) c += G_[(size_t)fg[q++]].rows;
          pend[p] = Pending{base + (int)p, (int)b, pos, c, -1, o};
          ++p;
          pos += c;
        }
      }
      // extra rows: runs of equal destination in rowlist (destinations ascending)
      int64_t i = 0;
      while (i < f.nextra) {
        const int t = dest[f.dest_off + (size_t)(rowlist[f.dest_off + (size_t)i] - f.c)];
        int64_t j = i + 1;
        while (j < f.nextra && dest[f.dest_off + (size_t)(rowlist[f.dest_off + (size_t)j] - f.c)] == t) ++j;
        pend[p] = Pending{base + (int)p, (int)b, 0, (int)(j - i), (int64_t)f.dest_off + i, f.cols[(size_t)t + 1]};
        ++p;
        i = j;
      }
      for (size_t q = pfirst[b]; q < p; ++q)
        make_group(G_[(size_t)pend[q].id], pend[q].owner, pend[q].cnt, f.cols.data() + 1, f.cols.data() + f.cols.size());
    }
  }, 64);
  lap("elim: pending groups");
  std::vector<int> ids(pend.size());
  std::iota(ids.begin(), ids.end(), base);
  {
    std::vector<int> dead;
    for (size_t b = 0; b < batch.size(); ++b) {
      dead.insert(dead.end(), batch[b].second.begin(), batch[b].second.end());
      calive_[(size_t)fi[b].s] = 0;
    }
    kill_many(dead);
  }
  lap("elim: kill");
  assign_buffer(ids, false);
  std::vector<CopyDesc<T>> sc;
  lap("elim: new groups");
  int32_t* d_rows = rowlist.empty() ? nullptr : up_.put(rowlist);
  for (size_t i = 0; i < pend.size(); ++i) {
    const Pending& p = pend[i];
    const Group& g = G_[(size_t)p.id];
    const FrontInfo& f = fi[(size_t)p.front];
    if (g.rows == 0 || g.width == 0) continue;
    const T* src = W + f.foff + (size_t)f.c * f.m;
    if (p.roff < 0)
      sc.push_back(CopyDesc<T>{src + p.r0, g.ptr, nullptr, f.m, g.ld, g.rows, g.width, 0, 0});
    else
      sc.push_back(CopyDesc<T>{src, g.ptr, d_rows + p.roff, f.m, g.ld, g.rows, g.width, 0, 0});
  }
  copies(sc);
  pool_.release(W);
  lap("elim: scatter");
}

// ---------------------------------------------------------------- scale
template <typename T>
void Factorizer<T>::scale() {
  NT nt_f(this, "scale");
  phase_ = "scale";
  HT ht(ht_[4]);
  Lap lap(this);
  GroupIndex own, touch;
  index_groups(own, touch);
  p1_of_.assign(ccols_.size(), -1);
  p2_of_.assign(ccols_.size(), -1);
  struct SInfo {
    int p, rp, c, n;
    std::vector<int> cols, coff;
    size_t foff;
    T* R;
  };
  std::vector<SInfo> si;
  size_t ws = 0;
  for (size_t p = 0; p < ccols_.size(); ++p) {
    if (!calive_[p] || ccols_[p] == 0) continue;
    SInfo s;
    s.p = (int)p;
    s.c = ccols_[p];
    si.push_back(std::move(s));
  }
  // interfaces are independent: rows, column lists and gather counts in parallel
  std::vector<size_t> gfirst(si.size() + 1, 0);
  parallel_for((int64_t)si.size(), [&](int64_t q0, int64_t q1, int) {
    std::vector<int> u;
    for (int64_t qq = q0; qq < q1; ++qq) {
      SInfo& s = si[(size_t)qq];
      const size_t p = (size_t)s.p;
      s.rp = 0;
      u.clear();
      size_t ng = 0;
      for (int g : own[p]) {
        const Group& gg = G_[(size_t)g];
        s.rp += gg.rows;
        u.insert(u.end(), gg.sup.begin(), gg.sup.end());
        if (gg.rows)
          for (int c : gg.sup) ng += ccols_[(size_t)c] ? 1 : 0;
      }
      std::sort(u.begin(), u.end());
      u.erase(std::unique(u.begin(), u.end()), u.end());
      s.cols.push_back((int)p);
      for (int c : u)
        if (c != (int)p) s.cols.push_back(c);
      s.coff.assign(s.cols.size() + 1, 0);
      for (size_t t = 0; t < s.cols.size(); ++t) s.coff[t + 1] = s.coff[t] + ccols_[(size_t)s.cols[t]];
      s.n = s.coff.back();
      gfirst[(size_t)qq + 1] = ng;
    }
  }, 64);
  for (size_t q = 0; q < si.size(); ++q) {
    SInfo& s = si[q];
    if (s.rp < s.c)
      throw Error(SPAQR_ERR_RANK_DEFICIENT, "interface " + std::to_string(s.p) + " at stage " + std::to_string(k_) +
                                                ": " + std::to_string(s.rp) + " rows < " + std::to_string(s.c) +
                                                " columns");
    s.foff = ws;
    ws += (size_t)s.rp * s.n;
    gfirst[q + 1] += gfirst[q];
  }
  lap("scale: info");
  if (si.empty()) return;
  T* W = static_cast<T*>(pool_.alloc(std::max<size_t>(ws, 1) * sizeof(T)));
  SPAQR_CUDA(cudaMemsetAsync(W, 0, std::max<size_t>(ws, 1) * sizeof(T), st_));
  std::vector<CopyDesc<T>> gat(gfirst.back());
  std::vector<FrontDesc<T>> fr(si.size());
  parallel_for((int64_t)si.size(), [&](int64_t q0, int64_t q1, int) {
    for (int64_t qq = q0; qq < q1; ++qq) {
      const SInfo& s = si[(size_t)qq];
      T* F = W + s.foff;
      int row = 0;
      size_t q = gfirst[(size_t)qq];
      for (int g : own[(size_t)s.p]) {
        const Group& gg = G_[(size_t)g];
        for (size_t t = 0; t < gg.sup.size(); ++t) {
          const int c = gg.sup[t];
          if (gg.rows == 0 || ccols_[(size_t)c] == 0) continue;
          // s.cols = p, then the other clusters ascending
          const size_t ci = c == s.p ? 0
                                     : (size_t)(std::lower_bound(s.cols.begin() + 1, s.cols.end(), c) - s.cols.begin());
          gat[q++] = CopyDesc<T>{gg.ptr + (size_t)gg.off[t] * gg.ld, F + row + (size_t)s.coff[ci] * s.rp, nullptr,
                                 gg.ld, s.rp, gg.rows, ccols_[(size_t)c], 0, 0};
        }
        row += gg.rows;
      }
      fr[(size_t)qq] = FrontDesc<T>{F, s.rp, s.n, s.c, s.rp};
    }
  }, 64);
  for (auto& s : si) {
    slog_.scaled++;
    slog_.max_rp = std::max(slog_.max_rp, s.rp);
    const double m = s.rp, c = s.c, t = s.n - s.c;
    h_.stats.flops_front += 2.0 * c * c * (m - c / 3.0) + (4.0 * m * c - 2.0 * c * c) * t;
  }
  lap("scale: gather plan");
  copies(gat);
  front_qr(fr);
  lap("scale: gather+front launch");
  // R_pp into the W store; new groups p1 (identity on p) and p2
  std::vector<CopyDesc<T>> rc, idn, cp;
  std::vector<int> ids;
  // serial: W store blocks, ops in order, kills and group ids; parallel: the group layouts
  {
    size_t ng = 0;
    for (auto& s : si) ng += 1 + ((s.rp > s.c && s.cols.size() > 1) ? 1 : 0);
    const int base = add_groups(ng);
    int next = base;
    std::vector<int> dead;
    h_.ops.reserve(h_.ops.size() + si.size());
    const size_t op0 = h_.ops.size();
    h_.ops.resize(op0 + si.size());
    parallel_for((int64_t)si.size(), [&](int64_t q0, int64_t q1, int) {
      for (int64_t q = q0; q < q1; ++q) h_.ops[op0 + (size_t)q].slots = slots_[(size_t)si[(size_t)q].p];
    }, 256);
    size_t opi = op0;
    for (auto& s : si) {
      WOp& op = h_.ops[opi++];
      op.kind = 1;
      op.stage = k_;
      op.c = s.c;
      s.R = wstore((size_t)s.c * s.c);
      op.R = s.R;
      rc.push_back(CopyDesc<T>{W + s.foff, s.R, nullptr, s.rp, s.c, s.c, s.c, 0, 0});
      dead.insert(dead.end(), own[(size_t)s.p].begin(), own[(size_t)s.p].end());
      p1_of_[(size_t)s.p] = next;
      ids.push_back(next++);
      if (s.rp > s.c && s.cols.size() > 1) {
        p2_of_[(size_t)s.p] = next;
        ids.push_back(next++);
      }
    }
    lap("scale: ops");
    kill_many(dead);
    lap("scale: kill");
    parallel_for((int64_t)si.size(), [&](int64_t b, int64_t e, int) {
      for (int64_t q = b; q < e; ++q) {
        const SInfo& s = si[(size_t)q];
        std::vector<int> sup1(s.cols.begin(), s.cols.end());
        std::sort(sup1.begin(), sup1.end());
        make_group(G_[(size_t)p1_of_[(size_t)s.p]], s.p, s.c, sup1.data(), sup1.data() + sup1.size());
        if (p2_of_[(size_t)s.p] >= 0) {
          std::vector<int> rest(s.cols.begin() + 1, s.cols.end());
          std::sort(rest.begin(), rest.end());
          make_group(G_[(size_t)p2_of_[(size_t)s.p]], s.p, s.rp - s.c, rest.data(), rest.data() + rest.size());
        }
      }
    }, 1024);
  }
  lap("scale: groups");
  assign_buffer(ids, false);
  for (auto& s : si) {
    const T* F = W + s.foff;
    const Group& g1 = G_[(size_t)p1_of_[(size_t)s.p]];
    for (size_t t = 0; t < s.cols.size(); ++t) {
      const int c = s.cols[t];
      const int wc = ccols_[(size_t)c];
      if (wc == 0) continue;
      T* dst1 = g1.ptr + (size_t)col_off(g1, c) * g1.ld;
      if (t == 0)
        idn.push_back(CopyDesc<T>{nullptr, dst1, nullptr, 0, g1.ld, s.c, s.c, 0, 0});
      else
        cp.push_back(CopyDesc<T>{F + (size_t)s.coff[t] * s.rp, dst1, nullptr, s.rp, g1.ld, s.c, wc, 0, 0});
      if (t > 0 && p2_of_[(size_t)s.p] >= 0) {
        const Group& g2 = G_[(size_t)p2_of_[(size_t)s.p]];
        cp.push_back(CopyDesc<T>{F + s.c + (size_t)s.coff[t] * s.rp, g2.ptr + (size_t)col_off(g2, c) * g2.ld,
                                 nullptr, s.rp, g2.ld, g2.rows, wc, 0, 0});
      }
    }
  }
  copies(rc);
  copies(cp);
  if (!idn.empty()) {
    auto* d = up_.put(idn);
    check(launch_identity<T>(d, (int)idn.size(), st_), "identity");
  }
  lap("scale: p1/p2 copies");
  pool_.release(W);
  // X <- X R_pp^{-1} on every block column p of the other owners' rows
  std::vector<T*> Rof(ccols_.size(), nullptr);
  for (auto& s : si) Rof[(size_t)s.p] = s.R;
  std::vector<TrsmDesc<T>> tr;
  int maxr = 0;
  for (int id : live()) {
    const Group& g = G_[(size_t)id];
    if (g.rows == 0) continue;
    for (size_t t = 0; t < g.sup.size(); ++t) {
      const int c = g.sup[t];
      if (c == g.owner || !Rof[(size_t)c]) continue;
      tr.push_back(TrsmDesc<T>{g.ptr + (size_t)g.off[t] * g.ld, Rof[(size_t)c], g.ld, g.rows, ccols_[(size_t)c],
                               ccols_[(size_t)c]});
      maxr = std::max(maxr, g.rows);
    }
  }
  lap("scale: trsm plan");
  if (checking_)
    for (auto& t : tr) {
      in_bounds(t.ptr, t.rows, t.c, t.ld, sizeof(T), "trsm X");
      in_bounds(t.R, t.c, t.c, t.rld, sizeof(T), "trsm R");
    }
  if (!tr.empty()) {
    auto* d = up_.put(tr);
    auto its = items_for(tr.size(), kRowsPerItem, [&](size_t i) { return tr[i].rows; });
    int2* di = up_.put(its);
    tm_.begin(st_, 3);
    check(launch_trsm<T>(d, di, (int)its.size(), st_), "trsm");
    tm_.end(st_);
  }
}

// ---------------------------------------------------------------- step 1
template <typename T>
void Factorizer<T>::step1() {
  NT nt_f(this, "step1");
  phase_ = "step1";
  std::vector<QrcpDesc<T>> qs;
  std::vector<int> who;
  for (size_t p = 0; p < ccols_.size(); ++p) {
    const int id = p2_of_.empty() ? -1 : p2_of_[p];
    if (id < 0) continue;
    Group& g = G_[(size_t)id];
    if (g.rows == 0 || g.width == 0) continue;
    who.push_back(id);
  }
  if (who.empty()) return;
  int* d_rank = static_cast<int*>(up_.scratch(who.size() * sizeof(int)));
  // A tall block X (rows well above its width) is first reduced by a
  // Householder QR to its width x width triangle R0; the column-pivoted QR of R0
  // then takes the same pivots, rank and, up to row signs, the same rows as that
  // of X, since every partial column norm is invariant under the orthogonal
  // factor.  Both routes write the kept rows with R_ii >= 0.
  // The QR pays off for wide blocks (measured: the 3D separator blocks gain, the
  // narrower 2D blocks lose a little), hence a width floor next to the aspect ratio.
  const double qr_ratio = 1.1;
  const int qr_min_width = h_.opt.step1_qr_width;
  std::vector<FrontDesc<T>> fr;
  std::vector<char> tall(who.size(), 0);
  for (size_t i = 0; i < who.size(); ++i) {
    Group& g = G_[(size_t)who[i]];
    slog_.s1++;
    slog_.s1_max_m = std::max(slog_.s1_max_m, g.rows);
    slog_.s1_max_n = std::max(slog_.s1_max_n, g.width);
    tall[i] = qr_min_width > 0 && g.width >= std::max(32, qr_min_width) && g.rows >= qr_ratio * g.width;
    if (tall[i]) {
      fr.push_back(FrontDesc<T>{g.ptr, g.rows, g.width, g.width, g.ld});
      qs.push_back(QrcpDesc<T>{g.ptr, nullptr, g.ptr, nullptr, nullptr, d_rank + i, g.width, g.width, g.ld, g.ld,
                               kQrcpSignFix | kQrcpAlwaysOut});
    } else {
      qs.push_back(QrcpDesc<T>{g.ptr, nullptr, g.ptr, nullptr, nullptr, d_rank + i, g.rows, g.width, g.ld, g.ld,
                               kQrcpSignFix});
    }
  }
  front_qr(fr);
  std::vector<T*> work;
  qrcp(qs, work);
  prepare_step2();  // while the device runs step 1
  std::vector<int> rank(who.size());
  sync_read(rank.data(), d_rank, who.size());
  for (T* w : work) pool_.release(w);
  for (size_t i = 0; i < who.size(); ++i) {
    Group& g = G_[(size_t)who[i]];
    if (rank[i] < 0)  // only an expired exchange wait writes a negative rank
      throw Error(SPAQR_ERR_TIMEOUT, "step 1: column-pivoted QR exchange wait timed out");
    if (rank[i] < 0 || rank[i] > std::min(g.rows, g.width))
      throw Error(SPAQR_ERR_CUDA, "step 1: rank " + std::to_string(rank[i]) + " out of range for a " +
                                      std::to_string(g.rows) + " x " + std::to_string(g.width) + " block at stage " +
                                      std::to_string(k_));
    const double n = g.width, m = tall[i] ? n : (double)g.rows, k = rank[i];
    if (tall[i]) {  // the Householder QR of the tall block runs as a front
      h_.stats.flops_sparsify += 2.0 * n * n * (g.rows - n / 3.0);
      h_.stats.flops_front += 2.0 * n * n * (g.rows - n / 3.0);
    }
    h_.stats.flops_sparsify += 4.0 * m * n * k - 2.0 * k * k * (m + n) + 4.0 * k * k * k / 3.0;
    h_.stats.flops_qrcp += 4.0 * m * n * k - 2.0 * k * k * (m + n) + 4.0 * k * k * k / 3.0;
    h_.stats.bytes_qrcp += sizeof(T) * (k * m * n - k * k * (m + n) / 2.0 + k * k * k / 3.0 + 2.0 * m * n);
    if (rank[i] < g.rows) {
      g.rows = rank[i];
      if (g.rows == 0) {
        kill(who[i]);
        p2_of_[(size_t)g.owner] = -1;
      }
    }
  }
}

// ---------------------------------------------------------------- step 2
template <typename T>
void Factorizer<T>::prepare_step2() {
  NT nt_f(this, "step2: prepare");
  S2Plan& P = s2_;
  P = S2Plan();
  P.ready = true;
  for (size_t p = 0; p < ccols_.size(); ++p)
    if (!p1_of_.empty() && p1_of_[p] >= 0) P.ps.push_back((int)p);
  if (P.ps.empty()) return;
  // greedy colouring of q ~ p  <=>  q in support(p1 of p) or p in support(p1 of q)
  const size_t nc = ccols_.size();
  std::vector<std::vector<int>> adj(nc);
  for (int p : P.ps) {
    for (int q : G_[(size_t)p1_of_[(size_t)p]].sup)
      if (q != p && p1_of_[(size_t)q] >= 0) {
        adj[(size_t)p].push_back(q);
        adj[(size_t)q].push_back(p);
      }
  }
  std::vector<int> colour(nc, -1);
  int ncol = 0;
  std::vector<char> used;
  for (int p : P.ps) {
    used.assign((size_t)ncol + 1, 0);
    for (int q : adj[(size_t)p])
      if (colour[(size_t)q] >= 0) used[(size_t)colour[(size_t)q]] = 1;
    int c = 0;
    while (c < ncol && used[(size_t)c]) ++c;
    colour[(size_t)p] = c;
    ncol = std::max(ncol, c + 1);
  }
  P.ncol = ncol;
  P.members.assign((size_t)ncol, {});
  for (int p : P.ps) P.members[(size_t)colour[(size_t)p]].push_back(p);
  GroupIndex own, touch;
  index_groups(own, touch);
  P.pre.resize((size_t)ncol);
  std::vector<std::pair<int, int>> all;  // (colour, member)
  for (int col = 0; col < ncol; ++col) {
    P.pre[(size_t)col].resize(P.members[(size_t)col].size());
    for (size_t q = 0; q < P.members[(size_t)col].size(); ++q) all.emplace_back(col, (int)q);
  }
  parallel_for((int64_t)all.size(), [&](int64_t b, int64_t e, int) {
    for (int64_t t = b; t < e; ++t) {
      const int col = all[(size_t)t].first, q = all[(size_t)t].second;
      const int p = P.members[(size_t)col][(size_t)q];
      S2Member& x = P.pre[(size_t)col][(size_t)q];
      for (int g : touch[(size_t)p])
        if (G_[(size_t)g].alive) x.nb.push_back(g);
      std::sort(x.nb.begin(), x.nb.end(), [&](int a, int c) {
        const int oa = G_[(size_t)a].owner, oc = G_[(size_t)c].owner;
        return oa != oc ? oa < oc : a < c;
      });
      const Group& g1 = G_[(size_t)p1_of_[(size_t)p]];
      for (int c : g1.sup)
        if (c != p) {
          x.ncols.push_back(c);
          x.cn += ccols_[(size_t)c];
        }
    }
  }, 16);
}

template <typename T>
void Factorizer<T>::step2() {
  NT nt_f(this, "step2");
  phase_ = "step2";
  Lap lap(this);
  HT ht(ht_[5]);
  if (!s2_.ready) prepare_step2();
  s2_.ready = false;
  const std::vector<int>& ps = s2_.ps;
  if (ps.empty()) return;
  const int ncol = s2_.ncol;
  slog_.colours = ncol;
  lap("step2: prepare (not overlapped)");
  // one device rank slot per interface of this phase, read back with a single copy
  int* kdev_all = static_cast<int*>(h_.wpool.alloc(ps.size() * sizeof(int)));
  size_t kdev_next = 0;
  struct P2 {
    int p;
    size_t op;
    int ncm;
  };
  std::vector<P2> recs;
  std::vector<T*> work_all;
  const size_t ops0 = h_.ops.size();  // this phase's ops are appended from here
  const auto& members = s2_.members;
  for (int col = 0; col < ncol; ++col) {
    struct MInfo {
      int p, cp, rn, cn;
      std::vector<int> nb, ncols;
      size_t moff, cfirst, rfirst;
    };
    const auto& mem = members[(size_t)col];
    std::vector<MInfo> mi(mem.size());
    // members of a colour are independent: M_p's blocks and descriptor counts in parallel
    parallel_for((int64_t)mem.size(), [&](int64_t q0, int64_t q1, int) {
      for (int64_t qq = q0; qq < q1; ++qq) {
        MInfo& x = mi[(size_t)qq];
        S2Member& pre = s2_.pre[(size_t)col][(size_t)qq];
        const int p = mem[(size_t)qq];
        x.p = p;
        x.cp = ccols_[(size_t)p];
        // groups that step 1 emptied (rank 0) are gone
        x.nb.swap(pre.nb);
        x.nb.erase(std::remove_if(x.nb.begin(), x.nb.end(), [&](int g) { return !G_[(size_t)g].alive; }), x.nb.end());
        x.rn = 0;
        size_t nc = 0;
        for (int g : x.nb) {
          x.rn += G_[(size_t)g].rows;
          nc += G_[(size_t)g].rows ? 1 : 0;
        }
        x.ncols.swap(pre.ncols);
        x.cn = pre.cn;
        for (int c : x.ncols) nc += ccols_[(size_t)c] ? 1 : 0;
        x.cfirst = nc;  // a count here, offsets below
      }
    }, 16);
    size_t ws = 0, ncps = 0;
    for (auto& x : mi) {
      x.moff = ws;
      ws += (size_t)x.cp * (x.rn + x.cn);
      const size_t n = x.cfirst;
      x.cfirst = ncps;
      x.rfirst = ncps;  // one reflector descriptor per copied block
      ncps += n;
    }
    T* M = static_cast<T*>(pool_.alloc(std::max<size_t>(ws, 1) * sizeof(T)));
    std::vector<CopyDesc<T>> cps(ncps);
    std::vector<ReflDesc<T>> rf(ncps);
    std::vector<QrcpDesc<T>> qs(mi.size());
    const size_t op0 = h_.ops.size();
    h_.ops.resize(op0 + mi.size());
    for (size_t q = 0; q < mi.size(); ++q) {
      const MInfo& x = mi[q];
      const int ncm = x.rn + x.cn;
      const int kmax = std::min(x.cp, ncm);
      slog_.s2++;
      slog_.s2_max_c = std::max(slog_.s2_max_c, x.cp);
      slog_.s2_max_w = std::max(slog_.s2_max_w, ncm);
      WOp& op = h_.ops[op0 + q];
      op.kind = 2;
      op.stage = k_;
      op.round = col;
      op.c = x.cp;
      op.w = kmax;
      op.V = wstore((size_t)x.cp * std::max(kmax, 1));
      op.tau = wstore((size_t)std::max(kmax, 1));
      op.kdev = kdev_all + kdev_next++;
      qs[q] = QrcpDesc<T>{M + x.moff, nullptr, nullptr, static_cast<T*>(op.V), static_cast<T*>(op.tau), op.kdev,
                          x.cp, ncm, x.cp, x.cp};
      recs.push_back(P2{x.p, op0 + q, ncm});
    }
    parallel_for((int64_t)mi.size(), [&](int64_t q0, int64_t q1, int) {
      for (int64_t qq = q0; qq < q1; ++qq) {
        const MInfo& x = mi[(size_t)qq];
        const WOp& op = h_.ops[op0 + (size_t)qq];
        h_.ops[op0 + (size_t)qq].slots = slots_[(size_t)x.p];
        T* Mp = M + x.moff;
        T* V = static_cast<T*>(op.V);
        T* tau = static_cast<T*>(op.tau);
        size_t ci = x.cfirst;
        int colm = 0;
        for (int g : x.nb) {
          const Group& gg = G_[(size_t)g];
          if (gg.rows) {
            T* blk = gg.ptr + (size_t)col_off(gg, x.p) * gg.ld;
            cps[ci] = CopyDesc<T>{blk, Mp + (size_t)colm * x.cp, nullptr, gg.ld, x.cp, gg.rows, x.cp, 1, 0};
            rf[ci] = ReflDesc<T>{blk, V, tau, op.kdev, gg.ld, x.cp, gg.rows, 0};
            ++ci;
          }
          colm += gg.rows;
        }
        const Group& g1 = G_[(size_t)p1_of_[(size_t)x.p]];
        for (int c : x.ncols) {
          if (ccols_[(size_t)c]) {
            T* blk = g1.ptr + (size_t)col_off(g1, c) * g1.ld;
            cps[ci] = CopyDesc<T>{blk, Mp + (size_t)colm * x.cp, nullptr, g1.ld, x.cp, x.cp, ccols_[(size_t)c], 0, 0};
            rf[ci] = ReflDesc<T>{blk, V, tau, op.kdev, g1.ld, x.cp, ccols_[(size_t)c], 1};
            ++ci;
          }
          colm += ccols_[(size_t)c];
        }
      }
    }, 16);
    lap("step2: colour plan");
    copies(cps);
    qrcp(qs, work_all);
    if (checking_)
      for (auto& r : rf) {
        if (r.mode == 0)
          in_bounds(r.ptr, r.nvec, r.len, r.ld, sizeof(T), "refl rows");
        else
          in_bounds(r.ptr, r.len, r.nvec, r.ld, sizeof(T), "refl cols");
      }
    if (!rf.empty()) {
      auto* d = up_.put(rf);
      std::vector<int2> its;
      for (size_t i = 0; i < rf.size(); ++i) {
        const int per = (rf[i].mode == 0 && sizeof(T) == 4) ? kReflRowsPerItem : kReflPerItem;
        for (int u = 0; u < rf[i].nvec; u += per) its.push_back(make_int2((int)i, u));
      }
      int2* di = up_.put(its);
      tm_.begin(st_, 3);
      check(launch_refl<T>(d, di, (int)its.size(), st_), "refl");
      tm_.end(st_);
    }
    pool_.release(M);
    lap("step2: colour launches");
  }
  // ranks back; keep the ops that drop something
  std::vector<int> kall(std::max<size_t>(kdev_next, 1));
  sync();
  if (kdev_next) SPAQR_CUDA(cudaMemcpy(kall.data(), kdev_all, kdev_next * sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<int> ks(recs.size());
  lap("step2: readback");
  for (size_t i = 0; i < recs.size(); ++i) {
    ks[i] = kall[(size_t)(h_.ops[recs[i].op].kdev - kdev_all)];
    if (ks[i] < 0)  // only an expired exchange wait writes a negative rank
      throw Error(SPAQR_ERR_TIMEOUT, "step 2: column-pivoted QR exchange wait timed out");
    if (ks[i] < 0 || ks[i] > std::min(h_.ops[recs[i].op].c, recs[i].ncm))
      throw Error(SPAQR_ERR_CUDA, "step 2: rank " + std::to_string(ks[i]) + " out of range at stage " +
                                      std::to_string(k_));
  }
  for (T* w : work_all) pool_.release(w);
  std::vector<char> drop(h_.ops.size() - ops0, 0);
  for (size_t i = 0; i < recs.size(); ++i) {
    WOp& op = h_.ops[recs[i].op];
    const int k = ks[i], p = recs[i].p;
    op.k = k;
    slog_.sum_c += op.c;
    slog_.sum_k += std::min(k, op.c);
    {
      // column-pivoted QR to rank k of the c_p x ncm block, then the two-sided application
      const double m = op.c, n = recs[i].ncm, kk = k;
      h_.stats.flops_sparsify += 4.0 * m * n * kk - 2.0 * kk * kk * (m + n) + 4.0 * kk * kk * kk / 3.0;
      h_.stats.flops_qrcp += 4.0 * m * n * kk - 2.0 * kk * kk * (m + n) + 4.0 * kk * kk * kk / 3.0;
      h_.stats.bytes_qrcp += sizeof(T) * (kk * m * n - kk * kk * (m + n) / 2.0 + kk * kk * kk / 3.0 + 2.0 * m * n);
      h_.stats.flops_sparsify += 4.0 * kk * m * n;
    }
    if (k >= op.c) {
      drop[recs[i].op - ops0] = 1;
      continue;
    }
    ccols_[(size_t)p] = k;
    slots_[(size_t)p].resize((size_t)k);
    Group& g1 = G_[(size_t)p1_of_[(size_t)p]];
    g1.rows = k;
    if (k == 0) {
      kill(p1_of_[(size_t)p]);
      p1_of_[(size_t)p] = -1;
    }
  }
  // remove identity ops (k == c) -- their device blocks stay in the W pool
  size_t w = ops0;
  for (size_t i = ops0; i < h_.ops.size(); ++i)
    if (!drop[i - ops0]) {
      if (w != i) h_.ops[w] = std::move(h_.ops[i]);
      ++w;
    }
  h_.ops.resize(w);
  lap("step2: rank bookkeeping");
}

// ---------------------------------------------------------------- merge
template <typename T>
void Factorizer<T>::merge() {
  NT nt_f(this, "merge");
  phase_ = "merge";
  Lap lap(this);
  HT ht(ht_[6]);
  const StageClusters& nxt = an_.stages[(size_t)k_ - 1];
  const size_t nnew = nxt.node.size();
  std::vector<int> nccols(nnew, 0);
  std::vector<std::vector<int32_t>> nslots(nnew);
  std::vector<int> choff(ccols_.size(), 0), nchild(nnew, 0);
  // children of every parent in ascending id (CSR), then each parent's slots in parallel
  std::vector<int64_t> cptr(nnew + 1, 0);
  for (size_t c = 0; c < ccols_.size(); ++c) {
    if (!calive_[c]) continue;
    const int P = sc_->parent[c];
    if (P < 0) throw Error(SPAQR_ERR_CUDA, "internal: live cluster without parent");
    choff[c] = nccols[(size_t)P];
    nccols[(size_t)P] += ccols_[c];
    nchild[(size_t)P]++;
    cptr[(size_t)P + 1]++;
  }
  for (size_t P = 0; P < nnew; ++P) cptr[P + 1] += cptr[P];
  std::vector<int> kids((size_t)cptr[nnew]);
  {
    std::vector<int64_t> at(cptr.begin(), cptr.end() - 1);
    for (size_t c = 0; c < ccols_.size(); ++c)
      if (calive_[c]) kids[(size_t)at[(size_t)sc_->parent[c]]++] = (int)c;
  }
  parallel_for((int64_t)nnew, [&](int64_t b, int64_t e, int) {
    for (int64_t P = b; P < e; ++P) {
      auto& v = nslots[(size_t)P];
      v.reserve((size_t)nccols[(size_t)P]);
      for (int64_t q = cptr[(size_t)P]; q < cptr[(size_t)P + 1]; ++q) {
        const auto& sl = slots_[(size_t)kids[(size_t)q]];
        v.insert(v.end(), sl.begin(), sl.end());
      }
    }
  }, 256);
  lap("merge: clusters");
  // groups whose column layout changes get a new block (groups are independent:
  // classified in parallel, moved ones listed in ascending id)
  std::vector<int> moved;
  std::vector<CopyDesc<T>> cps;
  {
    const std::vector<int>& lv = live();
    std::vector<char> mv(lv.size(), 0);
    parallel_for((int64_t)lv.size(), [&](int64_t b, int64_t e, int) {
      std::vector<int> nsup;
      for (int64_t i = b; i < e; ++i) {
        Group& g = G_[(size_t)lv[(size_t)i]];
        nsup.clear();
        for (int c : g.sup) nsup.push_back(sc_->parent[(size_t)c]);
        std::sort(nsup.begin(), nsup.end());
        nsup.erase(std::unique(nsup.begin(), nsup.end()), nsup.end());
        bool same = nsup.size() == g.sup.size();
        for (size_t t = 0; same && t < g.sup.size(); ++t) {
          const int c = g.sup[t], P = sc_->parent[(size_t)c];
          if (nchild[(size_t)P] != 1) same = false;
          // columns dropped by step 2 (block width larger than the cluster now)
          const int wold = (t + 1 < g.sup.size() ? g.off[t + 1] : g.width) - g.off[t];
          if (wold != ccols_[(size_t)c]) same = false;
        }
        g.owner = sc_->parent[(size_t)g.owner];
        if (same) {
          for (auto& c : g.sup) c = sc_->parent[(size_t)c];
          continue;
        }
        mv[(size_t)i] = 1;
      }
    }, 4096);
    for (size_t i = 0; i < lv.size(); ++i)
      if (mv[i]) moved.push_back(lv[i]);
  }
  lap("merge: classify groups");
  // new blocks for moved groups (one buffer, zero-filled); the old layout is kept for the copies
  std::vector<SmallInts> oldsup(moved.size()), oldoff(moved.size());
  std::vector<T*> oldptr(moved.size());
  std::vector<int> oldld(moved.size()), oldbuf(moved.size());
  parallel_for((int64_t)moved.size(), [&](int64_t b, int64_t e, int) {
    for (int64_t ii = b; ii < e; ++ii) {
      const size_t i = (size_t)ii;
      Group& g = G_[(size_t)moved[i]];
      oldsup[i].swap(g.sup);
      oldoff[i].swap(g.off);
      oldptr[i] = g.ptr;
      oldld[i] = g.ld;
      oldbuf[i] = g.buf;
      std::vector<int> nsup;
      nsup.reserve(oldsup[i].size());
      for (int c : oldsup[i]) nsup.push_back(sc_->parent[(size_t)c]);
      std::sort(nsup.begin(), nsup.end());
      nsup.erase(std::unique(nsup.begin(), nsup.end()), nsup.end());
      g.off.resize(nsup.size());
      int w = 0;
      for (size_t t = 0; t < nsup.size(); ++t) {
        g.off[t] = w;
        w += nccols[(size_t)nsup[t]];
      }
      g.sup.assign(nsup.data(), nsup.data() + nsup.size());
      g.width = w;
      g.ld = std::max(g.rows, 1);
      g.buf = -1;
      g.ptr = nullptr;
    }
  }, 4096);
  lap("merge: new layouts");
  {
    size_t total = 0;
    for (int id : moved) total += (size_t)G_[(size_t)id].ld * G_[(size_t)id].width;
    if (total) {
      T* base = static_cast<T*>(pool_.alloc(total * sizeof(T)));
      SPAQR_CUDA(cudaMemsetAsync(base, 0, total * sizeof(T), st_));
      bufs_.push_back(Buf{base, 0});
      const int b = (int)bufs_.size() - 1;
      size_t o = 0;
      for (int id : moved) {
        Group& g = G_[(size_t)id];
        const size_t sz = (size_t)g.ld * g.width;
        if (sz) {
          g.ptr = base + o;
          g.buf = b;
          bufs_[(size_t)b].refs++;
        }
        o += sz;
      }
      if (bufs_[(size_t)b].refs == 0) pool_.release(base);
    }
  }
  // relayout copies: counted, then filled in parallel in (group, old cluster) order
  {
    std::vector<size_t> first(moved.size() + 1, 0);
    for (size_t i = 0; i < moved.size(); ++i) {
      const Group& g = G_[(size_t)moved[i]];
      size_t cnt = 0;
      if (g.rows)
        for (int c : oldsup[i]) cnt += ccols_[(size_t)c] ? 1 : 0;
      first[i + 1] = first[i] + cnt;
    }
    cps.resize(first.back());
    parallel_for((int64_t)moved.size(), [&](int64_t b, int64_t e, int) {
      for (int64_t ii = b; ii < e; ++ii) {
        const size_t i = (size_t)ii;
        const Group& g = G_[(size_t)moved[i]];
        size_t q = first[i];
        for (size_t t = 0; t < oldsup[i].size(); ++t) {
          const int c = oldsup[i][t];
          const int P = sc_->parent[(size_t)c];
          const int wc = ccols_[(size_t)c];
          if (wc == 0 || g.rows == 0) continue;
          const int dcol = col_off(g, P) + choff[(size_t)c];
          cps[q++] = CopyDesc<T>{oldptr[i] + (size_t)oldoff[i][t] * oldld[i], g.ptr + (size_t)dcol * g.ld, nullptr,
                                 oldld[i], g.ld, g.rows, wc, 0, 0};
        }
      }
    }, 4096);
  }
  lap("merge: relayout plan");
  copies(cps);
  for (size_t i = 0; i < moved.size(); ++i) {
    if (oldbuf[i] >= 0) {
      Buf& b = bufs_[(size_t)oldbuf[i]];
      if (--b.refs == 0) {
        pool_.release(b.p);
        b.p = nullptr;
      }
    }
  }
  lap("merge: copies");
  // adopt the stage k-1 clusters
  sc_ = &nxt;
  ccols_.swap(nccols);
  slots_.swap(nslots);
  calive_.assign(nnew, 1);
  p1_of_.clear();
  p2_of_.clear();
}

template <typename T>
void Factorizer<T>::run(const spaqr_csr& A) {
  L_ = an_.depth;
  smem_max_ = max_smem_optin();
  grid_ctas_ = qrcp_grid_capacity(smem_max_, (int)sizeof(T));
  {
    const char* e = std::getenv("SPAQR_CHECK");
    checking_ = e && e[0] == '1';
  }
  double t0 = now();
  up_.init(st_, size_t(32) << 20);
  nt_add("upload arena", now() - t0);
  init_stage(A);
  double tp[6] = {0, 0, 0, 0, 0, 0};
  tp[1] = now() - t0;
  double kt_prev[6] = {0, 0, 0, 0, 0, 0};
  for (k_ = L_; k_ >= 1; --k_) {
    double a = now();
    eliminate();
    double b = now();
    tp[0] += b - a;
    if (sparsify_here()) {
      scale();
      double c = now();
      tp[2] += c - b;
      step1();
      double d = now();
      tp[3] += d - c;
      step2();
      double e = now();
      tp[4] += e - d;
      b = e;
    }
    if (k_ > 1) {
      merge();
      double f = now();
      tp[5] += f - b;
    }
    if (h_.opt.verbose) {
      const size_t live = this->live().size();
      const StageLog& g = slog_;
      std::fprintf(stderr,
                   "[spaqr] stage %2d: fronts %5d rounds %d max m/n/c %d/%d/%d | scaled %d max r_p %d | step1 %d max "
                   "%dx%d | step2 %d colours %d max c %d x %d, kept %lld of %lld | live groups %zu pool %.0f MB\n",
                   k_, g.fronts, g.rounds, g.max_m, g.max_n, g.max_c, g.scaled, g.max_rp, g.s1, g.s1_max_m, g.s1_max_n,
                   g.s2, g.colours, g.s2_max_c, g.s2_max_w, (long long)g.sum_k, (long long)g.sum_c, live,
                   pool_.in_use() / 1e6);
      std::fprintf(stderr, "[spaqr]           device ms: copy %.2f front %.2f qrcp %.2f other %.2f\n",
                   1e3 * (h_.stats.t_kernel[0] - kt_prev[0]), 1e3 * (h_.stats.t_kernel[1] - kt_prev[1]),
                   1e3 * (h_.stats.t_kernel[2] - kt_prev[2]), 1e3 * (h_.stats.t_kernel[3] - kt_prev[3]));
      for (int q = 0; q < 6; ++q) kt_prev[q] = h_.stats.t_kernel[q];
    }
    slog_ = StageLog();
  }
  sync();
  if (!live().empty()) throw Error(SPAQR_ERR_CUDA, "internal: rows left after the root");
  for (int i = 0; i < 6; ++i) h_.stats.t_phase[i] = tp[i];
  if (h_.opt.verbose)
    std::fprintf(stderr,
                 "[spaqr] host: waits %.3f s | index %.3f | elim plan %.3f | elim groups %.3f | scale %.3f | step2 "
                 "%.3f | merge %.3f (scale/step2/merge include their waits)\n",
                 ht_[0], ht_[1], ht_[2], ht_[3], ht_[4], ht_[5], ht_[6]);
  if (h_.opt.verbose) {
    std::sort(nt_.begin(), nt_.end(), [](const auto& a, const auto& b) { return a.second > b.second; });
    for (auto& e : nt_) std::fprintf(stderr, "[spaqr] host timer %-28s %8.3f ms\n", e.first.c_str(), 1e3 * e.second);
  }
  h_.stats.launches = launches_;
  h_.stats.syncs = up_.syncs;
  (void)t0;
}

}  // namespace

void run_factor(Handle& h, const spaqr_csr& A, const Analysis& an) {
  // the handle's timeout flag of the tensor-core kernels, cleared for this factorization
  if (!h.d_flag) SPAQR_CUDA(cudaMalloc(&h.d_flag, sizeof(int)));
  SPAQR_CUDA(cudaMemsetAsync(h.d_flag, 0, sizeof(int), h.st));
  double t_run = 0.0;
  const double t0 = now();
  if (h.precision == SPAQR_PREC_MIXED) {
    Factorizer<float> f(h, an);
    f.run(A);
    t_run = now() - t0;
  } else {
    Factorizer<double> f(h, an);
    f.run(A);
    t_run = now() - t0;
  }
  if (h.opt.verbose)
    std::fprintf(stderr, "[spaqr] factor: run %.3f ms, teardown %.3f ms\n", 1e3 * t_run, 1e3 * (now() - t0 - t_run));
  int late = 0;
  SPAQR_CUDA(cudaMemcpyAsync(&late, h.d_flag, sizeof(int), cudaMemcpyDeviceToHost, h.st));
  SPAQR_CUDA(cudaStreamSynchronize(h.st));
  if (late) throw Error(SPAQR_ERR_TIMEOUT, "tensor-core trailing update: MMA completion wait timed out");
}

}  // namespace spaqr
