// A small persistent host thread pool for the independent per-row, per-front
// and per-group loops of the host planning.  parallel_for(n, f) calls
// f(begin, end, worker) on disjoint chunks of [0, n) and returns when all are
// done; small n runs inline on the calling thread.
#pragma once
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace spaqr {

class ThreadPool {
 public:
  static ThreadPool& get() {
    static ThreadPool pool;
    return pool;
  }
  int workers() const { return (int)threads_.size() + 1; }

  template <typename F>
  void parallel_for(int64_t n, F&& f, int64_t min_chunk = 2048) {
    const int nw = workers();
    // one job at a time: a caller that finds the pool busy (another thread's
    // job, or a nested call from inside a job) runs its loop inline
    std::unique_lock<std::mutex> busy(busy_, std::try_to_lock);
    if (n <= min_chunk || nw == 1 || !busy.owns_lock()) {
      f((int64_t)0, n, 0);
      return;
    }
    const int parts = (int)std::min<int64_t>(nw, (n + min_chunk - 1) / min_chunk);
    std::function<void(int)> job = [&](int w) {
      const int64_t b = n * w / parts, e = n * (w + 1) / parts;
      if (b < e) f(b, e, w);
    };
    run(parts, job);
  }

 private:
  std::vector<std::thread> threads_;
  std::mutex mu_, busy_;
  std::condition_variable cv_, done_cv_;
  std::function<void(int)>* job_ = nullptr;
  int parts_ = 0;
  int64_t generation_ = 0;
  std::atomic<int> next_{0}, pending_{0};
  bool stop_ = false;

  ThreadPool() {
    int hw = (int)std::thread::hardware_concurrency();
    const int n = std::max(0, std::min(hw, 16) - 1);
    for (int i = 0; i < n; ++i) threads_.emplace_back([this] { loop(); });
  }
  ~ThreadPool() {
    {
      std::lock_guard<std::mutex> l(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
  }
  void work() {
    for (;;) {
      const int w = next_.fetch_add(1);
      if (w >= parts_) break;
      (*job_)(w);
      if (pending_.fetch_sub(1) == 1) {
        std::lock_guard<std::mutex> l(mu_);
        done_cv_.notify_all();
      }
    }
  }
  void loop() {
    int64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> l(mu_);
        cv_.wait(l, [&] { return stop_ || generation_ != seen; });
        if (stop_) return;
        seen = generation_;
      }
      work();
    }
  }
  void run(int parts, std::function<void(int)>& job) {
    {
      std::lock_guard<std::mutex> l(mu_);
      job_ = &job;
      parts_ = parts;
      next_.store(0);
      pending_.store(parts);
      ++generation_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> l(mu_);
    done_cv_.wait(l, [&] { return pending_.load() == 0; });
  }
};

template <typename F>
inline void parallel_for(int64_t n, F&& f, int64_t min_chunk = 2048) {
  ThreadPool::get().parallel_for(n, std::forward<F>(f), min_chunk);
}

}  // namespace spaqr
