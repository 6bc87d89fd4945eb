// zmc_pool.cpp -- a small pool of host threads for the per-descriptor host work
// (validation and FP64 precompute of the evaluation constants), which is
// independent per descriptor: large tables are cut into ranges that the
// calling thread and the workers take from a shared counter.  The workers are
// created at first use and live until the process exits.
#include <pthread.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "zmc_runtime.h"

namespace zmc {
namespace {

class HostPool {
 public:
  HostPool() {
    const unsigned hw = std::thread::hardware_concurrency();
    const unsigned n = std::min(15u, hw > 1 ? hw - 1 : 0u);
    for (unsigned i = 0; i < n; ++i) workers_.emplace_back([this] { loop(); });
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto &t : workers_) t.join();
  }
  size_t size() const { return workers_.size() + 1; }

  // fn(begin, end) over [0, n) in ranges of `grain`; returns when all are done.
  void run(size_t n, size_t grain, const std::function<void(size_t, size_t)> &fn) {
    std::lock_guard<std::mutex> one(call_mu_);  // one parallel loop at a time
    {
      std::lock_guard<std::mutex> g(mu_);
      fn_ = &fn;
      n_ = n;
      grain_ = grain;
      next_.store(0);
      active_ = workers_.size();
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return active_ == 0; });
    fn_ = nullptr;
  }

 private:
  void work() {
    for (;;) {
      const size_t b = next_.fetch_add(grain_);
      if (b >= n_) return;
      (*fn_)(b, std::min(n_, b + grain_));
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
      }
      work();
      std::lock_guard<std::mutex> g(mu_);
      if (--active_ == 0) done_cv_.notify_all();
    }
  }

  std::vector<std::thread> workers_;
  std::mutex mu_, call_mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(size_t, size_t)> *fn_ = nullptr;
  size_t n_ = 0, grain_ = 1, active_ = 0;
  std::atomic<size_t> next_{0};
  uint64_t gen_ = 0;
  bool stop_ = false;
};

// A child created by fork() has none of the parent's worker threads: from then
// on it runs every loop inline.
std::atomic<bool> g_forked{false};
void on_fork_child() { g_forked.store(true); }

// Created on first use and never destroyed: the workers wait until the process
// exits (no join at exit, where a forked child would have no threads to join).
HostPool &pool() {
  static HostPool *p = [] {
    pthread_atfork(nullptr, nullptr, on_fork_child);
    return new HostPool;
  }();
  return *p;
}

}  // namespace

void host_parallel_for(size_t n, size_t grain, const std::function<void(size_t, size_t)> &fn) {
  if (n <= grain || g_forked.load() || pool().size() == 1) {
    fn(0, n);
    return;
  }
  pool().run(n, grain, fn);
}

}  // namespace zmc
