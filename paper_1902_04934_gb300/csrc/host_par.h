// Host-side helper: a loop over [0, n) cut into parts, run by a process-wide pool of worker
// threads (started on first use and kept).  A worker that finishes a job, or is woken ahead of
// one (Pool::wake), keeps polling for the next job for a short while before it sleeps, so a call
// that follows soon after costs no thread wake-up.
#pragma once
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace host_par {

class Pool {
 public:
  static constexpr int kMaxWorkers = 7;
  static constexpr std::chrono::microseconds kSpin{300};   // polling time before a worker sleeps

  static Pool &get() {
    static Pool *p = new Pool;   // never destroyed: its threads live until the process exits
    return *p;
  }

  // Wakes the workers ahead of a job that will follow shortly (they poll for kSpin).
  void wake() {
    if (getpid() != pid_) return;
    {
      std::lock_guard<std::mutex> g(mu_);
      ++wake_;
    }
    cv_work_.notify_all();
  }

  // Runs job(part) for part in [0, parts) on the calling thread and the workers; returns false
  // (nothing run) when the pool is in use by another call or was started in another process.
  // Returns once every part has run and no worker is still inside the job.
  bool run(int parts, const std::function<void(int)> &job) {
    std::unique_lock<std::mutex> busy(busy_, std::try_to_lock);
    if (!busy.owns_lock() || getpid() != pid_) return false;
    {
      std::lock_guard<std::mutex> g(mu_);
      job_ = &job;
      parts_ = parts;
      next_.store(0);
      left_ = parts;
      gen_.fetch_add(1, std::memory_order_release);
    }
    cv_work_.notify_all();
    work();
    std::unique_lock<std::mutex> g(mu_);
    cv_done_.wait(g, [&] { return left_ == 0 && active_ == 0; });
    job_ = nullptr;
    return true;
  }

  int workers() const { return (int)threads_.size(); }

 private:
  Pool() : pid_(getpid()) {
    const int n = std::min(kMaxWorkers, std::max(0, (int)std::thread::hardware_concurrency() - 1));
    for (int i = 0; i < n; ++i) {
      try {
        threads_.emplace_back([this] { loop(); });
      } catch (...) {
        break;
      }
    }
  }

  // Takes parts until none is left; the thread that finishes the last one wakes the caller.  job_
  // and parts_ change only while no thread is in here.
  void work() {
    for (;;) {
      const int i = next_.fetch_add(1);
      if (i >= parts_) return;
      (*job_)(i);
      std::lock_guard<std::mutex> g(mu_);
      if (--left_ == 0) cv_done_.notify_all();
    }
  }

  // Joins the current job if it is still open.
  void join_job(unsigned long long &seen) {
    {
      std::lock_guard<std::mutex> g(mu_);
      seen = gen_.load();
      if (!job_) return;   // that job has finished
      ++active_;
    }
    work();
    std::lock_guard<std::mutex> g(mu_);
    if (--active_ == 0) cv_done_.notify_all();
  }

  void loop() {
    unsigned long long seen = 0, woken = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> g(mu_);
        cv_work_.wait(g, [&] { return gen_.load() != seen || wake_ != woken; });
        woken = wake_;
      }
      // jobs as they come, polling up to kSpin after the last one
      auto last = std::chrono::steady_clock::now();
      while (std::chrono::steady_clock::now() - last < kSpin) {
        if (gen_.load(std::memory_order_acquire) != seen) {
          join_job(seen);
          last = std::chrono::steady_clock::now();
        } else {
          std::this_thread::yield();
        }
      }
    }
  }

  std::mutex busy_, mu_;
  std::condition_variable cv_work_, cv_done_;
  const std::function<void(int)> *job_ = nullptr;
  int parts_ = 0, left_ = 0, active_ = 0;
  std::atomic<int> next_{0};
  std::atomic<unsigned long long> gen_{0};
  unsigned long long wake_ = 0;
  const pid_t pid_;
  std::vector<std::thread> threads_;
};

}  // namespace host_par

// Runs f(part, begin, end) over [0, n) cut into up to max_parts parts of at least min_part items:
// on the worker pool, or on the calling thread alone when the pool is busy.  Returns the number
// of parts (each part index < max_parts).
template <class F>
int parallel_parts(int n, int min_part, int max_parts, F &&f) {
  host_par::Pool &pool = host_par::Pool::get();
  int parts = std::min(max_parts, pool.workers() + 1);
  parts = std::max(1, std::min(parts, n / std::max(1, min_part)));
  auto lo = [&](int t) { return (int)((long long)n * t / parts); };
  if (parts > 1) {
    const std::function<void(int)> job = [&](int t) { f(t, lo(t), lo(t + 1)); };
    if (pool.run(parts, job)) return parts;
  }
  // alone: the same parts in order on this thread
  for (int t = 0; t < parts; ++t) f(t, lo(t), lo(t + 1));
  return parts;
}
