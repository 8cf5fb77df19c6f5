// pool.hpp — a small fixed thread pool for the host-side marshal and scatter.
// parallel_for(n, fn) runs fn(i) for i in [0, n) on the workers and the
// calling thread, and returns when every item is done.  One job runs at a
// time (callers on several threads take turns); a job whose items wait (the
// copy back's, for its chunks' transfers) holds the pool meanwhile, so such
// waits are kept short: the transfer runs ahead of the copying.
//
// Waking sleeping threads costs tens of microseconds on a virtual machine, so
// workers spin for a short while (SPIN rounds of a pause instruction) after a
// job before they sleep, and the caller spins the same way for the workers to
// finish: back-to-back jobs (a transfer's chunks) then start within a few
// microseconds.  Jobs of one or two items run on the calling thread alone.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#if defined(DC_POOL_YIELD) && DC_POOL_YIELD
#define DC_POOL_PAUSE() std::this_thread::yield()
#elif defined(__x86_64__) || defined(__i386__)
#include <immintrin.h>
#define DC_POOL_PAUSE() _mm_pause()
#else
#define DC_POOL_PAUSE() std::this_thread::yield()
#endif

namespace dc {

class Pool {
 public:
#ifndef DC_POOL_SPIN
#define DC_POOL_SPIN 4096
#endif
  static constexpr unsigned SPIN = DC_POOL_SPIN;  // pause rounds before sleeping (tens of microseconds)

  explicit Pool(unsigned nthreads) {
    if (nthreads == 0) nthreads = 1;
    for (unsigned i = 1; i < nthreads; i++) workers_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> g(m_);
      stop_ = true;
      gen_.fetch_add(1, std::memory_order_release);
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
  }
  unsigned size() const { return (unsigned)workers_.size() + 1; }

  void parallel_for(uint64_t n, const std::function<void(uint64_t)>& fn) {
    if (n == 0) return;
    if (workers_.empty() || n <= 2) {
      for (uint64_t i = 0; i < n; i++) fn(i);
      return;
    }
    std::lock_guard<std::mutex> one_job(job_);  // callers on several threads take turns
    fn_ = &fn;
    n_ = n;
    next_.store(0, std::memory_order_relaxed);
    active_.store((unsigned)workers_.size(), std::memory_order_relaxed);
    gen_.fetch_add(1, std::memory_order_release);  // publishes the job to spinning workers
    {
      std::lock_guard<std::mutex> g(m_);  // a worker between its check and its sleep holds m_
    }
    cv_.notify_all();
    drain();
    for (unsigned k = 0; k < SPIN && active_.load(std::memory_order_acquire); k++) DC_POOL_PAUSE();
    if (active_.load(std::memory_order_acquire)) {
      std::unique_lock<std::mutex> lk(m_);
      done_cv_.wait(lk, [this] { return active_.load(std::memory_order_acquire) == 0; });
    }
    fn_ = nullptr;
  }

 private:
  void drain() {
    for (;;) {
      const uint64_t i = next_.fetch_add(1, std::memory_order_relaxed);
      if (i >= n_) break;
      (*fn_)(i);
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      for (unsigned k = 0; k < SPIN && gen_.load(std::memory_order_acquire) == seen; k++) DC_POOL_PAUSE();
      if (gen_.load(std::memory_order_acquire) == seen) {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen; });
      }
      seen = gen_.load(std::memory_order_acquire);
      if (stop_) return;
      drain();
      if (active_.fetch_sub(1, std::memory_order_acq_rel) == 1) {
        { std::lock_guard<std::mutex> g(m_); }
        done_cv_.notify_all();
      }
    }
  }

  std::vector<std::thread> workers_;
  std::mutex job_;
  std::mutex m_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(uint64_t)>* fn_ = nullptr;
  uint64_t n_ = 0;
  std::atomic<uint64_t> next_{0};
  std::atomic<unsigned> active_{0};
  std::atomic<uint64_t> gen_{0};
  bool stop_ = false;
};

}  // namespace dc
