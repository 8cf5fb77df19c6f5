// pool.hpp — a small fixed thread pool for the host-side marshal and scatter.
// parallel_for(n, fn) runs fn(i) for i in [0, n) on the workers and the
// calling thread, and returns when every item is done.  Several callers (the
// server's slots) may have jobs in flight at once: each caller works on its
// own job, and the workers share themselves out over every job that still has
// items, taking a few items of one job and then moving on to the next in turn.
// So a small job is not queued behind a large one, and a job whose items wait
// (the copy back's, for its chunks' transfers) holds only the workers that run
// those items.
//
// Waking sleeping threads costs tens of microseconds on a virtual machine, so
// workers spin for a while (SPIN rounds of a yield to the scheduler) after
// their last item before they sleep, and a caller spins the same way for its
// job's items to finish: back-to-back jobs (a transfer's chunks) then start
// within a few microseconds.  The spin yields rather than pauses because the
// server's slot threads share the cores with the workers: a pausing worker
// holds a core a slot thread is waiting for (DC_POOL_YIELD=0 builds the pause
// form).  Jobs of one or two items run on the calling thread alone.
#pragma once

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#ifndef DC_POOL_YIELD
#define DC_POOL_YIELD 1
#endif
#if DC_POOL_YIELD
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
  static constexpr unsigned SPIN = DC_POOL_SPIN;  // spin rounds before sleeping
  static constexpr uint64_t TAKE = 2;              // items a worker takes from one job before moving on

  explicit Pool(unsigned nthreads) {
    if (nthreads == 0) nthreads = 1;
    for (unsigned i = 1; i < nthreads; i++) workers_.emplace_back([this, i] { loop(i); });
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
    Job job(&fn, n);
    {
      std::lock_guard<std::mutex> g(m_);
      jobs_.push_back(&job);
      gen_.fetch_add(1, std::memory_order_release);  // wakes spinning workers
    }
    cv_.notify_all();
    while (job.run_one()) {
    }
    for (unsigned k = 0; k < SPIN && job.done.load(std::memory_order_acquire) != n; k++) DC_POOL_PAUSE();
    if (job.done.load(std::memory_order_acquire) != n) {
      std::unique_lock<std::mutex> lk(m_);
      done_cv_.wait(lk, [&] { return job.done.load(std::memory_order_acquire) == n; });
    }
    {  // no worker finds the job any more; one that holds it has found no item left
      std::lock_guard<std::mutex> g(m_);
      jobs_.erase(std::find(jobs_.begin(), jobs_.end(), &job));
    }
    while (job.users.load(std::memory_order_acquire)) DC_POOL_PAUSE();
  }

 private:
  struct Job {
    Job(const std::function<void(uint64_t)>* f, uint64_t count) : fn(f), n(count) {}
    const std::function<void(uint64_t)>* fn;
    const uint64_t n;
    std::atomic<uint64_t> next{0}, done{0};
    std::atomic<unsigned> users{0};  // workers holding a pointer to the job
    bool has_items() const { return next.load(std::memory_order_relaxed) < n; }
    // Runs one item if any is left; false once every item has been taken.
    bool run_one() {
      const uint64_t i = next.fetch_add(1, std::memory_order_relaxed);
      if (i >= n) return false;
      (*fn)(i);
      done.fetch_add(1, std::memory_order_acq_rel);
      return true;
    }
  };

  // A job with items left, starting the search at `from` (worker i starts at a
  // different place each time, so the workers spread over the jobs); the
  // caller holds m_.  Marks the job as used.
  Job* pick(uint64_t from) {
    const size_t nj = jobs_.size();
    for (size_t k = 0; k < nj; k++) {
      Job* j = jobs_[(from + k) % nj];
      if (j->has_items()) {
        j->users.fetch_add(1, std::memory_order_acq_rel);
        return j;
      }
    }
    return nullptr;
  }

  void loop(unsigned id) {
    uint64_t seen = 0, turn = id;
    for (;;) {
      Job* j = nullptr;
      {
        std::unique_lock<std::mutex> lk(m_);
        j = pick(turn++);
        if (!j) {
          if (stop_) return;
          seen = gen_.load(std::memory_order_acquire);
          lk.unlock();
          for (unsigned k = 0; k < SPIN && gen_.load(std::memory_order_acquire) == seen; k++) DC_POOL_PAUSE();
          lk.lock();
          if (!stop_ && gen_.load(std::memory_order_acquire) == seen && !(j = pick(turn++)))
            cv_.wait(lk, [&] { return stop_ || gen_.load(std::memory_order_acquire) != seen; });
          if (!j) continue;
        }
      }
      bool finished_last = false;
      for (uint64_t t = 0; t < TAKE; t++) {
        const uint64_t i = j->next.fetch_add(1, std::memory_order_relaxed);
        if (i >= j->n) break;
        (*j->fn)(i);
        if (j->done.fetch_add(1, std::memory_order_acq_rel) + 1 == j->n) finished_last = true;
      }
      if (finished_last) {  // the caller may be asleep on its job
        { std::lock_guard<std::mutex> g(m_); }
        done_cv_.notify_all();
      }
      j->users.fetch_sub(1, std::memory_order_acq_rel);
    }
  }

  std::vector<std::thread> workers_;
  std::mutex m_;
  std::condition_variable cv_, done_cv_;
  std::vector<Job*> jobs_;  // jobs in flight, oldest first
  std::atomic<uint64_t> gen_{0};
  bool stop_ = false;
};

}  // namespace dc
