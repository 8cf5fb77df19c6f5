// pool.hpp — a small fixed thread pool for the host-side marshal and scatter.
// parallel_for(n, fn) runs fn(i) for i in [0, n) on the workers and the
// calling thread, and returns when every item is done.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace dc {

class Pool {
 public:
  explicit Pool(unsigned nthreads) {
    if (nthreads == 0) nthreads = 1;
    for (unsigned i = 1; i < nthreads; i++) workers_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> g(m_);
      stop_ = true;
      gen_++;
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
  }
  unsigned size() const { return (unsigned)workers_.size() + 1; }

  void parallel_for(uint64_t n, const std::function<void(uint64_t)>& fn) {
    if (n == 0) return;
    if (workers_.empty() || n == 1) {
      for (uint64_t i = 0; i < n; i++) fn(i);
      return;
    }
    std::lock_guard<std::mutex> one_job(job_);  // callers on several threads take turns
    {
      std::lock_guard<std::mutex> g(m_);
      fn_ = &fn;
      n_ = n;
      next_.store(0);
      active_ = (unsigned)workers_.size();
      gen_++;
    }
    cv_.notify_all();
    drain();
    std::unique_lock<std::mutex> lk(m_);
    done_cv_.wait(lk, [this] { return active_ == 0; });
    fn_ = nullptr;
  }

 private:
  void drain() {
    for (;;) {
      uint64_t i = next_.fetch_add(1);
      if (i >= n_) break;
      (*fn_)(i);
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
        if (stop_) return;
      }
      drain();
      {
        std::lock_guard<std::mutex> g(m_);
        if (--active_ == 0) done_cv_.notify_all();
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
  unsigned active_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

}  // namespace dc
