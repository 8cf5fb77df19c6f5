// pool_shim.cpp — test infrastructure: a stress run of the host thread pool
// (pool.hpp), built with ThreadSanitizer by tests/test_host_sanitizers.py and
// run on the CPU.  `callers` threads each submit `jobs` parallel_for jobs of
// 1 to 300 items to one pool of `threads` threads; some items sleep (as the
// copy back's wait for a transfer does), so jobs overlap.  Every item must run
// exactly once, and each call must return only after all its items are done.
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <random>
#include <thread>
#include <vector>

#include "pool.hpp"

namespace {
char g_msg[256];
}

extern "C" const char* pool_message() { return g_msg; }

// Returns 0, or 1000 with a message in pool_message().
extern "C" int pool_stress(unsigned threads, unsigned callers, unsigned jobs, uint64_t seed) {
  dc::Pool pool(threads);
  std::atomic<int> bad{0};
  std::vector<std::thread> cs;
  for (unsigned c = 0; c < callers; c++)
    cs.emplace_back([&, c] {
      std::mt19937_64 rng(seed * 1000 + c);
      for (unsigned j = 0; j < jobs && !bad.load(); j++) {
        const uint64_t n = 1 + rng() % 300;
        const bool slow = rng() % 4 == 0;
        std::vector<std::atomic<uint32_t>> hits(n);
        for (auto& h : hits) h.store(0);
        pool.parallel_for(n, [&](uint64_t i) {
          if (slow && i % 37 == 0) std::this_thread::sleep_for(std::chrono::microseconds(200));
          hits[i].fetch_add(1, std::memory_order_relaxed);
        });
        for (uint64_t i = 0; i < n; i++)
          if (hits[i].load(std::memory_order_relaxed) != 1 && bad.exchange(1) == 0)
            std::snprintf(g_msg, sizeof g_msg, "caller %u job %u item %llu ran %u times", c, j,
                          (unsigned long long)i, hits[i].load());
      }
    });
  for (auto& t : cs) t.join();
  return bad.load() ? 1000 : 0;
}
