// debug.cpp — switches read from the environment for testing and debugging.
//
//   DC_DEBUG=1             every plan runs with DC_PLAN_VERIFY (the relocation
//                          checks each slot's old value and each computed offset
//                          on the device).
//   DC_FAULT_HOST_ALLOC=1  every pinned host allocation of the library fails as
//                          if the host were out of page-locked memory, so callers
//                          can test their handling of DC_ENOMEM without a real
//                          shortage (and without touching a GPU).
//   DC_WAIT_LIMIT=N        the first wait of each pipeline step of the bulk-copy
//                          kernels (relocation, leaf update, fused launch) gives
//                          up after N try_wait rounds (0: without trying) instead
//                          of about a second, so a test can make a wait run out:
//                          the kernel records DC_ETIMEOUT, still waits (at the
//                          full limit) for the copies it has in flight, and
//                          returns.  Nothing traps or faults.
#include <cstdlib>
#include <cstring>

#include "internal.hpp"

namespace dc {

namespace {
bool env_on(const char* name) {
  const char* v = std::getenv(name);
  return v && *v && std::strcmp(v, "0") != 0;
}
}  // namespace

bool debug_on() { return env_on("DC_DEBUG"); }

uint32_t first_wait_limit() {
  const char* v = std::getenv("DC_WAIT_LIMIT");
  if (!v || !*v) return WAIT_LIMIT;
  char* end = nullptr;
  const unsigned long long n = std::strtoull(v, &end, 10);
  if (end == v || *end) return WAIT_LIMIT;  // not a number: the default
  return n < WAIT_LIMIT ? (uint32_t)n : WAIT_LIMIT;
}

cudaError_t host_alloc(void** ptr, size_t bytes, unsigned int flags) {
  if (env_on("DC_FAULT_HOST_ALLOC")) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaHostAlloc(ptr, bytes, flags);
}

}  // namespace dc
