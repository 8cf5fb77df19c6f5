// debug.cpp — switches read from the environment for testing and debugging.
//
//   DC_DEBUG=1             every plan runs with DC_PLAN_VERIFY (the relocation
//                          checks each slot's old value and each computed offset
//                          on the device).
//   DC_FAULT_HOST_ALLOC=1  every pinned host allocation of the library fails as
//                          if the host were out of page-locked memory, so callers
//                          can test their handling of DC_ENOMEM without a real
//                          shortage (and without touching a GPU).
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

cudaError_t host_alloc(void** ptr, size_t bytes, unsigned int flags) {
  if (env_on("DC_FAULT_HOST_ALLOC")) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaHostAlloc(ptr, bytes, flags);
}

}  // namespace dc
