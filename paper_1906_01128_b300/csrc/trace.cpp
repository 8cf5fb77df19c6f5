// trace.cpp — NVTX ranges and DC_TRACE phase timings (trace.hpp).
#include "trace.hpp"

#include <nvtx3/nvToolsExt.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>

namespace dc {

bool trace_on() {
  static const bool on = [] {
    const char* v = std::getenv("DC_TRACE");
    return v && std::strcmp(v, "0") != 0 && *v;
  }();
  return on;
}

Trace::Trace(const char* call, const char* phase) : call_(call), phase_(phase) {
  nvtxRangePushA(phase);
  if (trace_on()) t0_ = std::chrono::steady_clock::now();
}

Trace::~Trace() {
  nvtxRangePop();
  if (trace_on()) {
    const double us =
        std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0_).count();
    std::fprintf(stderr, "dc_trace %s %s %.1f\n", call_, phase_, us);
  }
}

}  // namespace dc
