// trace.hpp — tracing of the host side of every call.
//
// A Trace object opens an NVTX range (seen by ncu --nvtx and other NVTX
// tools; free when none is attached) and, when the environment has
// DC_TRACE=1, writes the host wall time between its construction and its
// destruction to stderr as one line: "dc_trace <call> <phase> <us>".  Phases
// that only enqueue device work measure the enqueue; phases that wait on the
// device (dc_sync, the round trip's final wait) include the device time.
#pragma once

#include <chrono>

namespace dc {

bool trace_on();  // DC_TRACE=1, read once

class Trace {
 public:
  Trace(const char* call, const char* phase);
  ~Trace();
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;

 private:
  const char* call_;
  const char* phase_;
  std::chrono::steady_clock::time_point t0_;
};

}  // namespace dc
