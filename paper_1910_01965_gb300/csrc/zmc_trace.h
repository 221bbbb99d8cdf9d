// zmc_trace.h — host-side tracing of the library: log levels and NVTX ranges.
//
// ZMC_LOG (environment, read once per process) sets what goes to stderr:
//   0  nothing (default)
//   1  every failed call's message
//   2  plus one line per scan (tile plan, chunks), batch and served request
//   3  plus one line per chunk launch and per server step
// NVTX ranges (NVTX3, header only: free unless a profiler is attached) mark
// each scan, each chunk, each batch run and each server step, so that an
// Nsight timeline shows the library's work by name.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <cstdlib>

#include <nvtx3/nvToolsExt.h>

namespace zmc {

inline int log_level() {
  static const int level = [] {
    const char* v = std::getenv("ZMC_LOG");
    const int l = v ? std::atoi(v) : 0;
    return l < 0 ? 0 : (l > 3 ? 3 : l);
  }();
  return level;
}

inline void log_msg(int level, const char* fmt, ...) {
  if (level > log_level()) return;
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  std::fprintf(stderr, "[zmc:%d] %s\n", level, buf);
}

// One NVTX range for the lifetime of the object.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace zmc
