// Launch counting and optional per-kernel CUDA-event timing.
//
// Every launcher wraps its launches in a ProfScope.  The launch counter is
// always maintained (library calls are timed with nlaunch = 0: they are not
// this library's kernels); when profiling is enabled (az_profile_begin) the scope
// also records a start/stop event pair on the launching stream and the
// algorithmic bytes of the launch (each input read once, each output written
// once), so that achieved bandwidth = bytes / event time per kernel class.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace az {

void prof_count(int64_t nlaunch);
bool prof_enabled();
void prof_record(const char* name, cudaEvent_t a, cudaEvent_t b, double bytes, int64_t nlaunch);
cudaEvent_t prof_event();

struct ProfScope {
  const char* name;
  double bytes;
  int64_t n;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(const char* nm, double by, cudaStream_t s, int64_t nlaunch = 1) : name(nm), bytes(by), n(nlaunch), st(s) {
    prof_count(nlaunch);
    if (prof_enabled()) { a = prof_event(); b = prof_event(); cudaEventRecord(a, st); }
  }
  // ends the timed region before the scope does
  void close() {
    if (a) { cudaEventRecord(b, st); prof_record(name, a, b, bytes, n); }
    a = nullptr;
  }
  ~ProfScope() { close(); }
};

}  // namespace az
