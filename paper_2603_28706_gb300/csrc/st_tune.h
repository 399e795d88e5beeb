// Launch-shape autotuner (internal, not part of the ABI).
//
// The first launch of a tuned kernel with a new key (kernel, dimension,
// degree, precision and the size of the launch) times every candidate launch
// shape on the real arguments: one warm-up run, then three timed runs per
// candidate with CUDA events on the launching stream.  The fastest shape is
// kept in a process-wide table and used for every later launch with that key.
// Every candidate computes the same values (the tuned kernels give each
// cell or patch to exactly one thread block and write it with plain stores),
// so the choice changes only the time.  No trials run while the stream is
// being captured into a CUDA graph (the first candidate, the untuned default,
// is used then), nor when the environment sets ST_AUTOTUNE=0.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>

namespace st {

struct LaunchShape {
  int threads;
  long grid;
};

// Index of the chosen candidate; run(i) enqueues candidate i on `s` and
// returns its launch status; label(i) describes candidate i for the report.
int tune_pick(const std::string& key, int ncand, const std::function<cudaError_t(int)>& run,
              const std::function<std::string(int)>& label, cudaStream_t s);

}  // namespace st
