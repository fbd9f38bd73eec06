// Per-stage CUDA-event tracing of the low-rank drivers (host side).
#pragma once

#include <cuda_runtime.h>

namespace bsrht {

// Starts a new trace for the calling host thread if tracing is enabled.
void trace_begin(cudaStream_t s);
// Marks the end of stage `name` (static storage) on stream s.
void trace_mark(cudaStream_t s, const char* name);

}  // namespace bsrht
