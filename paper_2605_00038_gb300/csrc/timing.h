// Hooks of the optional kernel timing (lbp_timing_enable / lbp_timing_read).
#pragma once

#include <cuda_runtime.h>

namespace lbp {

constexpr int kTimeBp = 0;
constexpr int kTimeOsd = 1;

// Returns a token when timing is enabled (null otherwise) after recording the
// start event on s; timing_end records the matching stop event.
void *timing_begin(cudaStream_t s);
void timing_end(void *tok, cudaStream_t s, int kind);

// Whether timing is enabled (lbp_timing_enable).
bool timing_on();

}  // namespace lbp
