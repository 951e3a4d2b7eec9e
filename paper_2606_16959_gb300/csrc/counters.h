// Process-wide count of the kernels libhs launches (exported as
// hs_kernel_launches).  Launches enqueued while this thread captures a CUDA
// graph are tallied for the graph instead, and every replay of the graph adds
// that tally.
#pragma once

#include <cstdint>

namespace hs {
void note_launches(uint64_t n = 1);
void begin_capture_count();
uint64_t end_capture_count();
}  // namespace hs
