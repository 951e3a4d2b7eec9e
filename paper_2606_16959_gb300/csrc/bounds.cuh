// Index checks of the HS_DEBUG_BOUNDS build.
//
// Built with -DHS_DEBUG_BOUNDS, every checked global-memory index (a state row,
// a diagonal element, a slot or row-base table entry, a value-table entry, a
// per-term record) is tested against the extent of the array it addresses.  A
// failed test never traps: it counts the failure in a device word of the
// translation unit, records the first failure's site, index and extent, and
// the access goes to element 0 instead (always in bounds), so the kernel runs
// to its end and the context stays usable.  The results of a launch that
// recorded a failure are meaningless; hs_debug_bounds reads and clears the
// words.  In the ordinary build HS_BCHK is the index itself.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace hs {

// Checked sites (reported by hs_debug_bounds as the site number).
enum BoundsSite : int {
  BS_PLAIN_VAL = 1,     // plain apply: diagonal element
  BS_PLAIN_X = 2,       // plain apply: input state row
  BS_SWEEP_STATE = 3,   // tile sweep: state row (load and store)
  BS_SWEEP_VAL = 4,     // tile sweep: diagonal element staged from the values
  BS_SWEEP_SLOT = 5,    // tile sweep: slot table entry
  BS_SWEEP_TAB = 6,     // tile sweep: row-base table entry
  BS_SWEEP_VT = 7,      // tile sweep: value-table entry
  BS_BUILD_VAL = 8,     // factor build: diagonal element written
  BS_BUILD_VT = 9,      // value-table build: entry written
  BS_REG_STATE = 10,    // register sweep: state row (load and store)
  BS_REG_VT = 11,       // register sweep: value-table entry
  BS_REG_TERM = 12,     // register sweep: per-term record
  BS_DIA_VAL = 13,      // DIA SpMV: diagonal element
  BS_DIA_X = 14,        // DIA SpMV: input state row
  BS_BATCH_JOB = 15,    // batched sweep: job descriptor index
};

#ifdef HS_DEBUG_BOUNDS
// Device word of this translation unit: failures, then the first failure's
// site, index and extent.
namespace {
__device__ unsigned long long g_bounds_word[4];
}

__device__ __forceinline__ int64_t bounds_check(int64_t i, int64_t n, int site) {
  if (i >= 0 && i < n) return i;
  if (atomicAdd(&g_bounds_word[0], 1ull) == 0ull) {
    g_bounds_word[1] = static_cast<unsigned long long>(site);
    g_bounds_word[2] = static_cast<unsigned long long>(i);
    g_bounds_word[3] = static_cast<unsigned long long>(n);
  }
  return 0;
}
#define HS_BCHK(i, n, site) (::hs::bounds_check(int64_t(i), int64_t(n), (site)))

// Host side: each translation unit registers a reader of its word.
using BoundsReader = int (*)(uint64_t* out4, bool reset);
void register_bounds_reader(BoundsReader r);
namespace {
int read_bounds_word(uint64_t* out4, bool reset) {
  unsigned long long w[4] = {0, 0, 0, 0};
  if (cudaMemcpyFromSymbol(w, g_bounds_word, sizeof(w)) != cudaSuccess) return -1;
  for (int k = 0; k < 4; ++k) out4[k] = w[k];
  if (reset) {
    const unsigned long long z[4] = {0, 0, 0, 0};
    if (cudaMemcpyToSymbol(g_bounds_word, z, sizeof(z)) != cudaSuccess) return -1;
  }
  return 0;
}
struct BoundsRegistrar {
  BoundsRegistrar() { register_bounds_reader(&read_bounds_word); }
};
BoundsRegistrar g_bounds_registrar;
}  // namespace
#else
#define HS_BCHK(i, n, site) (i)
#endif

}  // namespace hs
