// Batched FP64 inner products that allocate no device memory.
//
// Some callers cannot allocate: a serving loop that has reserved all of the
// device memory for resident states and factors (an allocation can then fail,
// or stall behind other work), or a host application whose device memory is
// owned by its own allocator and which hands the library only buffers it has
// already allocated.  hs_inner_batch_noalloc serves them: it computes the same
// reduction as hs_inner_device, for several state pairs at once, but keeps its
// per-block partial sums in the file-scope array below instead of a
// stream-ordered allocation.  The paper has no counterpart of this call.
//
// The array is a fixed 152 KiB that every GPU loading the library holds until
// the process exits.  In host code `g_noalloc_partials` only names a host-side
// stand-in, not a device address: every call looks up its device address on
// the current device with cudaGetSymbolAddress (a host-side lookup, no stream
// work), so a context that was torn down and created again never sees a stale
// address.  The first call on a device also loads the module there; make it
// before any stream capture.  All calls share the array and it keeps the
// contents of the last call; every partial sum a call reads was written
// earlier in that same call, so nothing needs clearing, but calls that overlap
// on the GPU (for example on two streams) race on it.
#include <cuda_runtime.h>

#include <string>

#include "counters.h"
#include "hs_internal.h"

namespace hs {
int report_error(int code, const std::string& msg);
}

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaBlocksPerState = 152 * 4;              // the per-state grid of hs_inner_device
constexpr int kNaMaxPartials = 8 * kNaBlocksPerState;   // 4864 partial sums of 32 bytes

struct NaAcc {
  double re, im, na, nb;
};

static __device__ __align__(256) NaAcc g_noalloc_partials[kNaMaxPartials];

__device__ __forceinline__ NaAcc na_warp_sum(NaAcc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
    v.na += __shfl_xor_sync(0xffffffffu, v.na, o);
    v.nb += __shfl_xor_sync(0xffffffffu, v.nb, o);
  }
  return v;
}

__device__ __forceinline__ NaAcc na_block_sum(NaAcc v) {
  __shared__ NaAcc part[kNaThreads / 32];
  v = na_warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) part[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < kNaThreads / 32) ? part[l] : NaAcc{0, 0, 0, 0};
    v = na_warp_sum(v);
  }
  return v;
}

__device__ __forceinline__ double2 na_ld(const float2* p, int64_t i) {
  const float2 v = p[i];
  return make_double2(v.x, v.y);
}
__device__ __forceinline__ double2 na_ld(const double2* p, int64_t i) { return p[i]; }

// blockIdx.y = state pair; partial sums land at partials[state * blocks + blockIdx.x].
template <typename T2>
__global__ void __launch_bounds__(kNaThreads) na_partial(const T2* __restrict__ a, const T2* __restrict__ b,
                                                         int64_t N, NaAcc* partials) {
  const T2* pa = a + int64_t(blockIdx.y) * N;
  const T2* pb = b + int64_t(blockIdx.y) * N;
  NaAcc s{0, 0, 0, 0};
  for (int64_t i = int64_t(blockIdx.x) * kNaThreads + threadIdx.x; i < N; i += int64_t(gridDim.x) * kNaThreads) {
    const double2 x = na_ld(pa, i), y = na_ld(pb, i);
    s.re = fma(x.x, y.x, fma(x.y, y.y, s.re));
    s.im = fma(x.x, y.y, fma(-x.y, y.x, s.im));
    s.na = fma(x.x, x.x, fma(x.y, x.y, s.na));
    s.nb = fma(y.x, y.x, fma(y.y, y.y, s.nb));
  }
  s = na_block_sum(s);
  if (threadIdx.x == 0) partials[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

// One block per state pair: reduce its `blocks` partial sums into out[4 * state ..].
__global__ void __launch_bounds__(kNaThreads) na_final(const NaAcc* partials, int blocks, double* out) {
  const NaAcc* p = partials + int64_t(blockIdx.x) * blocks;
  NaAcc s{0, 0, 0, 0};
  for (int i = threadIdx.x; i < blocks; i += kNaThreads) {
    s.re += p[i].re;
    s.im += p[i].im;
    s.na += p[i].na;
    s.nb += p[i].nb;
  }
  s = na_block_sum(s);
  if (threadIdx.x == 0) {
    double* o = out + 4 * int64_t(blockIdx.x);
    o[0] = s.re;
    o[1] = s.im;
    o[2] = s.na;
    o[3] = s.nb;
  }
}

// Device address of g_noalloc_partials on the current device, looked up on
// every call.
cudaError_t noalloc_partials(NaAcc** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
  if (e != cudaSuccess) return e;
  *out = static_cast<NaAcc*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" int hs_inner_batch_noalloc(const void* a, const void* b, int n_qubits, int n_states, hs_dtype dtype,
                                      double* out_device, void* cuda_stream) {
  if (!a || !b || !out_device) return hs::report_error(HS_EINVAL, "null buffer");
  if (dtype != HS_C64 && dtype != HS_C128) return hs::report_error(HS_EDTYPE, "dtype must be HS_C64 or HS_C128");
  if (n_qubits < 1 || n_qubits > HS_MAX_QUBITS) return hs::report_error(HS_EINVAL, "n_qubits out of range");
  if (n_states < 1) return hs::report_error(HS_EINVAL, "n_states must be >= 1");
  const int64_t N = int64_t(1) << n_qubits;
  int64_t blocks = (N + kNaThreads - 1) / kNaThreads;
  if (blocks > kNaBlocksPerState) blocks = kNaBlocksPerState;
  if (int64_t(n_states) * blocks > kNaMaxPartials)
    return hs::report_error(HS_EINVAL, "n_states * " + std::to_string(blocks) +
                                           " partial sums exceed the static scratch of " +
                                           std::to_string(kNaMaxPartials) + " (at most " +
                                           std::to_string(kNaMaxPartials / blocks) + " states of this size per call)");
  NaAcc* partials = nullptr;
  cudaError_t e = noalloc_partials(&partials);
  if (e != cudaSuccess)
    return hs::report_error(HS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const dim3 grid{static_cast<unsigned>(blocks), static_cast<unsigned>(n_states), 1u};
  if (dtype == HS_C64)
    na_partial<float2><<<grid, kNaThreads, 0, s>>>((const float2*)a, (const float2*)b, N, partials);
  else
    na_partial<double2><<<grid, kNaThreads, 0, s>>>((const double2*)a, (const double2*)b, N, partials);
  na_final<<<n_states, kNaThreads, 0, s>>>(partials, int(blocks), out_device);
  e = cudaGetLastError();
  if (e != cudaSuccess) return hs::report_error(HS_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  hs::note_launches(2);
  return HS_OK;
}
