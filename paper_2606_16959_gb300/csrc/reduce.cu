// FP64 reductions for the state-fidelity metric (evaluation section,
// Metrics): <a|b>, |a|^2 and |b|^2 accumulated in double precision whatever
// the storage precision, with warp shuffles inside a block and a fixed
// two-pass tree across blocks (deterministic: same bits on every call).
#include <cuda_runtime.h>

#include <cstdint>

#include "counters.h"
#include "hs_internal.h"

namespace hs {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 152 * 4;  // fixed grid: a multiple of the SM count

struct Acc4 {
  double re, im, na, nb;
};

__device__ __forceinline__ Acc4 warp_sum(Acc4 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
    v.na += __shfl_xor_sync(0xffffffffu, v.na, o);
    v.nb += __shfl_xor_sync(0xffffffffu, v.nb, o);
  }
  return v;
}

__device__ __forceinline__ Acc4 block_sum(Acc4 v) {
  __shared__ Acc4 part[kRedThreads / 32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) part[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < kRedThreads / 32) ? part[l] : Acc4{0, 0, 0, 0};
    v = warp_sum(v);
  }
  return v;
}

__device__ __forceinline__ double2 ld2(const float2* p, int64_t i) {
  float2 v = p[i];
  return make_double2(v.x, v.y);
}
__device__ __forceinline__ double2 ld2(const double2* p, int64_t i) { return p[i]; }

template <typename T2>
__global__ void __launch_bounds__(kRedThreads) inner_partial(const T2* __restrict__ a, const T2* __restrict__ b,
                                                             int64_t N, Acc4* __restrict__ partial) {
  Acc4 s{0, 0, 0, 0};
  for (int64_t i = int64_t(blockIdx.x) * kRedThreads + threadIdx.x; i < N; i += int64_t(gridDim.x) * kRedThreads) {
    const double2 x = ld2(a, i), y = ld2(b, i);
    s.re = fma(x.x, y.x, fma(x.y, y.y, s.re));
    s.im = fma(x.x, y.y, fma(-x.y, y.x, s.im));
    s.na = fma(x.x, x.x, fma(x.y, x.y, s.na));
    s.nb = fma(y.x, y.x, fma(y.y, y.y, s.nb));
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads) inner_final(const Acc4* __restrict__ partial, int n, double* out) {
  Acc4 s{0, 0, 0, 0};
  for (int i = threadIdx.x; i < n; i += kRedThreads) {
    s.re += partial[i].re;
    s.im += partial[i].im;
    s.na += partial[i].na;
    s.nb += partial[i].nb;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) {
    out[0] = s.re;
    out[1] = s.im;
    out[2] = s.na;
    out[3] = s.nb;
  }
}

}  // namespace

size_t inner_scratch_bytes() { return sizeof(Acc4) * kRedBlocks; }

// out4 = {Re<a|b>, Im<a|b>, |a|^2, |b|^2}; `scratch` holds inner_scratch_bytes().
cudaError_t launch_inner_scratch(const void* a, const void* b, int64_t N, hs_dtype dt, double* d_out4, void* scratch,
                                 cudaStream_t s) {
  int blocks = int((N + kRedThreads - 1) / kRedThreads);
  if (blocks > kRedBlocks) blocks = kRedBlocks;
  if (blocks < 1) blocks = 1;
  Acc4* part = reinterpret_cast<Acc4*>(scratch);
  if (dt == HS_C64)
    inner_partial<float2><<<blocks, kRedThreads, 0, s>>>((const float2*)a, (const float2*)b, N, part);
  else
    inner_partial<double2><<<blocks, kRedThreads, 0, s>>>((const double2*)a, (const double2*)b, N, part);
  inner_final<<<1, kRedThreads, 0, s>>>(part, blocks, d_out4);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_inner(const void* a, const void* b, int64_t N, hs_dtype dt, double* d_out4, cudaStream_t s) {
  void* scratch = nullptr;
  cudaError_t e = pool_malloc(&scratch, inner_scratch_bytes(), s);
  if (e != cudaSuccess) return e;
  e = launch_inner_scratch(a, b, N, dt, d_out4, scratch, s);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace hs
