// Single-factor Taylor mode: the paper's original pipeline (Alg. 3).
//
//   H as a Pauli sum -> H in the compact diagonal layout (Eq. 6), zero
//   diagonals dropped (the numeric counts of Tab. 3);
//   r from the diagonal budget (Eq. 5, adaptive timestep flowchart, Sec. 3.1);
//   U = exp(-i H t/r) by the truncated Taylor series of Alg. 2, whose products
//   are diagonal-pair SpGEMMs (Sec. 3.3);
//   psi <- U^r psi by repeated diagonal-times-vector products (Alg. 1).
//
// GPU layout.  A matrix keeps its diagonals back to back in one device
// buffer, each starting on a 128-byte boundary, plus a small device table of
// (offset, row base) pairs: the value of row i on diagonal k sits at element
// rowbase[k] + i, rowbase[k] = start[k] + min(0, d_k).  Element-parallel
// kernels (H from terms, SpGEMM, combine, statistics) walk a task table of
// (diagonal, first element) per 256-thread block, so every warp streams a
// contiguous run of one diagonal (and, in the SpGEMM, of its contributing
// diagonals).  The SpMV gives each thread one row and a few states, streaming
// every diagonal once per launch.  Host code decides structure (which
// diagonals a product or a sum can reach, which to drop, when the Taylor loop
// stops) from per-diagonal statistics reduced on the device in a fixed order,
// so results do not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <iterator>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/hs_dia.h"
#include "bounds.cuh"
#include "counters.h"
#include "hs_internal.h"

struct hs_dia {
  int n_qubits = 0;
  int64_t N = 0;
  hs_dtype dtype = HS_C128;
  std::vector<int64_t> offs;   // canonical order
  std::vector<int64_t> start;  // element index of element 0 of each diagonal (padded)
  int64_t total = 0;           // allocated elements
  int64_t nnz = -1;
  void* d_vals = nullptr;
  int64_t* d_meta = nullptr;   // [offs(D), rowbase(D)]
  int device = 0;
};

namespace hs {
int report_error(int code, const std::string& msg);
}

namespace {

using hs::pool_malloc;
using hs::report_error;

constexpr int kThreads = 256;               // elements per task block
constexpr int64_t kAlignElems = 8;          // 128 B for complex128, 64 B for complex64
constexpr int kMaxCandidates = 65536;       // structural diagonals of H from terms
constexpr double kDropRel = 1.0 / 70368744177664.0;  // 2^-46

int cuda_err(cudaError_t e, const char* what) {
  return report_error(e == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA,
                      std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

bool canonical_before(int64_t a, int64_t b) {
  const int64_t aa = a < 0 ? -a : a, bb = b < 0 ? -b : b;
  return aa != bb ? aa < bb : a < b;
}

int64_t iabs(int64_t v) { return v < 0 ? -v : v; }

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 ld(const double2* p, int64_t i) { return p[i]; }
__device__ __forceinline__ double2 ld(const float2* p, int64_t i) {
  const float2 v = p[i];
  return make_double2(v.x, v.y);
}
__device__ __forceinline__ void st(double2* p, int64_t i, double2 v) { p[i] = v; }
__device__ __forceinline__ void st(float2* p, int64_t i, double2 v) {
  p[i] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
}

struct Stat {
  double mx, s2;
  long long nz;
};

__device__ __forceinline__ Stat stat_merge(Stat a, Stat b) {
  return Stat{fmax(a.mx, b.mx), a.s2 + b.s2, a.nz + b.nz};
}

__device__ __forceinline__ Stat block_stat(Stat v) {
  __shared__ Stat part[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Stat w{__shfl_xor_sync(0xffffffffu, v.mx, o), __shfl_xor_sync(0xffffffffu, v.s2, o),
           __shfl_xor_sync(0xffffffffu, v.nz, o)};
    v = stat_merge(v, w);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < kThreads / 32 ? part[lane] : Stat{0.0, 0.0, 0};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Stat w{__shfl_xor_sync(0xffffffffu, v.mx, o), __shfl_xor_sync(0xffffffffu, v.s2, o),
             __shfl_xor_sync(0xffffffffu, v.nz, o)};
      v = stat_merge(v, w);
    }
  }
  return v;
}

__device__ __forceinline__ Stat stat_of(double2 v) {
  return Stat{hypot(v.x, v.y), fma(v.x, v.x, v.y * v.y), (v.x != 0.0 || v.y != 0.0) ? 1ll : 0ll};
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// H entries: row i, column c = i + d, u = i xor c; the terms with x mask u add
// c_t i^{y_t} (-1)^{popcount(z_t & c)} in input order.
struct TermsArgs {
  double2* vals;
  const int64_t* offs;
  const int64_t* start;
  const int2* task;
  const uint64_t* masks;  // distinct x masks, ascending
  const int* mrange;      // [n_masks + 1]: terms of mask m are [mrange[m], mrange[m+1])
  const uint64_t* tz;
  const double* tc;
  const int* ty;
  int n_masks;
  int64_t N;
  Stat* partial;
};

__global__ void __launch_bounds__(kThreads) terms_kernel(TermsArgs a) {
  const int2 tk = a.task[blockIdx.x];
  const int64_t d = a.offs[tk.x];
  const int64_t L = a.N - (d < 0 ? -d : d);
  const int64_t j = int64_t(tk.y) + threadIdx.x;
  Stat s{0.0, 0.0, 0};
  if (j < L) {
    const int64_t i = j - (d < 0 ? d : 0);
    const uint64_t c = uint64_t(i + d);
    const uint64_t u = uint64_t(i) ^ c;
    int lo = 0, hi = a.n_masks;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (a.masks[mid] < u) lo = mid + 1;
      else hi = mid;
    }
    double2 acc = make_double2(0.0, 0.0);
    if (lo < a.n_masks && a.masks[lo] == u) {
      for (int t = a.mrange[lo]; t < a.mrange[lo + 1]; ++t) {
        const int ph = (a.ty[t] + 2 * (__popcll(a.tz[t] & c) & 1)) & 3;
        const double cc = a.tc[t];
        switch (ph) {
          case 0: acc.x += cc; break;
          case 1: acc.y += cc; break;
          case 2: acc.x += -cc; break;
          default: acc.y += -cc; break;
        }
      }
    }
    a.vals[a.start[tk.x] + j] = acc;
    s = stat_of(acc);
  }
  s = block_stat(s);
  if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
}

// Statistics of an existing matrix (per task block).
template <typename T2>
__global__ void __launch_bounds__(kThreads) stat_kernel(const T2* vals, const int64_t* offs, const int64_t* start,
                                                        const int2* task, int64_t N, Stat* partial) {
  const int2 tk = task[blockIdx.x];
  const int64_t d = offs[tk.x];
  const int64_t L = N - (d < 0 ? -d : d);
  const int64_t j = int64_t(tk.y) + threadIdx.x;
  Stat s{0.0, 0.0, 0};
  if (j < L) s = stat_of(ld(vals, start[tk.x] + j));
  s = block_stat(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Per-diagonal reduction of the block partials, in block order.
__global__ void __launch_bounds__(kThreads) stat_final(const Stat* partial, const int* block0, Stat* out) {
  const int k = blockIdx.x;
  Stat s{0.0, 0.0, 0};
  for (int b = block0[k] + threadIdx.x; b < block0[k + 1]; b += kThreads) s = stat_merge(s, partial[b]);
  s = block_stat(s);
  if (threadIdx.x == 0) out[k] = s;
}

// One pair of diagonals contributing to a result diagonal: rows [lo, hi),
// A value at a_rb + i, B value at b_rb + i (B's row base already shifted by da).
struct Pair {
  int64_t a_rb, b_rb, lo, hi;
};

struct GemmArgs {
  const double2* A;
  const double2* B;
  double2* C;
  const int64_t* c_offs;
  const int64_t* c_start;
  const int* p0;  // [D_C + 1]
  const Pair* pairs;
  const int2* task;
  int64_t N;
  double alpha;
  Stat* partial;
};

// A task covers kThreads * kGemmEPT elements of one result diagonal; each
// thread owns elements j, j + kThreads, ...  The diagonal's contributing pairs
// are staged through shared memory in chunks, so every pair descriptor is read
// from global memory once per block and broadcast from shared memory.
constexpr int kGemmEPT = 4;
constexpr int kPairChunk = 256;

__global__ void __launch_bounds__(kThreads) gemm_kernel(GemmArgs a) {
  __shared__ Pair sp[kPairChunk];
  const int2 tk = a.task[blockIdx.x];
  const int64_t dc = a.c_offs[tk.x];
  const int64_t L = a.N - (dc < 0 ? -dc : dc);
  const int64_t shift = dc < 0 ? dc : 0;
  int64_t row[kGemmEPT];
  bool live[kGemmEPT];
  double2 acc[kGemmEPT];
#pragma unroll
  for (int e = 0; e < kGemmEPT; ++e) {
    const int64_t j = int64_t(tk.y) + threadIdx.x + e * kThreads;
    live[e] = j < L;
    row[e] = j - shift;
    acc[e] = make_double2(0.0, 0.0);
  }
  const int p0 = a.p0[tk.x], p1 = a.p0[tk.x + 1];
  for (int pc = p0; pc < p1; pc += kPairChunk) {
    const int n = min(kPairChunk, p1 - pc);
    __syncthreads();
    if (int(threadIdx.x) < n) sp[threadIdx.x] = a.pairs[pc + threadIdx.x];
    __syncthreads();
    for (int p = 0; p < n; ++p) {
      const Pair pr = sp[p];
#pragma unroll
      for (int e = 0; e < kGemmEPT; ++e) {
        if (live[e] && row[e] >= pr.lo && row[e] < pr.hi) {
          const double2 x = a.A[pr.a_rb + row[e]], y = a.B[pr.b_rb + row[e]];
          acc[e].x = fma(x.x, y.x, fma(-x.y, y.y, acc[e].x));
          acc[e].y = fma(x.x, y.y, fma(x.y, y.x, acc[e].y));
        }
      }
    }
  }
  Stat s{0.0, 0.0, 0};
#pragma unroll
  for (int e = 0; e < kGemmEPT; ++e) {
    if (live[e]) {
      const double2 v = make_double2(acc[e].x * a.alpha, acc[e].y * a.alpha);
      a.C[a.c_start[tk.x] + row[e] + shift] = v;
      s = stat_merge(s, stat_of(v));
    }
  }
  s = block_stat(s);
  if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
}

// out[k][j] = alpha0 * src0[s0 + j] + alpha1 * src1[s1 + j] (a source with
// start < 0 is absent).  Used for scaling, sums on the union of two diagonal
// sets, dropping diagonals and precision conversion.
struct CombineSrc {
  int64_t s0, s1;
  double2 alpha0, alpha1;
};

template <typename TI, typename TO>
__global__ void __launch_bounds__(kThreads) combine_kernel(const TI* src0, const TI* src1, TO* out,
                                                           const int64_t* offs, const int64_t* start,
                                                           const CombineSrc* srcs, const int2* task, int64_t N) {
  const int2 tk = task[blockIdx.x];
  const int64_t d = offs[tk.x];
  const int64_t L = N - (d < 0 ? -d : d);
  const int64_t j = int64_t(tk.y) + threadIdx.x;
  if (j >= L) return;
  const CombineSrc cs = srcs[tk.x];
  double2 v = make_double2(0.0, 0.0);
  if (cs.s0 >= 0) {
    const double2 x = ld(src0, cs.s0 + j);
    if (cs.alpha0.y == 0.0 && cs.alpha0.x == 1.0) v = x;
    else v = cmul(cs.alpha0, x);
  }
  if (cs.s1 >= 0) {
    const double2 y = ld(src1, cs.s1 + j);
    const double2 w = (cs.alpha1.y == 0.0 && cs.alpha1.x == 1.0) ? y : cmul(cs.alpha1, y);
    v.x += w.x;
    v.y += w.y;
  }
  st(out, start[tk.x] + j, v);
}

// U = exp(-i t A) for a diagonal-only A: exp(t Im a) (cos(t Re a) - i sin(t Re a)).
__global__ void expdiag_kernel(const double2* a, double2* u, int64_t N, double t) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    const double2 v = a[i];
    double sn, cs;
    sincos(t * v.x, &sn, &cs);
    const double m = exp(t * v.y);
    u[i] = make_double2(m * cs, -m * sn);
  }
}

__global__ void ones_kernel(double2* u, int64_t N) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
    u[i] = make_double2(1.0, 0.0);
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename R>
struct CT;
template <>
struct CT<float> {
  using T2 = float2;
};
template <>
struct CT<double> {
  using T2 = double2;
};

// y = A x for n_rhs states.  A block has W warps; warp w takes diagonals
// w, w + W, ... of a tile of 32 * RPT consecutive rows (lane-strided, RPT rows
// per thread), so a small state still keeps many independent loads in flight
// per row; the warps' partial sums meet in shared memory.  (One row per thread
// and 16 warps measured fastest on a 455-diagonal, 2^16-row complex64 matrix:
// 51 us against 52 us for two rows and 79 us for four.)  Rows outside a diagonal load
// element 0 and multiply by zero (no branch).  meta = [offs(D), rowbase(D)].
// FP32 accumulation for complex64, FP64 for complex128.
template <typename R, int RB, int W, int RPT>
__global__ void __launch_bounds__(32 * W) spmv_kernel(const typename CT<R>::T2* __restrict__ vals,
                                                      const int64_t* __restrict__ meta, int D,
                                                      const typename CT<R>::T2* __restrict__ x,
                                                      typename CT<R>::T2* __restrict__ y, int64_t N, int n_rhs,
                                                      int64_t n_vals) {
  using T2 = typename CT<R>::T2;
  constexpr int TILE = 32 * RPT;
  __shared__ R part[W > 1 ? W - 1 : 1][RB][2][TILE];
  pdl_wait();
  pdl_trigger();
  const int64_t* offs = meta;
  const int64_t* rb = meta + D;
  const int w = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
  for (int64_t tile = blockIdx.x; tile * TILE < N; tile += gridDim.x) {
    const int64_t i0 = tile * TILE + lane;
    for (int r0 = 0; r0 < n_rhs; r0 += RB) {
      R ax[RPT][RB], ay[RPT][RB];
#pragma unroll
      for (int e = 0; e < RPT; ++e)
#pragma unroll
        for (int q = 0; q < RB; ++q) ax[e][q] = ay[e][q] = R(0);
#pragma unroll 2
      for (int k = w; k < D; k += W) {
        const int64_t d = __ldg(offs + k);
        const int64_t base = __ldg(rb + k);
#pragma unroll
        for (int e = 0; e < RPT; ++e) {
          const int64_t i = i0 + 32 * e;
          const int64_t c = i + d;
          const bool ok = (uint64_t(c) < uint64_t(N)) && (i < N);
          const T2 v0 = vals[HS_BCHK(ok ? base + i : 0, n_vals, hs::BS_DIA_VAL)];
          const R vx = ok ? v0.x : R(0), vy = ok ? v0.y : R(0);
          const int64_t cc = ok ? c : 0;
#pragma unroll
          for (int q = 0; q < RB; ++q) {
            if (r0 + q < n_rhs) {
              const T2 u = x[HS_BCHK(int64_t(r0 + q) * N + cc, int64_t(n_rhs) * N, hs::BS_DIA_X)];
              ax[e][q] = fma(vx, u.x, fma(-vy, u.y, ax[e][q]));
              ay[e][q] = fma(vx, u.y, fma(vy, u.x, ay[e][q]));
            }
          }
        }
      }
      if (W > 1) {
        if (w > 0) {
#pragma unroll
          for (int e = 0; e < RPT; ++e)
#pragma unroll
            for (int q = 0; q < RB; ++q) {
              part[w - 1][q][0][lane + 32 * e] = ax[e][q];
              part[w - 1][q][1][lane + 32 * e] = ay[e][q];
            }
        }
        __syncthreads();
        if (w == 0) {
#pragma unroll
          for (int s2 = 0; s2 < W - 1; ++s2)
#pragma unroll
            for (int e = 0; e < RPT; ++e)
#pragma unroll
              for (int q = 0; q < RB; ++q) {
                ax[e][q] += part[s2][q][0][lane + 32 * e];
                ay[e][q] += part[s2][q][1][lane + 32 * e];
              }
        }
        __syncthreads();
      }
      if (w == 0) {
#pragma unroll
        for (int e = 0; e < RPT; ++e) {
          const int64_t i = i0 + 32 * e;
          if (i >= N) continue;
#pragma unroll
          for (int q = 0; q < RB; ++q) {
            if (r0 + q < n_rhs) {
              T2 o;
              o.x = ax[e][q];
              o.y = ay[e][q];
              y[int64_t(r0 + q) * N + i] = o;
            }
          }
        }
      }
    }
  }
}

// Expectation values: block b of state r sums conj(psi_i) (A psi)_i and |psi_i|^2
// over a grid-stride set of rows in FP64; partial[r * gridDim.x + b] gets the
// block sums (re, im, norm, unused).
template <typename T2>
__global__ void __launch_bounds__(kThreads) expect_kernel(const T2* __restrict__ vals,
                                                          const int64_t* __restrict__ meta, int D,
                                                          const T2* __restrict__ psi, int64_t N, double4* partial) {
  const int r = blockIdx.y;
  const T2* x = psi + int64_t(r) * N;
  const int64_t* offs = meta;
  const int64_t* rb = meta + D;
  double re = 0.0, im = 0.0, nn = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x; i < N; i += int64_t(gridDim.x) * kThreads) {
    double yr = 0.0, yi = 0.0;
    for (int k = 0; k < D; ++k) {
      const int64_t c = i + __ldg(offs + k);
      if (uint64_t(c) >= uint64_t(N)) continue;
      const double2 v = ld(vals, __ldg(rb + k) + i), u = ld(x, c);
      yr = fma(v.x, u.x, fma(-v.y, u.y, yr));
      yi = fma(v.x, u.y, fma(v.y, u.x, yi));
    }
    const double2 p = ld(x, i);
    re = fma(p.x, yr, fma(p.y, yi, re));   // conj(p) * y
    im = fma(p.x, yi, fma(-p.y, yr, im));
    nn = fma(p.x, p.x, fma(p.y, p.y, nn));
  }
  __shared__ double part_re[kThreads / 32], part_im[kThreads / 32], part_nn[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
    nn += __shfl_xor_sync(0xffffffffu, nn, o);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    part_re[wid] = re;
    part_im[wid] = im;
    part_nn[wid] = nn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      a0 += part_re[w];
      a1 += part_im[w];
      a2 += part_nn[w];
    }
    partial[int64_t(r) * gridDim.x + blockIdx.x] = make_double4(a0, a1, a2, 0.0);
  }
}

// One block per state: the blocks' partial sums in block order.
__global__ void __launch_bounds__(kThreads) expect_final(const double4* partial, int nb, double4* out) {
  const int r = blockIdx.x;
  __shared__ double4 sh[kThreads];
  double4 acc = make_double4(0.0, 0.0, 0.0, 0.0);
  for (int b = threadIdx.x; b < nb; b += kThreads) {
    const double4 p = partial[int64_t(r) * nb + b];
    acc.x += p.x;
    acc.y += p.y;
    acc.z += p.z;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if (int(threadIdx.x) < st) {
      sh[threadIdx.x].x += sh[threadIdx.x + st].x;
      sh[threadIdx.x].y += sh[threadIdx.x + st].y;
      sh[threadIdx.x].z += sh[threadIdx.x + st].z;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[r] = sh[0];
}

// psi[r][i] *= v[i] in place (one diagonal, offset 0).
template <typename R>
__global__ void __launch_bounds__(kThreads) scale_rows_kernel(const typename CT<R>::T2* __restrict__ v,
                                                              typename CT<R>::T2* psi, int64_t N, int n_rhs) {
  using T2 = typename CT<R>::T2;
  pdl_wait();
  pdl_trigger();
  const int64_t total = N * n_rhs;
  for (int64_t e = int64_t(blockIdx.x) * kThreads + threadIdx.x; e < total; e += int64_t(gridDim.x) * kThreads) {
    const T2 a = v[e % N], b = psi[e];
    T2 o;
    o.x = fma(a.x, b.x, -a.y * b.y);
    o.y = fma(a.x, b.y, a.y * b.x);
    psi[e] = o;
  }
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------

size_t esize(hs_dtype dt) { return dt == HS_C64 ? 8 : 16; }

// A device buffer allocated in stream order and freed in stream order.
struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  cudaError_t alloc(size_t bytes, cudaStream_t st) {
    s = st;
    return pool_malloc(&p, bytes ? bytes : 16, st);
  }
  template <typename T>
  cudaError_t upload(const std::vector<T>& v, cudaStream_t st) {
    cudaError_t e = alloc(v.size() * sizeof(T), st);
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

void destroy(hs_dia* m) {
  if (!m) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != m->device) cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  if (m->d_vals) cudaFree(m->d_vals);
  if (m->d_meta) cudaFree(m->d_meta);
  if (cur != m->device) cudaSetDevice(cur);
  delete m;
}

void destroy_async(hs_dia* m, cudaStream_t s) {
  if (!m) return;
  if (m->d_vals) cudaFreeAsync(m->d_vals, s);
  if (m->d_meta) cudaFreeAsync(m->d_meta, s);
  delete m;
}

// Owner of a matrix under construction (freed in stream order unless released).
struct DiaPtr {
  hs_dia* m = nullptr;
  cudaStream_t s = nullptr;
  DiaPtr() = default;
  DiaPtr(hs_dia* p, cudaStream_t st) : m(p), s(st) {}
  DiaPtr(const DiaPtr&) = delete;
  DiaPtr& operator=(const DiaPtr&) = delete;
  DiaPtr(DiaPtr&& o) noexcept : m(o.m), s(o.s) { o.m = nullptr; }
  DiaPtr& operator=(DiaPtr&& o) noexcept {
    if (this != &o) {
      destroy_async(m, s);
      m = o.m;
      s = o.s;
      o.m = nullptr;
    }
    return *this;
  }
  ~DiaPtr() { destroy_async(m, s); }
  hs_dia* release() {
    hs_dia* r = m;
    m = nullptr;
    return r;
  }
  hs_dia* get() const { return m; }
  hs_dia* operator->() const { return m; }
};

// Allocate a matrix with the given (canonical) offsets; values uninitialised.
int make_dia(int n_qubits, const std::vector<int64_t>& offs, hs_dtype dt, cudaStream_t s, DiaPtr& out) {
  DiaPtr m(new hs_dia(), s);
  m->n_qubits = n_qubits;
  m->N = int64_t(1) << n_qubits;
  m->dtype = dt;
  m->offs = offs;
  cudaGetDevice(&m->device);
  int64_t cur = 0;
  std::vector<int64_t> meta(2 * offs.size());
  for (size_t k = 0; k < offs.size(); ++k) {
    m->start.push_back(cur);
    meta[k] = offs[k];
    meta[offs.size() + k] = cur + std::min<int64_t>(0, offs[k]);
    cur += m->N - iabs(offs[k]);
    cur = (cur + kAlignElems - 1) / kAlignElems * kAlignElems;
  }
  m->total = cur;
  cudaError_t e = pool_malloc(&m->d_vals, size_t(std::max<int64_t>(cur, 1)) * esize(dt), s);
  if (e != cudaSuccess) return cuda_err(e, "cudaMallocAsync(matrix values)");
  e = pool_malloc(reinterpret_cast<void**>(&m->d_meta), std::max<size_t>(meta.size(), 1) * sizeof(int64_t), s);
  if (e != cudaSuccess) return cuda_err(e, "cudaMallocAsync(matrix offsets)");
  if (!meta.empty()) {
    e = cudaMemcpyAsync(m->d_meta, meta.data(), meta.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync(matrix offsets)");
  }
  out = std::move(m);
  return HS_OK;
}

// Task table: one (diagonal, first element) per `per` elements; block0[k]
// is the first task of diagonal k (block0[D] = number of tasks).
void make_tasks(const std::vector<int64_t>& offs, int64_t N, std::vector<int2>& task, std::vector<int>& block0,
                int64_t per = kThreads) {
  task.clear();
  block0.assign(offs.size() + 1, 0);
  for (size_t k = 0; k < offs.size(); ++k) {
    block0[k] = int(task.size());
    const int64_t L = N - iabs(offs[k]);
    for (int64_t j = 0; j < L; j += per) task.push_back(make_int2(int(k), int(j)));
  }
  block0[offs.size()] = int(task.size());
}

// Device copies of a matrix's per-diagonal offsets and starts (for task kernels).
struct DiagTables {
  DevBuf offs, start;
  cudaError_t upload(const hs_dia* m, cudaStream_t s) {
    cudaError_t e = offs.upload(m->offs, s);
    if (e == cudaSuccess) e = start.upload(m->start, s);
    return e;
  }
};

// Per-diagonal statistics from block partials (synchronises).
int finish_stats(const std::vector<int>& block0, const DevBuf& partial, size_t D, cudaStream_t s,
                 std::vector<Stat>& out) {
  out.assign(D, Stat{0.0, 0.0, 0});
  if (D == 0) return HS_OK;
  DevBuf d_b0, d_out;
  cudaError_t e = d_b0.upload(block0, s);
  if (e == cudaSuccess) e = d_out.alloc(D * sizeof(Stat), s);
  if (e != cudaSuccess) return cuda_err(e, "statistics buffers");
  stat_final<<<unsigned(D), kThreads, 0, s>>>(partial.as<Stat>(), d_b0.as<int>(), d_out.as<Stat>());
  hs::note_launches();
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), d_out.p, D * sizeof(Stat), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "statistics");
  return HS_OK;
}

// out = sum over sources of alpha * source diagonal, on out's offsets.  `which`
// maps each output diagonal to a diagonal index of a (or -1) and of b (or -1).
int combine(const hs_dia* a, const hs_dia* b, const std::vector<int64_t>& offs, const std::vector<int>& ka,
            const std::vector<int>& kb, double2 alpha_a, double2 alpha_b, hs_dtype out_dt, cudaStream_t s,
            DiaPtr& out) {
  DiaPtr m;
  int rc = make_dia(a->n_qubits, offs, out_dt, s, m);
  if (rc) return rc;
  if (offs.empty()) {
    out = std::move(m);
    return HS_OK;
  }
  std::vector<CombineSrc> src(offs.size());
  for (size_t k = 0; k < offs.size(); ++k) {
    src[k].s0 = ka[k] >= 0 ? a->start[ka[k]] : -1;
    src[k].s1 = (b && kb[k] >= 0) ? b->start[kb[k]] : -1;
    src[k].alpha0 = alpha_a;
    src[k].alpha1 = alpha_b;
  }
  std::vector<int2> task;
  std::vector<int> block0;
  make_tasks(offs, m->N, task, block0);
  DevBuf d_src, d_task;
  DiagTables tabs;
  cudaError_t e = d_src.upload(src, s);
  if (e == cudaSuccess) e = d_task.upload(task, s);
  if (e == cudaSuccess) e = tabs.upload(m.get(), s);
  if (e != cudaSuccess) return cuda_err(e, "combine tables");
  const hs_dtype in_dt = a->dtype;
  if (b && b->dtype != in_dt) return report_error(HS_EDTYPE, "combine: dtype mismatch");
  const void* pb = b ? b->d_vals : a->d_vals;
  const unsigned grid = unsigned(task.size());
  if (in_dt == HS_C128 && out_dt == HS_C128)
    combine_kernel<double2, double2><<<grid, kThreads, 0, s>>>(
        (const double2*)a->d_vals, (const double2*)pb, (double2*)m->d_vals, tabs.offs.as<int64_t>(),
        tabs.start.as<int64_t>(), d_src.as<CombineSrc>(), d_task.as<int2>(), m->N);
  else if (in_dt == HS_C128 && out_dt == HS_C64)
    combine_kernel<double2, float2><<<grid, kThreads, 0, s>>>(
        (const double2*)a->d_vals, (const double2*)pb, (float2*)m->d_vals, tabs.offs.as<int64_t>(),
        tabs.start.as<int64_t>(), d_src.as<CombineSrc>(), d_task.as<int2>(), m->N);
  else if (in_dt == HS_C64 && out_dt == HS_C128)
    combine_kernel<float2, double2><<<grid, kThreads, 0, s>>>(
        (const float2*)a->d_vals, (const float2*)pb, (double2*)m->d_vals, tabs.offs.as<int64_t>(),
        tabs.start.as<int64_t>(), d_src.as<CombineSrc>(), d_task.as<int2>(), m->N);
  else
    combine_kernel<float2, float2><<<grid, kThreads, 0, s>>>(
        (const float2*)a->d_vals, (const float2*)pb, (float2*)m->d_vals, tabs.offs.as<int64_t>(),
        tabs.start.as<int64_t>(), d_src.as<CombineSrc>(), d_task.as<int2>(), m->N);
  hs::note_launches();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "combine launch");
  out = std::move(m);
  return HS_OK;
}

// Keep the diagonals listed in `keep` (indices into m's diagonals).
int select_diagonals(const hs_dia* m, const std::vector<int>& keep, cudaStream_t s, DiaPtr& out) {
  std::vector<int64_t> offs;
  std::vector<int> ka, kb;
  for (int k : keep) {
    offs.push_back(m->offs[k]);
    ka.push_back(k);
    kb.push_back(-1);
  }
  return combine(m, nullptr, offs, ka, kb, make_double2(1.0, 0.0), make_double2(0.0, 0.0), m->dtype, s, out);
}

// A + B on the union of their offsets (canonical order), FP64.
int add_dia(const hs_dia* a, const hs_dia* b, cudaStream_t s, DiaPtr& out) {
  std::map<int64_t, std::pair<int, int>> u;
  for (size_t k = 0; k < a->offs.size(); ++k) u[a->offs[k]] = {int(k), -1};
  for (size_t k = 0; k < b->offs.size(); ++k) {
    auto it = u.find(b->offs[k]);
    if (it == u.end()) u[b->offs[k]] = {-1, int(k)};
    else it->second.second = int(k);
  }
  std::vector<int64_t> offs;
  for (auto& kv : u) offs.push_back(kv.first);
  std::sort(offs.begin(), offs.end(), canonical_before);
  std::vector<int> ka, kb;
  for (int64_t d : offs) {
    ka.push_back(u[d].first);
    kb.push_back(u[d].second);
  }
  // a source absent from a: take b as the first source so that the sum starts from it
  DiaPtr m;
  int rc = make_dia(a->n_qubits, offs, HS_C128, s, m);
  if (rc) return rc;
  std::vector<CombineSrc> src(offs.size());
  for (size_t k = 0; k < offs.size(); ++k) {
    src[k].s0 = ka[k] >= 0 ? a->start[ka[k]] : -1;
    src[k].s1 = kb[k] >= 0 ? b->start[kb[k]] : -1;
    src[k].alpha0 = make_double2(1.0, 0.0);
    src[k].alpha1 = make_double2(1.0, 0.0);
  }
  std::vector<int2> task;
  std::vector<int> block0;
  make_tasks(offs, m->N, task, block0);
  DevBuf d_src, d_task;
  DiagTables tabs;
  cudaError_t e = d_src.upload(src, s);
  if (e == cudaSuccess) e = d_task.upload(task, s);
  if (e == cudaSuccess) e = tabs.upload(m.get(), s);
  if (e != cudaSuccess) return cuda_err(e, "add tables");
  combine_kernel<double2, double2><<<unsigned(task.size()), kThreads, 0, s>>>(
      (const double2*)a->d_vals, (const double2*)b->d_vals, (double2*)m->d_vals, tabs.offs.as<int64_t>(),
      tabs.start.as<int64_t>(), d_src.as<CombineSrc>(), d_task.as<int2>(), m->N);
  hs::note_launches();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "add launch");
  out = std::move(m);
  return HS_OK;
}

int identity_dia(int n_qubits, cudaStream_t s, DiaPtr& out) {
  DiaPtr m;
  int rc = make_dia(n_qubits, std::vector<int64_t>{0}, HS_C128, s, m);
  if (rc) return rc;
  ones_kernel<<<152 * 4, kThreads, 0, s>>>((double2*)m->d_vals, m->N);
  hs::note_launches();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "identity");
  out = std::move(m);
  return HS_OK;
}

// C = alpha * A B with the structural pass on the host, then the drop of
// negligible diagonals.  fro: Frobenius norm of the kept result.
int spgemm_impl(const hs_dia* A, const hs_dia* B, double alpha, cudaStream_t s, DiaPtr& out, double* fro) {
  const int64_t N = A->N;
  std::map<int64_t, std::vector<Pair>> by_dc;
  for (size_t ka = 0; ka < A->offs.size(); ++ka) {
    const int64_t da = A->offs[ka];
    const int64_t a_rb = A->start[ka] + std::min<int64_t>(0, da);
    for (size_t kb = 0; kb < B->offs.size(); ++kb) {
      const int64_t db = B->offs[kb];
      const int64_t dc = da + db;
      if (iabs(dc) >= N) continue;
      const int64_t lo = std::max<int64_t>({0, -da, -dc}), hi = std::min<int64_t>({N, N - da, N - dc});
      if (lo >= hi) continue;
      const int64_t b_rb = B->start[kb] + std::min<int64_t>(0, db) + da;
      by_dc[dc].push_back(Pair{a_rb, b_rb, lo, hi});
    }
  }
  std::vector<int64_t> offs;
  for (auto& kv : by_dc) offs.push_back(kv.first);
  std::sort(offs.begin(), offs.end(), canonical_before);
  std::vector<Pair> pairs;
  std::vector<int> p0;
  for (int64_t dc : offs) {
    p0.push_back(int(pairs.size()));
    const auto& v = by_dc[dc];
    pairs.insert(pairs.end(), v.begin(), v.end());
  }
  p0.push_back(int(pairs.size()));
  DiaPtr C;
  int rc = make_dia(A->n_qubits, offs, HS_C128, s, C);
  if (rc) return rc;
  if (offs.empty()) {
    if (fro) *fro = 0.0;
    out = std::move(C);
    return HS_OK;
  }
  std::vector<int2> task;
  std::vector<int> block0;
  make_tasks(offs, N, task, block0, int64_t(kThreads) * kGemmEPT);
  DevBuf d_p0, d_pairs, d_task, d_part;
  DiagTables tabs;
  cudaError_t e = d_p0.upload(p0, s);
  if (e == cudaSuccess) e = d_pairs.upload(pairs, s);
  if (e == cudaSuccess) e = d_task.upload(task, s);
  if (e == cudaSuccess) e = tabs.upload(C.get(), s);
  if (e == cudaSuccess) e = d_part.alloc(task.size() * sizeof(Stat), s);
  if (e != cudaSuccess) return cuda_err(e, "spgemm tables");
  GemmArgs g{(const double2*)A->d_vals, (const double2*)B->d_vals, (double2*)C->d_vals, tabs.offs.as<int64_t>(),
             tabs.start.as<int64_t>(), d_p0.as<int>(), d_pairs.as<Pair>(), d_task.as<int2>(), N, alpha,
             d_part.as<Stat>()};
  gemm_kernel<<<unsigned(task.size()), kThreads, 0, s>>>(g);
  hs::note_launches();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "spgemm launch");
  std::vector<Stat> st;
  rc = finish_stats(block0, d_part, offs.size(), s, st);
  if (rc) return rc;
  double top = 0.0;
  for (const Stat& x : st) top = std::max(top, x.mx);
  const double thr = kDropRel * top;
  std::vector<int> keep;
  double s2 = 0.0;
  int64_t nnz = 0;
  for (size_t k = 0; k < st.size(); ++k)
    if (st[k].mx > thr) {
      keep.push_back(int(k));
      s2 += st[k].s2;
      nnz += st[k].nz;
    }
  if (fro) *fro = std::sqrt(s2);
  if (keep.size() == offs.size()) {
    C->nnz = nnz;
    out = std::move(C);
    return HS_OK;
  }
  DiaPtr K;
  rc = select_diagonals(C.get(), keep, s, K);
  if (rc) return rc;
  K->nnz = nnz;
  out = std::move(K);
  return HS_OK;
}

bool diagonal_only(const hs_dia* a) { return a->offs.empty() || (a->offs.size() == 1 && a->offs[0] == 0); }

// Alg. 2 (or the exact diagonal path).  max_diags > 0 stops early (not
// converged) once U holds more diagonals.
int spme_impl(const hs_dia* A, double t, double tol, int max_iter, int max_diags, cudaStream_t s, DiaPtr& out,
              int* n_terms, bool* converged) {
  if (diagonal_only(A)) {
    DiaPtr U;
    int rc = make_dia(A->n_qubits, std::vector<int64_t>{0}, HS_C128, s, U);
    if (rc) return rc;
    if (A->offs.empty()) {
      ones_kernel<<<152 * 4, kThreads, 0, s>>>((double2*)U->d_vals, U->N);
    } else {
      expdiag_kernel<<<152 * 8, kThreads, 0, s>>>((const double2*)A->d_vals, (double2*)U->d_vals, U->N, t);
    }
    hs::note_launches();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "exact diagonal exponential");
    *n_terms = 0;
    *converged = true;
    out = std::move(U);
    return HS_OK;
  }
  // X = A (-i t)
  std::vector<int> ka(A->offs.size()), kb(A->offs.size(), -1);
  for (size_t k = 0; k < ka.size(); ++k) ka[k] = int(k);
  DiaPtr X, U, T;
  int rc = combine(A, nullptr, A->offs, ka, kb, make_double2(0.0, -t), make_double2(0.0, 0.0), HS_C128, s, X);
  if (!rc) rc = identity_dia(A->n_qubits, s, U);
  if (!rc) rc = identity_dia(A->n_qubits, s, T);
  if (rc) return rc;
  *converged = false;
  *n_terms = max_iter;
  for (int k = 1; k <= max_iter; ++k) {
    DiaPtr T2;
    double fro = 0.0;
    rc = spgemm_impl(T.get(), X.get(), 1.0 / double(k), s, T2, &fro);
    if (rc) return rc;
    if (fro < tol) {
      *n_terms = k;
      *converged = true;
      break;
    }
    DiaPtr U2;
    rc = add_dia(U.get(), T2.get(), s, U2);
    if (rc) return rc;
    U = std::move(U2);
    T = std::move(T2);
    if (max_diags > 0 && int64_t(U->offs.size()) > max_diags) {
      *n_terms = k;
      break;
    }
  }
  out = std::move(U);
  return HS_OK;
}

int check_matrix(const hs_dia* a, const char* name) {
  if (!a) return report_error(HS_EINVAL, std::string(name) + " is NULL");
  return HS_OK;
}

// Element offset of a state buffer pointer check (16-byte alignment).
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Warps per block (diagonal slices) and rows per thread for a D-diagonal matrix.
constexpr int kSpmvRPT = 1;

template <typename R, int RB, int W>
cudaError_t launch_spmv_k(const hs_dia* a, const void* x, void* y, int n_rhs, cudaLaunchConfig_t& cfg) {
  using T2 = typename CT<R>::T2;
  const int64_t tiles = (a->N + 32 * kSpmvRPT - 1) / (32 * kSpmvRPT);
  const int64_t per_sm = std::max(1, 64 / W);  // blocks per SM for a full grid
  cfg.gridDim = dim3(unsigned(std::max<int64_t>(1, std::min<int64_t>(tiles, 152 * per_sm))), 1u, 1u);
  cfg.blockDim = dim3(32 * W, 1u, 1u);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, spmv_kernel<R, RB, W, kSpmvRPT>, (const T2*)a->d_vals,
                                           (const int64_t*)a->d_meta, int(a->offs.size()), (const T2*)x, (T2*)y,
                                           a->N, n_rhs, a->total);
  if (e == cudaSuccess) hs::note_launches();
  return e;
}

template <typename R, int RB>
cudaError_t launch_spmv_w(const hs_dia* a, const void* x, void* y, int n_rhs, cudaLaunchConfig_t& cfg) {
  const int D = int(a->offs.size());
  // 16 slices only while their partial sums fit 32 KB of static shared memory
  if constexpr (RB * sizeof(R) <= 8) {
    if (D >= 64) return launch_spmv_k<R, RB, 16>(a, x, y, n_rhs, cfg);
  }
  if (D >= 16) return launch_spmv_k<R, RB, 8>(a, x, y, n_rhs, cfg);
  if (D >= 4) return launch_spmv_k<R, RB, 4>(a, x, y, n_rhs, cfg);
  return launch_spmv_k<R, RB, 2>(a, x, y, n_rhs, cfg);
}

cudaError_t launch_spmv(const hs_dia* a, const void* x, void* y, int n_rhs, cudaStream_t s, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads, 1u, 1u);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  if (a->dtype == HS_C64) {
    if (n_rhs >= 4) return launch_spmv_w<float, 4>(a, x, y, n_rhs, cfg);
    if (n_rhs >= 2) return launch_spmv_w<float, 2>(a, x, y, n_rhs, cfg);
    return launch_spmv_w<float, 1>(a, x, y, n_rhs, cfg);
  }
  if (n_rhs >= 2) return launch_spmv_w<double, 2>(a, x, y, n_rhs, cfg);
  return launch_spmv_w<double, 1>(a, x, y, n_rhs, cfg);
}

cudaError_t launch_scale_rows(const hs_dia* a, void* psi, int n_rhs, cudaStream_t s, bool pdl) {
  int64_t blocks = (a->N * n_rhs + kThreads - 1) / kThreads;
  blocks = std::min<int64_t>(blocks, 152 * 8);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(std::max<int64_t>(blocks, 1)), 1u, 1u);
  cfg.blockDim = dim3(kThreads, 1u, 1u);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  const cudaError_t e =
      a->dtype == HS_C64
          ? cudaLaunchKernelEx(&cfg, scale_rows_kernel<float>, (const float2*)a->d_vals, (float2*)psi, a->N, n_rhs)
          : cudaLaunchKernelEx(&cfg, scale_rows_kernel<double>, (const double2*)a->d_vals, (double2*)psi, a->N, n_rhs);
  if (e == cudaSuccess) hs::note_launches();
  return e;
}

}  // namespace

namespace hs {
// Free a matrix in stream order on s (no device synchronisation): its memory
// returns to the pool once the work already enqueued on s has run.
void dia_free_async(hs_dia* m, cudaStream_t s) { destroy_async(m, s); }
}  // namespace hs

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

int hs_dia_from_masks(const uint64_t* x, const uint64_t* z, const double* coeffs, size_t n_terms, int n_qubits,
                      void* cuda_stream, hs_dia** out) {
  if (!out) return report_error(HS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!x || !z || !coeffs) return report_error(HS_EINVAL, "null term array");
  if (n_terms == 0) return report_error(HS_EINVAL, "no terms");
  if (n_qubits < 1 || n_qubits > HS_MAX_QUBITS) return report_error(HS_EINVAL, "n_qubits out of range");
  const uint64_t lim = n_qubits >= 64 ? ~0ull : ((1ull << n_qubits) - 1);
  for (size_t j = 0; j < n_terms; ++j) {
    if ((x[j] | z[j]) & ~lim) return report_error(HS_EINVAL, "mask bit beyond n_qubits");
    if (!std::isfinite(coeffs[j])) return report_error(HS_EINVAL, "non-finite coefficient");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int64_t N = int64_t(1) << n_qubits;
  // terms grouped by x mask, input order kept inside a group
  std::vector<size_t> order(n_terms);
  for (size_t j = 0; j < n_terms; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return x[a] < x[b]; });
  std::vector<uint64_t> masks, tz;
  std::vector<int> mrange, ty;
  std::vector<double> tc;
  for (size_t q = 0; q < n_terms; ++q) {
    const size_t j = order[q];
    if (masks.empty() || masks.back() != x[j]) {
      masks.push_back(x[j]);
      mrange.push_back(int(q));
    }
    tz.push_back(z[j]);
    tc.push_back(coeffs[j]);
    ty.push_back(__builtin_popcountll(x[j] & z[j]) & 3);
  }
  mrange.push_back(int(n_terms));
  // structural candidates: the union of offs(u) over the distinct masks
  std::vector<int64_t> cand;
  for (uint64_t u : masks) {
    if (__builtin_popcountll(u) > 16) return report_error(HS_EINVAL, "a term flips more than 16 qubits");
    std::vector<int64_t> o{0};
    for (int k = 0; k < n_qubits; ++k) {
      if (!((u >> k) & 1ull)) continue;
      const size_t m = o.size();
      for (size_t i = 0; i < m; ++i) {
        o.push_back(o[i] - (int64_t(1) << k));
        o[i] += int64_t(1) << k;
      }
    }
    cand.insert(cand.end(), o.begin(), o.end());
    if (cand.size() > size_t(8) * kMaxCandidates) {
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    }
  }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  if (cand.size() > size_t(kMaxCandidates)) return report_error(HS_EINVAL, "more than 65536 candidate diagonals");
  std::sort(cand.begin(), cand.end(), canonical_before);
  DiaPtr C;
  int rc = make_dia(n_qubits, cand, HS_C128, s, C);
  if (rc) return rc;
  std::vector<int2> task;
  std::vector<int> block0;
  make_tasks(cand, N, task, block0);
  DevBuf d_masks, d_mrange, d_tz, d_tc, d_ty, d_task, d_part;
  DiagTables tabs;
  cudaError_t e = d_masks.upload(masks, s);
  if (e == cudaSuccess) e = d_mrange.upload(mrange, s);
  if (e == cudaSuccess) e = d_tz.upload(tz, s);
  if (e == cudaSuccess) e = d_tc.upload(tc, s);
  if (e == cudaSuccess) e = d_ty.upload(ty, s);
  if (e == cudaSuccess) e = d_task.upload(task, s);
  if (e == cudaSuccess) e = tabs.upload(C.get(), s);
  if (e == cudaSuccess) e = d_part.alloc(task.size() * sizeof(Stat), s);
  if (e != cudaSuccess) return cuda_err(e, "H tables");
  TermsArgs a{(double2*)C->d_vals, tabs.offs.as<int64_t>(), tabs.start.as<int64_t>(), d_task.as<int2>(),
              d_masks.as<uint64_t>(), d_mrange.as<int>(), d_tz.as<uint64_t>(), d_tc.as<double>(), d_ty.as<int>(),
              int(masks.size()), N, d_part.as<Stat>()};
  terms_kernel<<<unsigned(task.size()), kThreads, 0, s>>>(a);
  hs::note_launches();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "H launch");
  std::vector<Stat> st;
  rc = finish_stats(block0, d_part, cand.size(), s, st);
  if (rc) return rc;
  std::vector<int> keep;
  int64_t nnz = 0;
  for (size_t k = 0; k < st.size(); ++k)
    if (st[k].nz > 0) {
      keep.push_back(int(k));
      nnz += st[k].nz;
    }
  DiaPtr H;
  if (keep.size() == cand.size()) {
    H = std::move(C);
  } else {
    rc = select_diagonals(C.get(), keep, s, H);
    if (rc) return rc;
  }
  H->nnz = nnz;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "H build");
  *out = H.release();
  return HS_OK;
}

int hs_dia_from_terms(const char* const* pauli_terms, const double* coeffs, size_t n_terms, void* cuda_stream,
                      hs_dia** out) {
  if (!out) return report_error(HS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!pauli_terms || !coeffs) return report_error(HS_EINVAL, "null term array");
  std::vector<uint64_t> x, z;
  int n = 0;
  std::string err;
  int rc = hs::parse_labels(pauli_terms, n_terms, x, z, n, &err);
  if (rc) return report_error(rc, err);
  return hs_dia_from_masks(x.data(), z.data(), coeffs, n_terms, n, cuda_stream, out);
}

int hs_dia_create(int n_qubits, const int64_t* offsets, size_t n_diags, const double* values, hs_dtype dtype,
                  void* cuda_stream, hs_dia** out) {
  if (!out) return report_error(HS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > HS_MAX_QUBITS) return report_error(HS_EINVAL, "n_qubits out of range");
  if (dtype != HS_C64 && dtype != HS_C128) return report_error(HS_EDTYPE, "dtype must be HS_C64 or HS_C128");
  if (n_diags > 0 && (!offsets || !values)) return report_error(HS_EINVAL, "null offsets or values");
  const int64_t N = int64_t(1) << n_qubits;
  std::vector<int64_t> given(offsets, offsets + n_diags);
  std::vector<int64_t> srt = given;
  std::sort(srt.begin(), srt.end());
  for (size_t k = 0; k < srt.size(); ++k) {
    if (iabs(srt[k]) >= N) return report_error(HS_EINVAL, "offset out of range");
    if (k && srt[k] == srt[k - 1]) return report_error(HS_EINVAL, "duplicate offset");
  }
  std::vector<int64_t> offs = given;
  std::sort(offs.begin(), offs.end(), canonical_before);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  DiaPtr m;
  int rc = make_dia(n_qubits, offs, dtype, s, m);
  if (rc) return rc;
  // host image in the padded layout
  std::map<int64_t, size_t> src_at;
  size_t pos = 0;
  for (int64_t d : given) {
    src_at[d] = pos;
    pos += size_t(N - iabs(d));
  }
  const size_t es = esize(dtype);
  std::vector<unsigned char> img(size_t(m->total) * es, 0);
  for (size_t k = 0; k < offs.size(); ++k) {
    const size_t L = size_t(N - iabs(offs[k]));
    const double* v = values + 2 * src_at[offs[k]];
    unsigned char* dst = img.data() + size_t(m->start[k]) * es;
    if (dtype == HS_C128) {
      std::memcpy(dst, v, L * 16);
    } else {
      float* f = reinterpret_cast<float*>(dst);
      for (size_t i = 0; i < 2 * L; ++i) f[i] = float(v[i]);
    }
  }
  cudaError_t e = img.empty() ? cudaSuccess : cudaMemcpyAsync(m->d_vals, img.data(), img.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "matrix upload");
  *out = m.release();
  return HS_OK;
}

int hs_spgemm(const hs_dia* a, const hs_dia* b, void* cuda_stream, hs_dia** out, double* fro_norm) {
  if (!out) return report_error(HS_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_matrix(a, "a");
  if (!rc) rc = check_matrix(b, "b");
  if (rc) return rc;
  if (a->N != b->N) return report_error(HS_EINVAL, "matrix sizes differ");
  if (a->dtype != HS_C128 || b->dtype != HS_C128) return report_error(HS_EDTYPE, "hs_spgemm needs HS_C128 matrices");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  DiaPtr C;
  double fro = 0.0;
  rc = spgemm_impl(a, b, 1.0, s, C, &fro);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "spgemm");
  if (fro_norm) *fro_norm = fro;
  *out = C.release();
  return HS_OK;
}

int hs_spme(const hs_dia* a, double t, double tol, int max_iter, void* cuda_stream, hs_dia** out, int* n_terms,
            int* converged) {
  if (!out) return report_error(HS_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_matrix(a, "a");
  if (rc) return rc;
  if (a->dtype != HS_C128) return report_error(HS_EDTYPE, "hs_spme needs an HS_C128 matrix");
  if (!std::isfinite(t)) return report_error(HS_EINVAL, "t must be finite");
  if (!(tol > 0.0) || max_iter < 1) return report_error(HS_EINVAL, "tol must be > 0 and max_iter >= 1");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  DiaPtr U;
  int k = 0;
  bool ok = false;
  rc = spme_impl(a, t, tol, max_iter, 0, s, U, &k, &ok);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "spme");
  if (n_terms) *n_terms = k;
  if (converged) *converged = ok ? 1 : 0;
  *out = U.release();
  return HS_OK;
}

int hs_estimate_timesteps(const hs_dia* a, double t, int diag_budget, double tol, int max_iter, int max_steps,
                          void* cuda_stream, int* n_steps) {
  if (!n_steps) return report_error(HS_EINVAL, "n_steps is NULL");
  int rc = check_matrix(a, "a");
  if (rc) return rc;
  if (a->dtype != HS_C128) return report_error(HS_EDTYPE, "hs_estimate_timesteps needs an HS_C128 matrix");
  if (!(t > 0.0) || !std::isfinite(t)) return report_error(HS_EINVAL, "t must be > 0");
  if (diag_budget < 1 || max_steps < 1 || max_iter < 1 || !(tol > 0.0))
    return report_error(HS_EINVAL, "diag_budget, max_steps, max_iter must be >= 1 and tol > 0");
  if (diagonal_only(a)) {
    *n_steps = 1;
    return HS_OK;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  // The Taylor terms at step dt are T_k = (-i dt)^k A^k / k!: their diagonal
  // sets are those of A^k (the drop rule is relative, so scale-free) and their
  // norms dt^k ||A^k||_F / k!.  The powers are formed once, until the union of
  // their diagonal sets (with the main diagonal of I) passes the budget; every
  // candidate r is then decided on the host: feasible iff the first k whose
  // term norm is below tol comes before that point (and within max_iter).
  std::vector<double> nrm(1, 0.0);  // nrm[k] = ||A^k||_F, k >= 1
  int kstar = max_iter;            // terms T_1 .. T_{K-1} fit the budget iff K <= kstar
  {
    DiaPtr P;
    int rc2 = identity_dia(a->n_qubits, s, P);
    if (rc2) return rc2;
    std::vector<int64_t> uni{0};
    for (int k = 1; k <= max_iter; ++k) {
      DiaPtr P2;
      double fro = 0.0;
      rc2 = spgemm_impl(P.get(), a, 1.0, s, P2, &fro);
      if (rc2) return rc2;
      nrm.push_back(fro);
      std::vector<int64_t> merged;
      std::vector<int64_t> sk = P2->offs;
      std::sort(sk.begin(), sk.end());
      std::set_union(uni.begin(), uni.end(), sk.begin(), sk.end(), std::back_inserter(merged));
      uni.swap(merged);
      P = std::move(P2);
      if (int64_t(uni.size()) > diag_budget) {
        kstar = k;
        break;
      }
    }
  }
  auto feasible = [&](int r) -> bool {
    const double dt = t / double(r);
    double term = 1.0;  // dt^k / k!
    for (int k = 1; k < int(nrm.size()); ++k) {
      term = term * dt / double(k);
      if (term * nrm[k] < tol) return k <= kstar;
    }
    return false;  // no term under tol within the powers formed: not converged, or over budget
  };
  int64_t lo = 0, hi = 1;
  while (!feasible(int(hi))) {
    lo = hi;
    hi *= 2;
    if (hi > max_steps) return report_error(HS_EINVAL, "diagonal budget not met within max_steps");
  }
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    if (feasible(int(mid))) hi = mid;
    else lo = mid;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "estimate_timesteps");
  *n_steps = int(hi);
  return HS_OK;
}

int hs_spmv(const hs_dia* a, const void* x, void* y, int n_rhs, void* cuda_stream) {
  int rc = check_matrix(a, "a");
  if (rc) return rc;
  if (!x || !y) return report_error(HS_EINVAL, "null state buffer");
  if (!aligned16(x) || !aligned16(y)) return report_error(HS_EINVAL, "state buffers must be 16-byte aligned");
  if (n_rhs < 1) return report_error(HS_EINVAL, "n_rhs must be >= 1");
  const size_t bytes = size_t(n_rhs) * size_t(a->N) * esize(a->dtype);
  const char* xb = static_cast<const char*>(x);
  const char* yb = static_cast<const char*>(y);
  if (xb < yb + bytes && yb < xb + bytes) return report_error(HS_EINVAL, "x and y overlap");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = launch_spmv(a, x, y, n_rhs, s, false);
  if (e != cudaSuccess) return cuda_err(e, "spmv launch");
  return HS_OK;
}

int hs_expectation(const hs_dia* a, const void* psi, int n_rhs, void* cuda_stream, double* values, double* norms) {
  int rc = check_matrix(a, "a");
  if (rc) return rc;
  if (!psi || !values) return report_error(HS_EINVAL, "null argument");
  if (!aligned16(psi)) return report_error(HS_EINVAL, "psi must be 16-byte aligned");
  if (n_rhs < 1 || n_rhs > 65535) return report_error(HS_EINVAL, "n_rhs must be 1..65535");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int nb = int(std::max<int64_t>(1, std::min<int64_t>((a->N + kThreads - 1) / kThreads, 152 * 4)));
  DevBuf part, out;
  cudaError_t e = part.alloc(size_t(nb) * n_rhs * sizeof(double4), s);
  if (e == cudaSuccess) e = out.alloc(size_t(n_rhs) * sizeof(double4), s);
  if (e != cudaSuccess) return cuda_err(e, "expectation buffers");
  const int D = int(a->offs.size());
  const dim3 grid{unsigned(nb), unsigned(n_rhs), 1u};
  if (a->dtype == HS_C64)
    expect_kernel<float2><<<grid, kThreads, 0, s>>>((const float2*)a->d_vals, (const int64_t*)a->d_meta, D,
                                                    (const float2*)psi, a->N, part.as<double4>());
  else
    expect_kernel<double2><<<grid, kThreads, 0, s>>>((const double2*)a->d_vals, (const int64_t*)a->d_meta, D,
                                                     (const double2*)psi, a->N, part.as<double4>());
  expect_final<<<unsigned(n_rhs), kThreads, 0, s>>>(part.as<double4>(), nb, out.as<double4>());
  hs::note_launches(2);
  std::vector<double4> h(n_rhs);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), out.p, h.size() * sizeof(double4), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "expectation");
  for (int r = 0; r < n_rhs; ++r) {
    values[2 * r] = h[r].x;
    values[2 * r + 1] = h[r].y;
    if (norms) norms[r] = h[r].z;
  }
  return HS_OK;
}

int hs_dia_evolve(const hs_dia* u, void* psi, int n_rhs, int n_steps, void* cuda_stream) {
  int rc = check_matrix(u, "u");
  if (rc) return rc;
  if (!psi) return report_error(HS_EINVAL, "psi is NULL");
  if (!aligned16(psi)) return report_error(HS_EINVAL, "psi must be 16-byte aligned");
  if (n_rhs < 1 || n_steps < 0) return report_error(HS_EINVAL, "n_rhs must be >= 1 and n_steps >= 0");
  if (n_steps == 0) return HS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (u->offs.size() == 1 && u->offs[0] == 0) {
    for (int k = 0; k < n_steps; ++k) {
      cudaError_t e = launch_scale_rows(u, psi, n_rhs, s, k > 0);
      if (e != cudaSuccess) return cuda_err(e, "diagonal evolve launch");
    }
    return HS_OK;
  }
  const size_t bytes = size_t(n_rhs) * size_t(u->N) * esize(u->dtype);
  DevBuf tmp;
  cudaError_t e = tmp.alloc(bytes, s);
  if (e != cudaSuccess) return cuda_err(e, "cudaMallocAsync(scratch state)");
  void* a = psi;
  void* b = tmp.p;
  for (int k = 0; k < n_steps; ++k) {
    e = launch_spmv(u, a, b, n_rhs, s, k > 0);
    if (e != cudaSuccess) return cuda_err(e, "evolve launch");
    std::swap(a, b);
  }
  if (a != psi) {
    e = cudaMemcpyAsync(psi, a, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_err(e, "evolve copy-back");
  }
  return HS_OK;
}

int hs_dia_convert(const hs_dia* a, hs_dtype dtype, void* cuda_stream, hs_dia** out) {
  if (!out) return report_error(HS_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_matrix(a, "a");
  if (rc) return rc;
  if (dtype != HS_C64 && dtype != HS_C128) return report_error(HS_EDTYPE, "dtype must be HS_C64 or HS_C128");
  std::vector<int> ka(a->offs.size()), kb(a->offs.size(), -1);
  for (size_t k = 0; k < ka.size(); ++k) ka[k] = int(k);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  DiaPtr m;
  rc = combine(a, nullptr, a->offs, ka, kb, make_double2(1.0, 0.0), make_double2(0.0, 0.0), dtype, s, m);
  if (rc) return rc;
  *out = m.release();
  return HS_OK;
}

int hs_dia_info(const hs_dia* a, int* n_qubits, int* n_diags, int64_t* nnz, hs_dtype* dtype) {
  int rc = check_matrix(a, "a");
  if (rc) return rc;
  if (n_qubits) *n_qubits = a->n_qubits;
  if (n_diags) *n_diags = int(a->offs.size());
  if (nnz) *nnz = a->nnz;
  if (dtype) *dtype = a->dtype;
  return HS_OK;
}

int hs_dia_get(const hs_dia* a, int64_t* offsets, double* values) {
  int rc = check_matrix(a, "a");
  if (rc) return rc;
  if (offsets) std::memcpy(offsets, a->offs.data(), a->offs.size() * sizeof(int64_t));
  if (!values) return HS_OK;
  const size_t es = esize(a->dtype);
  std::vector<unsigned char> img(size_t(a->total) * es);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && !img.empty()) e = cudaMemcpy(img.data(), a->d_vals, img.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(e, "matrix download");
  size_t pos = 0;
  for (size_t k = 0; k < a->offs.size(); ++k) {
    const size_t L = size_t(a->N - iabs(a->offs[k]));
    const unsigned char* src = img.data() + size_t(a->start[k]) * es;
    if (a->dtype == HS_C128) {
      std::memcpy(values + 2 * pos, src, L * 16);
    } else {
      const float* f = reinterpret_cast<const float*>(src);
      for (size_t i = 0; i < 2 * L; ++i) values[2 * pos + i] = double(f[i]);
    }
    pos += L;
  }
  return HS_OK;
}

void hs_dia_free(hs_dia* a) { destroy(a); }

}  // extern "C"
