// Factor application kernels (Alg. 1 and the evolution loop of Alg. 3).
//
// A factor in the compact layout is applied as
//     y[r] = sum_k v_k(r) * x[r + d_k]   over diagonals k with 0 <= r + d_k < N,
// where v_k(r) is element min(r, r + d_k) of diagonal k, stored at
// vals[rowbase_k + r] (rowbase_k is a multiple of the 32-byte alignment, so
// a warp's reads along a diagonal are aligned and coalesced).
//
// Two kernels:
//  * apply_plain: one launch per factor application, out of place, one thread
//    per row, factor values read once per launch and reused for every state
//    of a multi-RHS block.
//  * sweep: a CTA holds a TILE of 2^T amplitudes (for rhs_block states) in
//    shared memory -- the amplitudes whose bits outside a "local" bit set L are
//    fixed by the CTA index -- and applies a run of consecutive factors whose
//    flip masks lie inside L.  For such a factor every structural nonzero of
//    row r sits in a column r xor u with u spanned by L, i.e. inside the same
//    tile; a stored value on a column outside the tile is an exact zero written
//    by the build, so the column is read at its in-tile image (the bits of
//    r + d_k selected by L), which is always a valid shared-memory address and
//    contributes 0.  The tile is read from and written to global memory once
//    per sweep instead of once per factor.
//
//    Factor values do not depend on the state, so they are staged into a ring
//    of shared-memory stages with cp.async several factors ahead of their use,
//    and the kernel is launched with programmatic dependent launch: the next
//    sweep's CTAs start, stage their first factors while the previous sweep is
//    still finishing, and only then wait (griddepcontrol.wait) before they read
//    the state.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "hs_internal.h"

namespace hs {
namespace {

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename T2>
__device__ __forceinline__ void cfma(T2& acc, const T2 v, const T2 x) {
  acc.x = fma(v.x, x.x, acc.x);
  acc.x = fma(-v.y, x.y, acc.x);
  acc.y = fma(v.x, x.y, acc.y);
  acc.y = fma(v.y, x.x, acc.y);
}

// ---------------------------------------------------------------------------
// Plain row-parallel diagonal-times-vector product.
// ---------------------------------------------------------------------------
template <typename R, int RB>
__global__ void __launch_bounds__(256) apply_plain_kernel(const typename C2<R>::T* __restrict__ vals,
                                                          const int64_t* __restrict__ offs,
                                                          const int64_t* __restrict__ rowbase, int D,
                                                          const typename C2<R>::T* __restrict__ x,
                                                          typename C2<R>::T* __restrict__ y, int64_t N, int n_rhs) {
  using T2 = typename C2<R>::T;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < N; r += int64_t(gridDim.x) * blockDim.x) {
    for (int q0 = 0; q0 < n_rhs; q0 += RB) {
      T2 acc[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) acc[q] = T2{0, 0};
      for (int k = 0; k < D; ++k) {
        const int64_t c = r + offs[k];
        if (c < 0 || c >= N) continue;
        const T2 v = vals[rowbase[k] + r];
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (q0 + q < n_rhs) cfma(acc[q], v, x[int64_t(q0 + q) * N + c]);
      }
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (q0 + q < n_rhs) y[int64_t(q0 + q) * N + r] = acc[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Fused tile sweep.
// ---------------------------------------------------------------------------
struct SweepArgs {
  const void* src;
  void* dst;
  const void* vals;
  const int64_t* offs;
  const int64_t* rowbase;
  int64_t N;
  int n_rhs;
  int rhs_block;
  int tile_bits;
  int n_tiles_log2;
  int n_stages;      // factor stages in the shared-memory ring
  int stage_diags;   // diagonals per stage (max D over the sweep's factors)
  int n_meta;        // diagonals listed in the shared-memory metadata table
  // Local bits [0, a) U [h, h + w): local index of row r is
  // (r & m0) | ((r >> sh) & m1), with m0 = 2^a - 1, m1 = (2^w - 1) << a, sh = h - a.
  uint32_t m0, m1;
  int sh;
  Runs rest;         // the other bits, enumerated by the CTA index
  int n_factors;
  // Per factor of the sweep: first diagonal in the global diagonal arrays,
  // diagonal count, and position of its first diagonal in the metadata table.
  int fdiag0[kMaxSweepFactors];
  int16_t fD[kMaxSweepFactors];
  int16_t fmeta[kMaxSweepFactors];
};

// Scatter the low bits of v into the positions of the runs.
__device__ __forceinline__ uint32_t deposit_runs(uint32_t v, const Runs& R) {
  uint32_t out = 0;
  int q = 0;
  for (int i = 0; i < R.n; ++i) {
    out |= ((v >> q) & ((1u << R.len[i]) - 1u)) << R.pos[i];
    q += R.len[i];
  }
  return out;
}

__device__ __forceinline__ uint32_t local_of(uint32_t c, uint32_t m0, uint32_t m1, int sh) {
  return (c & m0) | ((c >> sh) & m1);
}
__device__ __forceinline__ uint32_t global_of(uint32_t l, uint32_t m0, uint32_t m1, int sh) {
  return (l & m0) | ((l & m1) << sh);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, uint32_t src_bytes) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most n of the most recently committed groups are pending.
__device__ __forceinline__ void cp_async_wait(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
  }
}
// Programmatic dependent launch controls (no-ops when launched without the attribute).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Block of TS / ROWS threads; thread t owns local rows t + i * blockDim.x.
template <typename R, int ROWS, int RB>
__global__ void __launch_bounds__(256) sweep_kernel(const __grid_constant__ SweepArgs a) {
  using T2 = typename C2<R>::T;
  constexpr int V = 16 / sizeof(T2);  // elements per 16-byte chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  const uint32_t TS = 1u << a.tile_bits;
  const uint32_t m0 = a.m0, m1 = a.m1;
  const int sh = a.sh;
  // Shared memory: [diagonal metadata (offset, rowbase)][tile][factor stages]
  longlong2* meta = reinterpret_cast<longlong2*>(smem_raw);
  T2* tile = reinterpret_cast<T2*>(smem_raw + size_t(a.n_meta) * sizeof(longlong2));
  T2* stages = tile + size_t(a.rhs_block) * TS;
  const uint32_t stage_elems = uint32_t(a.stage_diags) * TS;
  // src and dst may be the same buffer (in-place sweep): every CTA reads its
  // own tile completely before it writes it back, and tiles are disjoint.
  const T2* src = reinterpret_cast<const T2*>(a.src);
  T2* dst = reinterpret_cast<T2*>(a.dst);
  const T2* __restrict__ vals = reinterpret_cast<const T2*>(a.vals);

  const uint32_t tile_id = blockIdx.x & ((1u << a.n_tiles_log2) - 1u);
  const int rhs0 = int(blockIdx.x >> a.n_tiles_log2) * a.rhs_block;
  const int nrb = min(a.rhs_block, a.n_rhs - rhs0);
  const uint32_t base = deposit_runs(tile_id, a.rest);
  const uint32_t n_chunks = TS / V;
  const int N = int(a.N);  // N <= 2^30

  // Diagonal metadata of every factor of the sweep, loaded in parallel once.
  for (int i = 0; i < a.n_factors; ++i)
    for (int k = threadIdx.x; k < a.fD[i]; k += NT)
      meta[a.fmeta[i] + k] = make_longlong2(a.offs[a.fdiag0[i] + k], a.rowbase[a.fdiag0[i] + k]);
  __syncthreads();

  // Stage the tile rows of factor fi's diagonals.  A row without an element on
  // a diagonal (r + d outside [0, N)) gets the value 0, so the multiply loop
  // needs no bounds test: its column is read at a valid in-tile index and
  // contributes nothing.
  auto issue_factor = [&](int fi, int stage) {
    const int D = a.fD[fi];
    const longlong2* m = meta + a.fmeta[fi];
    T2* st = stages + size_t(stage) * stage_elems;
    for (int k = 0; k < D; ++k) {
      const int d = int(m[k].x);
      const T2* vk = vals + m[k].y;
      for (uint32_t j = threadIdx.x; j < n_chunks; j += NT) {
        const uint32_t l = j * V;
        const int r = int(global_of(l, m0, m1, sh) | base);
        T2* dst_s = st + size_t(k) * TS + l;
        const bool first_ok = r + d >= 0 && r + d < N;
        const bool last_ok = r + (V - 1) + d >= 0 && r + (V - 1) + d < N;
        if (first_ok && last_ok) {
          cp_async16(dst_s, vk + r, 16);
        } else if (!first_ok && !last_ok) {
          cp_async16(dst_s, vals, 0);  // zero fill, nothing read
        } else {
#pragma unroll
          for (int e = 0; e < V; ++e) {
            const bool ok = r + e + d >= 0 && r + e + d < N;
            dst_s[e] = ok ? vk[r + e] : T2{0, 0};
          }
        }
      }
    }
  };

  const int S = a.n_stages;
  for (int s = 0; s < S; ++s) {
    if (s < a.n_factors) issue_factor(s, s);
    cp_async_commit();
  }
  // The state written by the previous launch is visible only after this.
  grid_dependency_wait();
  for (int q = 0; q < nrb; ++q) {
    const T2* sq = src + int64_t(rhs0 + q) * a.N;
    for (uint32_t j = threadIdx.x; j < n_chunks; j += NT) {
      const uint32_t l = j * V;
      cp_async16(tile + size_t(q) * TS + l, sq + (global_of(l, m0, m1, sh) | base), 16);
    }
  }
  cp_async_commit();

  uint32_t myrow[ROWS];
#pragma unroll
  for (int i = 0; i < ROWS; ++i) myrow[i] = global_of(threadIdx.x + uint32_t(i) * NT, m0, m1, sh) | base;

  for (int fi = 0; fi < a.n_factors; ++fi) {
    cp_async_wait(fi == 0 ? 0 : S - 1);
    __syncthreads();
    const int D = a.fD[fi];
    const longlong2* m = meta + a.fmeta[fi];
    const T2* st = stages + size_t(fi % S) * stage_elems + threadIdx.x;
    T2 acc[ROWS][RB];
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
#pragma unroll
      for (int q = 0; q < RB; ++q) acc[i][q] = T2{0, 0};
    for (int k = 0; k < D; ++k) {
      const int d = int(m[k].x);
#pragma unroll
      for (int i = 0; i < ROWS; ++i) {
        const T2 v = st[k * TS + i * NT];
        const uint32_t lc = local_of(uint32_t(int(myrow[i]) + d), m0, m1, sh);
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (q < nrb) cfma(acc[i][q], v, tile[q * TS + lc]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (q < nrb) tile[q * TS + threadIdx.x + i * NT] = acc[i][q];
    // Refill the stage just consumed (every thread is past the barrier above).
    if (fi + S < a.n_factors) issue_factor(fi + S, fi % S);
    cp_async_commit();
  }
  __syncthreads();

  // Store the tile.
  for (int q = 0; q < nrb; ++q) {
    T2* dq = dst + int64_t(rhs0 + q) * a.N;
    for (uint32_t j = threadIdx.x; j < n_chunks; j += NT) {
      const uint32_t l = j * V;
      *reinterpret_cast<uint4*>(dq + (global_of(l, m0, m1, sh) | base)) =
          *reinterpret_cast<const uint4*>(tile + size_t(q) * TS + l);
    }
  }
  grid_launch_dependents();
}

constexpr int kSweepMaxThreads = 256;

// Accumulators per thread (rows x states) kept in registers: 16 complex for
// complex64, 8 for complex128.
constexpr int acc_budget(hs_dtype dt) { return dt == HS_C64 ? 16 : 8; }

using SweepFn = void (*)(SweepArgs);

// Instantiation for (precision, rows per thread, rhs block); nullptr if unsupported.
template <typename R>
SweepFn sweep_fn(int rows, int rb) {
#define HS_SWEEP_CASE(RW, B) \
  if (rows == RW && rb == B) return sweep_kernel<R, RW, B>;
  HS_SWEEP_CASE(1, 1) HS_SWEEP_CASE(2, 1) HS_SWEEP_CASE(4, 1) HS_SWEEP_CASE(8, 1)
  HS_SWEEP_CASE(1, 2) HS_SWEEP_CASE(2, 2) HS_SWEEP_CASE(4, 2)
  HS_SWEEP_CASE(1, 4) HS_SWEEP_CASE(2, 4)
  HS_SWEEP_CASE(1, 8)
  if (sizeof(R) == 4) {
    HS_SWEEP_CASE(16, 1) HS_SWEEP_CASE(8, 2) HS_SWEEP_CASE(4, 4) HS_SWEEP_CASE(2, 8) HS_SWEEP_CASE(1, 16)
  }
#undef HS_SWEEP_CASE
  return nullptr;
}

}  // namespace

// Raise the dynamic shared-memory limit of every sweep instantiation once per
// device (before any launch or stream capture).
cudaError_t prepare_kernels() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && done[dev]) return cudaSuccess;
  cudaError_t r = cudaSuccess;
  for (int rows = 1; rows <= 16; rows *= 2)
    for (int rb = 1; rb <= 16; rb *= 2) {
      SweepFn f32 = sweep_fn<float>(rows, rb), f64 = sweep_fn<double>(rows, rb);
      if (f32 && r == cudaSuccess)
        r = cudaFuncSetAttribute((const void*)f32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSweepSmemMax));
      if (f64 && r == cudaSuccess)
        r = cudaFuncSetAttribute((const void*)f64, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSweepSmemMax));
    }
  if (r == cudaSuccess && dev < 64) done[dev] = true;
  return r;
}

size_t sweep_smem_bytes(hs_dtype dt, int rhs_block, int tile_bits, int stage_diags, int n_stages) {
  return (size_t(rhs_block) + size_t(stage_diags) * n_stages) * (size_t(1) << tile_bits) * elem_bytes(dt);
}

// Metadata table of a sweep: one (offset, rowbase) pair per listed diagonal.
static size_t meta_bytes(int n_meta) { return size_t(n_meta) * 16; }

int max_rows_per_thread(hs_dtype dt, int rhs_block) {
  const int r = acc_budget(dt) / rhs_block;
  return r < 1 ? 1 : r;
}

int max_tile_bits(hs_dtype dt, int rhs_block, int stage_diags, size_t budget) {
  // Largest T whose tile plus two factor stages fit the budget, with at most
  // max_rows_per_thread rows per thread at 256 threads.
  const int rows = max_rows_per_thread(dt, rhs_block);
  int t = 0;
  while (sweep_smem_bytes(dt, rhs_block, t + 1, stage_diags, 2) <= budget &&
         (1 << (t + 1)) <= kSweepMaxThreads * rows)
    ++t;
  return t;
}

cudaError_t launch_apply_plain(const hs_factors* f, int g, const void* x, void* y, int n_rhs, cudaStream_t s) {
  const Plan& p = f->plan;
  const Group& G = p.groups[g];
  const int threads = 256;
  int64_t blocks = (p.N + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const int64_t* offs = f->d_offs + G.diag0;
  const int64_t* rb = f->d_rowbase + G.diag0;
  if (f->dtype == HS_C64) {
    auto v = reinterpret_cast<const float2*>(f->d_vals);
    if (n_rhs >= 4)
      apply_plain_kernel<float, 4><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, (const float2*)x, (float2*)y, p.N, n_rhs);
    else
      apply_plain_kernel<float, 1><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, (const float2*)x, (float2*)y, p.N, n_rhs);
  } else {
    auto v = reinterpret_cast<const double2*>(f->d_vals);
    if (n_rhs >= 4)
      apply_plain_kernel<double, 4><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, (const double2*)x, (double2*)y, p.N, n_rhs);
    else
      apply_plain_kernel<double, 1><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, (const double2*)x, (double2*)y, p.N, n_rhs);
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep(const hs_factors* f, const SweepLaunch& L, cudaStream_t s) {
  const Plan& p = f->plan;
  SweepArgs a;
  a.src = L.src;
  a.dst = L.dst;
  a.vals = f->d_vals;
  a.offs = f->d_offs;
  a.rowbase = f->d_rowbase;
  a.N = p.N;
  a.n_rhs = L.n_rhs;
  a.rhs_block = L.rhs_block;
  a.tile_bits = L.tile_bits;
  a.n_tiles_log2 = p.n_qubits - L.tile_bits;
  // Split the two-run local mask into [0, lo) and [h, h + w).
  const uint32_t lm = L.local_mask;
  int lo = 0;
  while (lo < 32 && ((lm >> lo) & 1u)) ++lo;
  const uint32_t hi = lo < 32 ? (lm & ~((1u << lo) - 1u)) : 0u;
  const int w = __builtin_popcount(hi);
  const int h = hi ? __builtin_ctz(hi) : lo;
  if (lo + w != L.tile_bits || (hi && hi != (((1u << w) - 1u) << h))) return cudaErrorInvalidValue;
  a.m0 = lo >= 32 ? 0xffffffffu : ((1u << lo) - 1u);
  a.m1 = ((1u << w) - 1u) << lo;
  a.sh = h - lo;
  a.rest = L.rest;
  a.n_factors = L.n_factors;
  int dmax = 1, n_meta = 0;
  for (int i = 0; i < L.n_factors; ++i) {
    const Group& G = p.groups[L.factors[i]];
    a.fdiag0[i] = G.diag0;
    a.fD[i] = int16_t(G.D);
    a.fmeta[i] = int16_t(n_meta);
    n_meta += G.D;
    dmax = G.D > dmax ? G.D : dmax;
  }
  if (n_meta > 32767) return cudaErrorInvalidValue;
  a.n_meta = n_meta;
  a.stage_diags = dmax;
  // As many stages (<= 8, <= n_factors) as the shared-memory budget allows.
  int S = 1;
  while (S < 8 && S < L.n_factors &&
         meta_bytes(n_meta) + sweep_smem_bytes(f->dtype, L.rhs_block, L.tile_bits, dmax, S + 1) <= L.smem_budget)
    ++S;
  a.n_stages = S;
  const size_t smem = meta_bytes(n_meta) + sweep_smem_bytes(f->dtype, L.rhs_block, L.tile_bits, dmax, S);
  if (smem > kSweepSmemMax || L.tile_bits > p.n_qubits) return cudaErrorInvalidValue;
  const int TS = 1 << L.tile_bits;
  const int rows = TS > kSweepMaxThreads ? TS / kSweepMaxThreads : 1;
  const int threads = TS / rows;
  const bool c64 = f->dtype == HS_C64;
  if (TS < (c64 ? 2 : 1)) return cudaErrorInvalidValue;
  SweepFn fn = c64 ? sweep_fn<float>(rows, L.rhs_block) : sweep_fn<double>(rows, L.rhs_block);
  if (!fn) return cudaErrorInvalidValue;
  const int n_rhs_blocks = (L.n_rhs + L.rhs_block - 1) / L.rhs_block;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned((1 << a.n_tiles_log2) * n_rhs_blocks), 1u, 1u);
  cfg.blockDim = dim3(unsigned(threads), 1u, 1u);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = L.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fn, a);
}

}  // namespace hs
