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
  const int* fac_D;
  const int* fac_diag0;
  int64_t N;
  int n_rhs;
  int rhs_block;
  int tile_bits;
  int n_tiles_log2;
  int n_stages;      // factor stages in the shared-memory ring
  int stage_diags;   // diagonals per stage (max D over the sweep's factors)
  int n_meta;        // diagonals listed in the shared-memory metadata table
  Runs local, rest;
  int n_factors;
  // Per factor of the sweep: first diagonal in the global diagonal arrays,
  // diagonal count, and position of its first diagonal in the metadata table.
  int fdiag0[kMaxSweepFactors];
  int16_t fD[kMaxSweepFactors];
  int16_t fmeta[kMaxSweepFactors];
};

// Scatter the low bits of v into the positions of the runs.
__device__ __forceinline__ uint32_t deposit(uint32_t v, const Runs& R) {
  uint32_t out = 0;
  int q = 0;
#pragma unroll
  for (int i = 0; i < kMaxRuns + 2; ++i) {
    if (i < R.n) {
      out |= ((v >> q) & ((1u << R.len[i]) - 1u)) << R.pos[i];
      q += R.len[i];
    }
  }
  return out;
}

// Gather the bits of c at the runs' positions into the low bits.
__device__ __forceinline__ uint32_t extract(uint32_t c, const Runs& R) {
  uint32_t out = 0;
  int q = 0;
#pragma unroll
  for (int i = 0; i < kMaxRuns + 2; ++i) {
    if (i < R.n) {
      out |= ((c >> R.pos[i]) & ((1u << R.len[i]) - 1u)) << q;
      q += R.len[i];
    }
  }
  return out;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
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

template <typename R, int NT, int MAXROWS, int RB>
__global__ void __launch_bounds__(NT) sweep_kernel(const __grid_constant__ SweepArgs a) {
  using T2 = typename C2<R>::T;
  constexpr int V = 16 / sizeof(T2);  // elements per 16-byte chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t TS = 1u << a.tile_bits;
  // Shared memory: [diagonal metadata (offset, rowbase)][tile][factor stages]
  longlong2* meta = reinterpret_cast<longlong2*>(smem_raw);
  T2* tile = reinterpret_cast<T2*>(smem_raw + size_t(a.n_meta) * sizeof(longlong2));
  T2* stages = tile + size_t(a.rhs_block) * TS;
  const size_t stage_elems = size_t(a.stage_diags) * TS;
  // src and dst may be the same buffer (in-place sweep): every CTA reads its
  // own tile completely before it writes it back, and tiles are disjoint.
  const T2* src = reinterpret_cast<const T2*>(a.src);
  T2* dst = reinterpret_cast<T2*>(a.dst);
  const T2* __restrict__ vals = reinterpret_cast<const T2*>(a.vals);

  const uint32_t tile_id = blockIdx.x & ((1u << a.n_tiles_log2) - 1u);
  const int rhs0 = int(blockIdx.x >> a.n_tiles_log2) * a.rhs_block;
  const int nrb = min(a.rhs_block, a.n_rhs - rhs0);
  const uint32_t base = deposit(tile_id, a.rest);
  const uint32_t n_chunks = TS / V;

  // Diagonal metadata of every factor of the sweep, loaded in parallel once.
  for (int i = 0; i < a.n_factors; ++i)
    for (int k = threadIdx.x; k < a.fD[i]; k += NT)
      meta[a.fmeta[i] + k] = make_longlong2(a.offs[a.fdiag0[i] + k], a.rowbase[a.fdiag0[i] + k]);
  __syncthreads();

  // Stage the tile rows of factor fi's diagonals (16-byte chunks; a chunk is
  // skipped when none of its rows has an element on that diagonal).
  auto issue_factor = [&](int fi, int stage) {
    const int D = a.fD[fi];
    const longlong2* m = meta + a.fmeta[fi];
    T2* st = stages + size_t(stage) * stage_elems;
    for (int k = 0; k < D; ++k) {
      const longlong2 dk = m[k];
      const T2* vk = vals + dk.y;
      for (uint32_t j = threadIdx.x; j < n_chunks; j += NT) {
        const uint32_t l = j * V;
        const int64_t r = int64_t(deposit(l, a.local) | base);
        if (r + (V - 1) + dk.x >= 0 && r + dk.x < a.N) cp_async16(st + size_t(k) * TS + l, vk + r);
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
      cp_async16(tile + size_t(q) * TS + l, sq + (deposit(l, a.local) | base));
    }
  }
  cp_async_commit();

  uint32_t myrow[MAXROWS];
  bool valid[MAXROWS];
#pragma unroll
  for (int i = 0; i < MAXROWS; ++i) {
    const uint32_t l = threadIdx.x + uint32_t(i) * NT;
    valid[i] = l < TS;
    myrow[i] = valid[i] ? (deposit(l, a.local) | base) : 0u;
  }

  for (int fi = 0; fi < a.n_factors; ++fi) {
    cp_async_wait(fi == 0 ? 0 : S - 1);
    __syncthreads();
    const int D = a.fD[fi];
    const longlong2* m = meta + a.fmeta[fi];
    const T2* st = stages + size_t(fi % S) * stage_elems;
    T2 acc[MAXROWS][RB];
#pragma unroll
    for (int i = 0; i < MAXROWS; ++i)
#pragma unroll
      for (int q = 0; q < RB; ++q) acc[i][q] = T2{0, 0};
    for (int k = 0; k < D; ++k) {
      const int64_t d = m[k].x;
#pragma unroll
      for (int i = 0; i < MAXROWS; ++i) {
        const int64_t c = int64_t(myrow[i]) + d;
        if (valid[i] && c >= 0 && c < a.N) {
          const T2 v = st[size_t(k) * TS + threadIdx.x + i * NT];
          const uint32_t lc = extract(uint32_t(c), a.local);
#pragma unroll
          for (int q = 0; q < RB; ++q)
            if (q < nrb) cfma(acc[i][q], v, tile[size_t(q) * TS + lc]);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXROWS; ++i)
      if (valid[i])
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (q < nrb) tile[size_t(q) * TS + threadIdx.x + i * NT] = acc[i][q];
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
      *reinterpret_cast<uint4*>(dq + (deposit(l, a.local) | base)) =
          *reinterpret_cast<const uint4*>(tile + size_t(q) * TS + l);
    }
  }
  grid_launch_dependents();
}

constexpr int kSweepThreads = 256;

// Accumulators per thread (rows x states) kept in registers: 16 complex for
// complex64, 8 for complex128.
template <typename R> constexpr int acc_budget() { return sizeof(R) == 4 ? 16 : 8; }
constexpr int max_rows(hs_dtype dt, int rb) { return (dt == HS_C64 ? 16 : 8) / rb < 1 ? 1 : (dt == HS_C64 ? 16 : 8) / rb; }

template <typename R, int RB>
constexpr auto sweep_fn() {
  constexpr int MR = acc_budget<R>() / RB < 1 ? 1 : acc_budget<R>() / RB;
  return sweep_kernel<R, kSweepThreads, MR, RB>;
}

template <typename R, int RB>
cudaError_t launch_sweep_t(const SweepArgs& a, int n_blocks, size_t smem, bool pdl, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(n_blocks), 1u, 1u);
  cfg.blockDim = dim3(unsigned(kSweepThreads), 1u, 1u);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, sweep_fn<R, RB>(), a);
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
  const int b = int(kSweepSmemMax);
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t r = cudaSuccess;
  auto set = [&](const void* fn) { if (r == cudaSuccess) r = cudaFuncSetAttribute(fn, A, b); };
  set((const void*)sweep_fn<float, 1>());
  set((const void*)sweep_fn<float, 2>());
  set((const void*)sweep_fn<float, 4>());
  set((const void*)sweep_fn<float, 8>());
  set((const void*)sweep_fn<float, 16>());
  set((const void*)sweep_fn<double, 1>());
  set((const void*)sweep_fn<double, 2>());
  set((const void*)sweep_fn<double, 4>());
  set((const void*)sweep_fn<double, 8>());
  if (r == cudaSuccess && dev < 64) done[dev] = true;
  return r;
}

size_t sweep_smem_bytes(hs_dtype dt, int rhs_block, int tile_bits, int stage_diags, int n_stages) {
  return (size_t(rhs_block) + size_t(stage_diags) * n_stages) * (size_t(1) << tile_bits) * elem_bytes(dt);
}

// Metadata table of a sweep: one (offset, rowbase) pair per listed diagonal.
static size_t meta_bytes(int n_meta) { return size_t(n_meta) * 16; }

int max_rows_per_thread(hs_dtype dt, int rhs_block) { return max_rows(dt, rhs_block); }

int max_tile_bits(hs_dtype dt, int rhs_block, int stage_diags, size_t budget) {
  // Largest T whose tile plus two factor stages fit the budget, with at most
  // max_rows rows per thread.
  const int rows = max_rows(dt, rhs_block);
  int t = 0;
  while (sweep_smem_bytes(dt, rhs_block, t + 1, stage_diags, 2) <= budget && (1 << (t + 1)) <= kSweepThreads * rows)
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
  a.fac_D = f->d_fac_D;
  a.fac_diag0 = f->d_fac_diag0;
  a.N = p.N;
  a.n_rhs = L.n_rhs;
  a.rhs_block = L.rhs_block;
  a.tile_bits = L.tile_bits;
  a.n_tiles_log2 = p.n_qubits - L.tile_bits;
  a.local = L.local;
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
  const int rows = max_rows(f->dtype, L.rhs_block);
  if ((1 << L.tile_bits) > kSweepThreads * rows) return cudaErrorInvalidValue;
  if (L.tile_bits < (f->dtype == HS_C64 ? 1 : 0)) return cudaErrorInvalidValue;
  const int n_rhs_blocks = (L.n_rhs + L.rhs_block - 1) / L.rhs_block;
  const int n_blocks = (1 << a.n_tiles_log2) * n_rhs_blocks;
  const bool c64 = f->dtype == HS_C64;
  switch (L.rhs_block) {
    case 1: return c64 ? launch_sweep_t<float, 1>(a, n_blocks, smem, L.pdl, s) : launch_sweep_t<double, 1>(a, n_blocks, smem, L.pdl, s);
    case 2: return c64 ? launch_sweep_t<float, 2>(a, n_blocks, smem, L.pdl, s) : launch_sweep_t<double, 2>(a, n_blocks, smem, L.pdl, s);
    case 4: return c64 ? launch_sweep_t<float, 4>(a, n_blocks, smem, L.pdl, s) : launch_sweep_t<double, 4>(a, n_blocks, smem, L.pdl, s);
    case 8: return c64 ? launch_sweep_t<float, 8>(a, n_blocks, smem, L.pdl, s) : launch_sweep_t<double, 8>(a, n_blocks, smem, L.pdl, s);
    case 16: return c64 ? launch_sweep_t<float, 16>(a, n_blocks, smem, L.pdl, s) : cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hs
