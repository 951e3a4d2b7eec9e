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
  const uint32_t* slot_u;
  const int32_t* slot_tab;
  const int64_t* tab_rb;
  int64_t N;
  int n_rhs;
  int rhs_block;
  int tile_bits;
  int n_tiles_log2;
  int n_stages;      // factor stages in the shared-memory ring
  int stage_planes;  // planes per stage (max slot count over the sweep's factors)
  int n_mslot;       // slots listed in the shared-memory slot table
  int n_mtab;        // entries in the shared-memory row-base table
  // Local bits [0, a) U [h, h + w): local index of row r is
  // (r & m0) | ((r >> sh) & m1), with m0 = 2^a - 1, m1 = (2^w - 1) << a, sh = h - a.
  uint32_t m0, m1;
  int sh;
  Runs rest;         // the other bits, enumerated by the CTA index
  int n_factors;
  // Per factor of the sweep: first global slot, slot count, position of its
  // first slot in the shared slot table, first global / shared row-base table
  // entry and the number of entries.
  int fslot0[kMaxSweepFactors];
  int ftab_g[kMaxSweepFactors];
  int16_t fnslot[kMaxSweepFactors];
  int16_t fmslot[kMaxSweepFactors];
  int16_t ftab_s[kMaxSweepFactors];
  int16_t ftab_n[kMaxSweepFactors];
};

struct SlotMeta {
  uint32_t u;    // x-mask of the slot
  uint32_t U;    // its local image (u lies inside the tile's local bits)
  int32_t tab;   // first row-base table entry in shared memory
  int32_t pad;
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
// Bits of r at the set bits of u, packed (lowest set bit of u -> bit 0).
__device__ __forceinline__ uint32_t pattern_of(uint32_t r, uint32_t u) {
  uint32_t p = 0;
  int j = 0;
  for (uint32_t t = u; t; t &= t - 1u, ++j) p |= ((r >> (__ffs(t) - 1)) & 1u) << j;
  return p;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
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

// The factor loop of a sweep.  NRB = RB when the CTA's block of states is
// full (no per-state guard), 0 for the last, partial block.
template <typename T2, int ROWS, int RB, int NRB, typename Issue>
__device__ __forceinline__ void sweep_body(const SweepArgs& a, T2* tile, const T2* stages, uint32_t stage_elems,
                                           const SlotMeta* mslot, uint32_t TS, int NT, Issue& issue_factor) {
  const int rhs0 = int(blockIdx.x >> a.n_tiles_log2) * a.rhs_block;
  const int nrb = NRB ? NRB : min(a.rhs_block, a.n_rhs - rhs0);
  const int S = a.n_stages;
  for (int fi = 0; fi < a.n_factors; ++fi) {
    cp_async_wait(fi == 0 ? 0 : S - 1);
    __syncthreads();
    const int ns = a.fnslot[fi];
    const SlotMeta* ms = mslot + a.fmslot[fi];
    const T2* st = stages + size_t(fi % S) * stage_elems + threadIdx.x;
    T2 acc[ROWS][RB];
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
#pragma unroll
      for (int q = 0; q < RB; ++q) acc[i][q] = T2{0, 0};
#pragma unroll 2
    for (int j = 0; j < ns; ++j) {
      const uint32_t U = ms[j].U;
#pragma unroll
      for (int i = 0; i < ROWS; ++i) {
        const T2 v = st[j * TS + i * NT];
        const T2* xp = tile + ((threadIdx.x + uint32_t(i) * NT) ^ U);
#pragma unroll
        for (int q = 0; q < RB; ++q, xp += TS)
          if (NRB || q < nrb) cfma(acc[i][q], v, *xp);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
      T2* yp = tile + threadIdx.x + i * NT;
#pragma unroll
      for (int q = 0; q < RB; ++q, yp += TS)
        if (NRB || q < nrb) *yp = acc[i][q];
    }
    // Refill the stage just consumed (every thread is past the barrier above).
    if (fi + S < a.n_factors) issue_factor(fi + S, fi % S);
    cp_async_commit();
  }
  __syncthreads();
}

// Block of TS / ROWS threads; thread t owns local rows t + i * blockDim.x.
//
// For a factor whose x-mask set X lies in the local bits, row r of the factor
// has exactly one structural entry per u in X, in column r ^ u (always inside
// [0, N) and inside the tile); every other stored value on that row is an
// exact zero.  The sweep therefore stages, for every slot u and tile row, the
// value of entry (r, r ^ u) -- element min(r, r ^ u) of diagonal (r ^ u) - r,
// found through the slot's row-base table -- into plane u of the stage, and
// the multiply is acc[l] += plane_u[l] * x[l ^ U] with U the local image of u.
// The sum is the diagonal-times-vector product without its zero terms.
template <typename R, int ROWS, int RB>
__global__ void __launch_bounds__(512) sweep_kernel(const __grid_constant__ SweepArgs a) {
  using T2 = typename C2<R>::T;
  constexpr int V = 16 / sizeof(T2);  // elements per 16-byte chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  const uint32_t TS = 1u << a.tile_bits;
  const uint32_t m0 = a.m0, m1 = a.m1;
  const int sh = a.sh;
  // Shared memory: [slot table][row-base table][tile][factor stages]
  SlotMeta* mslot = reinterpret_cast<SlotMeta*>(smem_raw);
  int64_t* mtab = reinterpret_cast<int64_t*>(mslot + a.n_mslot);
  T2* tile = reinterpret_cast<T2*>(mtab + ((a.n_mtab + 1) & ~1));
  T2* stages = tile + size_t(a.rhs_block) * TS;
  const uint32_t stage_elems = uint32_t(a.stage_planes) * TS;
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

  // Slot and row-base tables of every factor of the sweep, loaded once.
  for (int i = 0; i < a.n_factors; ++i) {
    for (int j = threadIdx.x; j < a.fnslot[i]; j += NT) {
      const uint32_t u = a.slot_u[a.fslot0[i] + j];
      mslot[a.fmslot[i] + j] = SlotMeta{u, local_of(u, m0, m1, sh), a.ftab_s[i] + (a.slot_tab[a.fslot0[i] + j] - a.ftab_g[i]), 0};
    }
    for (int e = threadIdx.x; e < a.ftab_n[i]; e += NT) mtab[a.ftab_s[i] + e] = a.tab_rb[a.ftab_g[i] + e];
  }
  __syncthreads();

  // Stage plane u of factor fi for the tile rows.
  auto issue_factor = [&](int fi, int stage) {
    const int ns = a.fnslot[fi];
    T2* st = stages + size_t(stage) * stage_elems;
    for (int j = 0; j < ns; ++j) {
      const SlotMeta m = mslot[a.fmslot[fi] + j];
      const int64_t* tab = mtab + m.tab;
      T2* plane = st + size_t(j) * TS;
      if (V == 1 || !(m.u & 1u)) {
        for (uint32_t c = threadIdx.x; c < n_chunks; c += NT) {
          const uint32_t l = c * V;
          const uint32_t r = global_of(l, m0, m1, sh) | base;
          cp_async16(plane + l, vals + tab[pattern_of(r, m.u)] + r);
        }
      } else {
        // u flips bit 0: the two rows of a 16-byte chunk lie on different diagonals.
        for (uint32_t c = threadIdx.x; c < n_chunks; c += NT) {
          const uint32_t l = c * V;
          const uint32_t r = global_of(l, m0, m1, sh) | base;
          const uint32_t p0 = pattern_of(r, m.u);  // bit 0 of r is 0
          cp_async8(plane + l, vals + tab[p0] + r);
          cp_async8(plane + l + 1, vals + tab[p0 | 1u] + r + 1);
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
  // Let the next sweep start its own prologue (tables and factor staging, which
  // read no state) while this one computes; it waits for this grid to finish
  // before it touches the state.
  grid_launch_dependents();
  for (uint32_t c = threadIdx.x; c < n_chunks; c += NT) {
    const uint32_t l = c * V;
    const T2* sp = src + int64_t(rhs0) * a.N + (global_of(l, m0, m1, sh) | base);
    T2* tp = tile + l;
    for (int q = 0; q < nrb; ++q, sp += a.N, tp += TS) cp_async16(tp, sp);
  }
  cp_async_commit();

  if (nrb == RB)
    sweep_body<T2, ROWS, RB, RB>(a, tile, stages, stage_elems, mslot, TS, NT, issue_factor);
  else
    sweep_body<T2, ROWS, RB, 0>(a, tile, stages, stage_elems, mslot, TS, NT, issue_factor);

  // Store the tile.
  for (uint32_t c = threadIdx.x; c < n_chunks; c += NT) {
    const uint32_t l = c * V;
    T2* dp = dst + int64_t(rhs0) * a.N + (global_of(l, m0, m1, sh) | base);
    const T2* tp = tile + l;
    for (int q = 0; q < nrb; ++q, dp += a.N, tp += TS)
      *reinterpret_cast<uint4*>(dp) = *reinterpret_cast<const uint4*>(tp);
  }
}

constexpr int kSweepMaxThreads = 512;

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

size_t sweep_smem_bytes(hs_dtype dt, int rhs_block, int tile_bits, int stage_planes, int n_stages) {
  return (size_t(rhs_block) + size_t(stage_planes) * n_stages) * (size_t(1) << tile_bits) * elem_bytes(dt);
}

// Slot and row-base tables of a sweep in shared memory.
static size_t meta_bytes(int n_mslot, int n_mtab) { return size_t(n_mslot) * 16 + size_t((n_mtab + 1) & ~1) * 8; }

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
  a.slot_u = f->d_slot_u;
  a.slot_tab = f->d_slot_tab;
  a.tab_rb = f->d_tab_rb;
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
  int planes = 1, n_mslot = 0, n_mtab = 0;
  for (int i = 0; i < L.n_factors; ++i) {
    const Group& G = p.groups[L.factors[i]];
    if (G.nslot <= 0) return cudaErrorInvalidValue;
    const int t0 = p.slot_tab[G.slot0], t1 = p.slot_tab[G.slot0 + G.nslot];
    a.fslot0[i] = G.slot0;
    a.fnslot[i] = int16_t(G.nslot);
    a.fmslot[i] = int16_t(n_mslot);
    a.ftab_g[i] = t0;
    a.ftab_s[i] = int16_t(n_mtab);
    a.ftab_n[i] = int16_t(t1 - t0);
    n_mslot += G.nslot;
    n_mtab += t1 - t0;
    planes = G.nslot > planes ? G.nslot : planes;
  }
  if (n_mslot > 32767 || n_mtab > 32767) return cudaErrorInvalidValue;
  a.n_mslot = n_mslot;
  a.n_mtab = n_mtab;
  a.stage_planes = planes;
  const size_t mb = meta_bytes(n_mslot, n_mtab);
  // As many stages (<= 8, <= n_factors) as the shared-memory budget allows.
  int S = 1;
  while (S < 8 && S < L.n_factors &&
         mb + sweep_smem_bytes(f->dtype, L.rhs_block, L.tile_bits, planes, S + 1) <= L.smem_budget)
    ++S;
  a.n_stages = S;
  const size_t smem = mb + sweep_smem_bytes(f->dtype, L.rhs_block, L.tile_bits, planes, S);
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
