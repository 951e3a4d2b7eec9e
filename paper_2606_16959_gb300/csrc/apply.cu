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

#include "counters.h"
#include "hs_internal.h"
#include "sweep_core.cuh"

namespace hs {
namespace {

using sweep::C2;
using sweep::cfma;
using sweep::SweepArgs;
using sweep::meta_bytes;

// ---------------------------------------------------------------------------
// Plain row-parallel diagonal-times-vector product.
// ---------------------------------------------------------------------------
template <typename R, int RB>
__global__ void __launch_bounds__(256) apply_plain_kernel(const typename C2<R>::T* __restrict__ vals,
                                                          const int64_t* __restrict__ offs,
                                                          const int64_t* __restrict__ rowbase, int D,
                                                          const typename C2<R>::T* __restrict__ x,
                                                          typename C2<R>::T* __restrict__ y, int64_t N, int n_rhs,
                                                          int64_t n_vals) {
  using T2 = typename C2<R>::T;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < N; r += int64_t(gridDim.x) * blockDim.x) {
    for (int q0 = 0; q0 < n_rhs; q0 += RB) {
      T2 acc[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) acc[q] = T2{0, 0};
      for (int k = 0; k < D; ++k) {
        const int64_t c = r + offs[k];
        if (c < 0 || c >= N) continue;
        const T2 v = vals[HS_BCHK(rowbase[k] + r, n_vals, BS_PLAIN_VAL)];
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (q0 + q < n_rhs) cfma(acc[q], v, x[HS_BCHK(int64_t(q0 + q) * N + c, int64_t(n_rhs) * N, BS_PLAIN_X)]);
      }
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (q0 + q < n_rhs) y[int64_t(q0 + q) * N + r] = acc[q];
    }
  }
}

template <typename R, int ROWS, int RB>
__global__ void __launch_bounds__(512) sweep_kernel(const __grid_constant__ sweep::SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t u0 = blockIdx.x * uint32_t(a.tiles_per_cta);
  const uint32_t u1 = min(uint32_t(a.n_units), u0 + uint32_t(a.tiles_per_cta));
  sweep::sweep_tiles<R, ROWS, RB, RB == 1>(a, u0, u1, smem_raw);
}

constexpr int kSweepMaxThreads = 512;
constexpr int kSweepMaxTilesPerCta = 8;

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
  // States per pass: the factor's values are read once per block of RB
  // states, so the block is as large as the accumulators allow.
  if (f->dtype == HS_C64) {
    auto v = reinterpret_cast<const float2*>(f->d_vals);
    auto xs = static_cast<const float2*>(x);
    auto ys = static_cast<float2*>(y);
    if (n_rhs >= 16)
      apply_plain_kernel<float, 16><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, xs, ys, p.N, n_rhs, p.total_elems);
    else if (n_rhs >= 8)
      apply_plain_kernel<float, 8><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, xs, ys, p.N, n_rhs, p.total_elems);
    else if (n_rhs >= 4)
      apply_plain_kernel<float, 4><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, xs, ys, p.N, n_rhs, p.total_elems);
    else
      apply_plain_kernel<float, 1><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, xs, ys, p.N, n_rhs, p.total_elems);
  } else {
    auto v = reinterpret_cast<const double2*>(f->d_vals);
    auto xs = static_cast<const double2*>(x);
    auto ys = static_cast<double2*>(y);
    if (n_rhs >= 8)
      apply_plain_kernel<double, 8><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, xs, ys, p.N, n_rhs, p.total_elems);
    else if (n_rhs >= 4)
      apply_plain_kernel<double, 4><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, xs, ys, p.N, n_rhs, p.total_elems);
    else
      apply_plain_kernel<double, 1><<<blocks, threads, 0, s>>>(v, offs, rb, G.D, xs, ys, p.N, n_rhs, p.total_elems);
  }
  note_launches();
  return cudaGetLastError();
}

cudaError_t launch_sweep(const hs_factors* f, const SweepLaunch& L, cudaStream_t s) {
  const Plan& p = f->plan;
  SweepArgs a;
  a.src = L.src;
  a.dst = L.dst;
  a.vals = f->d_vals;
  a.vt = f->d_vt;
  a.slot_u = f->d_slot_u;
  a.slot_tab = f->d_slot_tab;
  a.tab_rb = f->d_tab_rb;
  a.N = p.N;
  a.n_vals = p.total_elems;
  a.n_vt_g = p.total_vt;
  a.n_slot_g = int(p.slot_u.size());
  a.n_tab_g = int(p.tab_rb.size());
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
  int planes = 1, n_mslot = 0, n_mtab = 0, n_vt = 0;
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
    a.fvts[i] = int16_t(n_vt);
    const bool table = L.value_tables && G.vt0 >= 0 && n_vt + G.vt_n <= kMaxVtSweep;
    a.fvt[i] = table ? G.vt0 : -1;
    a.fsm[i] = table ? G.smask : 0u;
    a.fsh[i] = sweep::pattern_shift(a.fsm[i]);
    if (table) n_vt += G.vt_n;
    n_mslot += G.nslot;
    n_mtab += t1 - t0;
    if (!table) planes = G.nslot > planes ? G.nslot : planes;
  }
  if (n_mslot > 32767 || n_mtab > 32767) return cudaErrorInvalidValue;
  a.n_mslot = n_mslot;
  a.n_mtab = n_mtab;
  a.n_vt = n_vt;
  a.stage_planes = planes;
  // Register path: every factor from a value table, one row per thread, one
  // state per tile; lane-only factors are those whose slots' local images are
  // below 32 (lane bits of the thread's row).
  a.all_tables = 0;
  a.flane = 0;
  const size_t mb = meta_bytes(n_mslot, n_mtab, n_vt, elem_bytes(f->dtype));
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
  // (The path's second exchange buffer is the stage ring, which holds at least
  // one plane of a whole tile.)
  if (L.rhs_block == 1 && threads >= 32) {
    bool all = n_vt > 0;
    for (int i = 0; i < L.n_factors; ++i) {
      if (a.fvt[i] < 0) { all = false; break; }
      const Group& G = p.groups[L.factors[i]];
      bool lane = true;
      for (int sl = 0; sl < G.nslot; ++sl) {
        const uint32_t u = p.slot_u[G.slot0 + sl];
        const uint32_t U = (u & a.m0) | ((u >> a.sh) & a.m1);
        if ((U & uint32_t(threads - 1)) >= 32u) lane = false;
      }
      if (lane) a.flane |= 1ull << i;
    }
    a.all_tables = all ? 1 : 0;
  }
  const bool c64 = f->dtype == HS_C64;
  if (TS < (c64 ? 2 : 1)) return cudaErrorInvalidValue;
  SweepFn fn = c64 ? sweep_fn<float>(rows, L.rhs_block) : sweep_fn<double>(rows, L.rhs_block);
  if (!fn) return cudaErrorInvalidValue;
  const int n_rhs_blocks = (L.n_rhs + L.rhs_block - 1) / L.rhs_block;
  cudaLaunchConfig_t cfg = {};
  // One-state tiles: several units per CTA once the grid is large (tables
  // loaded once per CTA), keeping at least ~16 CTAs per SM.  A multi-state
  // tile already carries enough work for its tables (measured: 8 units per
  // CTA slowed the 16-state MaxCut sweeps by 12%).
  a.n_units = (1 << a.n_tiles_log2) * n_rhs_blocks;
  a.tiles_per_cta =
      L.rhs_block == 1 ? std::max(1, std::min(kSweepMaxTilesPerCta, a.n_units / (152 * 16))) : 1;
  cfg.gridDim = dim3(unsigned((a.n_units + a.tiles_per_cta - 1) / a.tiles_per_cta), 1u, 1u);
  cfg.blockDim = dim3(unsigned(threads), 1u, 1u);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = L.pdl ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fn, a);
  if (e == cudaSuccess) note_launches();
  return e;
}

}  // namespace hs
