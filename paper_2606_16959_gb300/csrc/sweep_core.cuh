// Shared device code of the fused tile sweep (per-sweep launches in apply.cu
// and batched launches in batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bounds.cuh"
#include "hs_internal.h"

namespace hs {
namespace sweep {

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
// Fused tile sweep.
// ---------------------------------------------------------------------------
struct SweepArgs {
  const void* src;
  void* dst;
  const void* vals;
  const void* vt;    // the factor set's value tables
  const uint32_t* slot_u;
  const int32_t* slot_tab;
  const int64_t* tab_rb;
  int64_t N;
  // Extents of vals, vt, slot_u / slot_tab and tab_rb (index checks only).
  int64_t n_vals, n_vt_g;
  int n_slot_g, n_tab_g;
  int n_rhs;
  int rhs_block;
  int tile_bits;
  int n_tiles_log2;
  int n_stages;      // factor stages in the shared-memory ring
  int stage_planes;  // planes per stage (max slot count over the sweep's factors)
  int n_mslot;       // slots listed in the shared-memory slot table
  int n_mtab;        // entries in the shared-memory row-base table
  int n_vt;          // value-table entries held in shared memory
  // Local bits [0, a) U [h, h + w): local index of row r is
  // (r & m0) | ((r >> sh) & m1), with m0 = 2^a - 1, m1 = (2^w - 1) << a, sh = h - a.
  uint32_t m0, m1;
  int sh;
  Runs rest;         // the other bits, enumerated by the CTA index
  int n_factors;
  int tiles_per_cta;  // units one CTA of a per-sweep launch runs back to back
  int n_units;        // 2^n_tiles_log2 * rhs blocks
  // Per factor of the sweep: first global slot, slot count, position of its
  // first slot in the shared slot table, first global / shared row-base table
  // entry and the number of entries.
  int fslot0[kMaxSweepFactors];
  int ftab_g[kMaxSweepFactors];
  int16_t fnslot[kMaxSweepFactors];
  int16_t fmslot[kMaxSweepFactors];
  int16_t ftab_s[kMaxSweepFactors];
  int16_t ftab_n[kMaxSweepFactors];
  // Value tables: first global entry of the factor's table (-1: the factor is
  // staged from its diagonals instead), first shared entry (a running prefix,
  // so factors without a table repeat the next factor's start) and the bit
  // mask whose bits of a row index the table.
  int fvt[kMaxSweepFactors];
  int16_t fvts[kMaxSweepFactors];
  uint32_t fsm[kMaxSweepFactors];
  int8_t fsh[kMaxSweepFactors];  // lowest bit of fsm when its bits are consecutive, else -1
  // Register path (one row per thread, one state per tile, every factor from a
  // value table): bit i of flane set when factor i's slots flip only local
  // bits 0..4, i.e. exchange amplitudes within a warp.
  int all_tables;
  uint64_t flane;
};

struct SlotMeta {
  uint32_t u;    // x-mask of the slot
  uint32_t U;    // its local image (u lies inside the tile's local bits)
  int32_t tab;   // first row-base table entry in shared memory
  int32_t pos;   // plane position in the stage ring (factors staged by the prologue); -1: value table
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
// The same with sh = the lowest bit of u when u's bits are consecutive (a
// shift and a mask), -1 otherwise.
__device__ __forceinline__ uint32_t pattern_fast(uint32_t r, uint32_t u, int sh) {
  return sh >= 0 ? (r & u) >> sh : pattern_of(r, u);
}
// Host side: the shift pattern_fast takes for mask u.
inline int8_t pattern_shift(uint32_t u) {
  if (!u) return 0;
  const int lo = __builtin_ctz(u);
  const uint32_t w = u >> lo;
  return (w & (w + 1u)) == 0 ? int8_t(lo) : int8_t(-1);
}

// The copies carry no memory clobber: shared memory they write is read only
// after cp.async.wait_group and a barrier, which do.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
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
// full (no per-state guard), 0 for the last, partial block.  grow[i] is the
// global index of the thread's local row threadIdx.x + i * NT; vts holds the
// sweep's value tables.
template <typename T2, int ROWS, int RB, int NRB, typename Issue>
__device__ __forceinline__ void sweep_body(const SweepArgs& a, int nrb, T2* tile, const T2* stages, uint32_t stage_elems,
                                           const SlotMeta* mslot, const T2* vts, const uint32_t (&grow)[ROWS],
                                           uint32_t TS, int NT, Issue& issue_factor) {
  const int S = a.n_stages;
  int stage = 0;  // fi % S
  for (int fi = 0; fi < a.n_factors; ++fi) {
    cp_async_wait(fi == 0 ? 0 : S - 1);
    __syncthreads();
    const int ns = a.fnslot[fi];
    const SlotMeta* ms = mslot + a.fmslot[fi];
    T2 acc[ROWS][RB];
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
#pragma unroll
      for (int q = 0; q < RB; ++q) acc[i][q] = T2{0, 0};
    // acc[i][q] += v(j, i) * x[q][row_i ^ U_j] over the factor's slots j.
    auto multiply = [&](auto value_of) {
#pragma unroll 2
      for (int j = 0; j < ns; ++j) {
        const uint32_t U = ms[j].U;
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
          const T2 v = value_of(j, i);
          const T2* xp = tile + ((threadIdx.x + uint32_t(i) * NT) ^ U);
#pragma unroll
          for (int q = 0; q < RB; ++q, xp += TS)
            if (NRB || q < nrb) cfma(acc[i][q], v, *xp);
        }
      }
    };
    if (a.fvt[fi] >= 0) {
      // Value table: entry (pattern of the row's bits at fsm) * ns + slot.
      const T2* tb = vts + a.fvts[fi];
      const uint32_t sm = a.fsm[fi];
      const int psh = a.fsh[fi];
      uint32_t pat[ROWS];
#pragma unroll
      for (int i = 0; i < ROWS; ++i) pat[i] = pattern_fast(grow[i], sm, psh) * uint32_t(ns);
      multiply([&](int j, int i) { return tb[pat[i] + j]; });
    } else {
      const T2* st = stages + size_t(stage) * stage_elems + threadIdx.x;
      multiply([&](int j, int i) { return st[j * TS + i * NT]; });
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
    if (fi + S < a.n_factors) issue_factor(fi + S, stage);
    cp_async_commit();
    stage = (stage + 1 == S) ? 0 : stage + 1;
  }
  __syncthreads();
}

// Register-resident sweep: one state per tile, every factor read from its
// value table.  The thread keeps its rows' amplitudes (local rows t + i * NT)
// in registers.  A factor whose slots' local images U have no bits between the
// lane bits (0..4) and the row-select bits (log2 NT and up) is applied without
// shared memory or barriers: the partner of row i is row i ^ (U >> log2 NT) of
// lane lane ^ (U & 31), fetched by a warp shuffle.  Any other factor exchanges
// through one of two shared-memory buffers with one barrier (a buffer is
// written again only after a later barrier, by which every thread has finished
// reading it).  Each row's sum is the one the shared-memory path forms, in the
// same slot order.
template <typename T2, int ROWS>
__device__ __forceinline__ void sweep_reg(const SweepArgs& a, T2* tile, T2* other, const SlotMeta* mslot,
                                          const T2* vts, const uint32_t (&grow)[ROWS], int NT, int lg_nt,
                                          T2* dst_state) {
  cp_async_wait(0);
  __syncthreads();
  T2 xr[ROWS];
#pragma unroll
  for (int i = 0; i < ROWS; ++i) xr[i] = tile[threadIdx.x + i * NT];
  bool second = false;
  for (int fi = 0; fi < a.n_factors; ++fi) {
    const int ns = a.fnslot[fi];
    const SlotMeta* ms = mslot + a.fmslot[fi];
    const T2* tb = vts + a.fvts[fi];
    const uint32_t sm = a.fsm[fi];
    const int psh = a.fsh[fi];
    uint32_t pat[ROWS];
#pragma unroll
    for (int i = 0; i < ROWS; ++i) pat[i] = pattern_fast(grow[i], sm, psh) * uint32_t(ns);
    T2 acc[ROWS];
#pragma unroll
    for (int i = 0; i < ROWS; ++i) acc[i] = T2{0, 0};
    if ((a.flane >> fi) & 1ull) {
      for (int j = 0; j < ns; ++j) {
        const uint32_t U = ms[j].U;
        const int hi = int(U >> lg_nt);
        const int lane_x = int(U & 31u);
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
          T2 src = xr[0];
#pragma unroll
          for (int k = 1; k < ROWS; ++k)
            if (k == (i ^ hi)) src = xr[k];
          T2 x;
          x.x = __shfl_xor_sync(0xffffffffu, src.x, lane_x);
          x.y = __shfl_xor_sync(0xffffffffu, src.y, lane_x);
          cfma(acc[i], tb[pat[i] + j], x);
        }
      }
    } else {
      T2* t = second ? other : tile;
#pragma unroll
      for (int i = 0; i < ROWS; ++i) t[threadIdx.x + i * NT] = xr[i];
      __syncthreads();
      for (int j = 0; j < ns; ++j) {
        const uint32_t U = ms[j].U;
#pragma unroll
        for (int i = 0; i < ROWS; ++i) cfma(acc[i], tb[pat[i] + j], t[(threadIdx.x + uint32_t(i) * NT) ^ U]);
      }
      second = !second;
    }
#pragma unroll
    for (int i = 0; i < ROWS; ++i) xr[i] = acc[i];
  }
#pragma unroll
  for (int i = 0; i < ROWS; ++i) dst_state[HS_BCHK(grow[i], a.N, BS_SWEEP_STATE)] = xr[i];
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
//
// Units u0 .. u1-1 (unit = rhs block * 2^n_tiles_log2 + tile) run one after
// the other on this CTA: the sweep's tables are loaded once for all of them.
// MULTI = false compiles a single unit (u1 = u0 + 1), which keeps the
// multi-state instantiations at their single-tile register count.
template <typename R, int ROWS, int RB, bool MULTI = true>
__device__ __forceinline__ void sweep_tiles(const SweepArgs& a, uint32_t u0, uint32_t u1, unsigned char* smem_raw) {
  using T2 = typename C2<R>::T;
  constexpr int V = 16 / sizeof(T2);  // elements per 16-byte chunk
  const int NT = blockDim.x;
  const uint32_t TS = 1u << a.tile_bits;
  const uint32_t m0 = a.m0, m1 = a.m1;
  const int sh = a.sh;
  // Shared memory: [slot table][row-base table][value tables][tile][factor stages]
  SlotMeta* mslot = reinterpret_cast<SlotMeta*>(smem_raw);
  int64_t* mtab = reinterpret_cast<int64_t*>(mslot + a.n_mslot);
  T2* vts = reinterpret_cast<T2*>(mtab + ((a.n_mtab + 1) & ~1));
  T2* tile = vts + ((a.n_vt + V - 1) & ~(V - 1));
  T2* stages = tile + size_t(a.rhs_block) * TS;
  const uint32_t stage_elems = uint32_t(a.stage_planes) * TS;
  // src and dst may be the same buffer (in-place sweep): every CTA reads its
  // own tile completely before it writes it back, and tiles are disjoint.
  const T2* src = reinterpret_cast<const T2*>(a.src);
  T2* dst = reinterpret_cast<T2*>(a.dst);
  const T2* __restrict__ vals = reinterpret_cast<const T2*>(a.vals);

  const uint32_t n_chunks = TS / V;

  // Slot and row-base tables of every factor of the sweep, loaded once: each
  // thread takes table entries t, t + NT, ... and finds the factor that owns
  // an entry by binary search, so all global loads are independent.
  for (int t = threadIdx.x; t < a.n_mslot; t += NT) {
    int lo = 0, hi = a.n_factors - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.fmslot[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int gs = int(HS_BCHK(a.fslot0[lo] + (t - a.fmslot[lo]), a.n_slot_g, BS_SWEEP_SLOT));
    const uint32_t u = a.slot_u[gs];
    mslot[t] = SlotMeta{u, local_of(u, m0, m1, sh), a.ftab_s[lo] + (a.slot_tab[gs] - a.ftab_g[lo]),
                        a.fvt[lo] >= 0 ? -1 : lo * a.stage_planes + (t - a.fmslot[lo])};
  }
  for (int e = threadIdx.x; e < a.n_mtab; e += NT) {
    int lo = 0, hi = a.n_factors - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.ftab_s[mid] <= e) lo = mid; else hi = mid - 1;
    }
    mtab[e] = a.tab_rb[HS_BCHK(a.ftab_g[lo] + (e - a.ftab_s[lo]), a.n_tab_g, BS_SWEEP_TAB)];
  }
  // Value tables: entry e belongs to the last factor whose shared start is <= e
  // (factors without a table have empty ranges, so that factor owns it).
  {
    const T2* __restrict__ gvt = reinterpret_cast<const T2*>(a.vt);
    for (int e = threadIdx.x; e < a.n_vt; e += NT) {
      int lo = 0, hi = a.n_factors - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.fvts[mid] <= e) lo = mid; else hi = mid - 1;
      }
      vts[e] = gvt[HS_BCHK(a.fvt[lo] + (e - a.fvts[lo]), a.n_vt_g, BS_SWEEP_VT)];
    }
  }
  __syncthreads();

  const uint32_t u_end = MULTI ? u1 : u0 + 1;
  for (uint32_t unit = u0; unit < u_end; ++unit) {
  const uint32_t tile_id = unit & ((1u << a.n_tiles_log2) - 1u);
  const int rhs_blk = int(unit >> a.n_tiles_log2);
  const int rhs0 = rhs_blk * a.rhs_block;
  const int nrb = min(a.rhs_block, a.n_rhs - rhs0);
  const uint32_t base = deposit_runs(tile_id, a.rest);
  // the previous unit's threads are done with the tile and the stages
  if (unit != u0) __syncthreads();

  // Stage slots [p0, p1) of the slot table for the tile rows: plane u of a
  // factor receives, for every tile row r, the value of entry (r, r ^ u).  The
  // items (slot, 16-byte chunk) are independent, so one flat loop keeps many
  // copies in flight.  stage < 0: the prologue, whose planes sit at the
  // positions recorded in the slot table; otherwise the planes of one factor go
  // to that stage.
  const int chunk_log2 = a.tile_bits - (V == 2 ? 1 : 0);
  auto issue_slots = [&](int p0, int p1, int stage) {
    const int items = (p1 - p0) << chunk_log2;
#pragma unroll 4
    for (int k = threadIdx.x; k < items; k += NT) {
      const int p = p0 + (k >> chunk_log2);
      const uint32_t c = uint32_t(k) & (n_chunks - 1u);
      const SlotMeta m = mslot[p];
      if (stage < 0 && m.pos < 0) continue;  // read from its value table
      const int pos = stage < 0 ? m.pos : stage * a.stage_planes + (p - p0);
      T2* dst_s = stages + size_t(pos) * TS + c * V;
      const uint32_t r = global_of(c * V, m0, m1, sh) | base;
      const int64_t* tab = mtab + m.tab;
      const uint32_t pat = pattern_of(r, m.u);
#ifdef HS_DEBUG_BOUNDS
      HS_BCHK(m.tab + ((m.u & 1u) ? (pat | 1u) : pat), a.n_mtab, BS_SWEEP_TAB);
#endif
      if (V == 1 || !(m.u & 1u)) {
        cp_async16(dst_s, vals + HS_BCHK(tab[pat] + r, a.n_vals - (V - 1), BS_SWEEP_VAL));
      } else {
        // u flips bit 0: the two rows of a 16-byte chunk lie on different diagonals.
        cp_async8(dst_s, vals + HS_BCHK(tab[pat] + r, a.n_vals, BS_SWEEP_VAL));
        cp_async8(dst_s + 1, vals + HS_BCHK(tab[pat | 1u] + r + 1, a.n_vals, BS_SWEEP_VAL));
      }
    }
  };
  auto issue_factor = [&](int fi, int stage) {
    if (a.fvt[fi] < 0) issue_slots(a.fmslot[fi], a.fmslot[fi] + a.fnslot[fi], stage);
  };

  // Prologue: the first S factors, as one copy group.
  const int S = a.n_stages;
  issue_slots(0, S < a.n_factors ? a.fmslot[S] : a.n_mslot, -1);
  cp_async_commit();
  if (unit == u0) {
    // The state written by the previous launch is visible only after this.
    grid_dependency_wait();
    // Let the next sweep start its own prologue (tables and factor staging,
    // which read no state) while this one computes; it waits for this grid to
    // finish before it touches the state.
    grid_launch_dependents();
  }
  for (uint32_t c = threadIdx.x; c < n_chunks; c += NT) {
    const uint32_t l = c * V;
    const T2* sp = src + int64_t(rhs0) * a.N + HS_BCHK(global_of(l, m0, m1, sh) | base, a.N - (V - 1), BS_SWEEP_STATE);
    T2* tp = tile + l;
    for (int q = 0; q < nrb; ++q, sp += a.N, tp += TS) cp_async16(tp, sp);
  }
  cp_async_commit();

  uint32_t grow[ROWS];
#pragma unroll
  for (int i = 0; i < ROWS; ++i) grow[i] = global_of(threadIdx.x + uint32_t(i) * NT, m0, m1, sh) | base;
  if constexpr (RB == 1) {
    if (a.all_tables) {
      sweep_reg<T2, ROWS>(a, tile, stages, mslot, vts, grow, NT, __ffs(NT) - 1, dst + int64_t(rhs0) * a.N);
      continue;
    }
  }
  if (nrb == RB)
    sweep_body<T2, ROWS, RB, RB>(a, nrb, tile, stages, stage_elems, mslot, vts, grow, TS, NT, issue_factor);
  else
    sweep_body<T2, ROWS, RB, 0>(a, nrb, tile, stages, stage_elems, mslot, vts, grow, TS, NT, issue_factor);

  // Store the tile.
  for (uint32_t c = threadIdx.x; c < n_chunks; c += NT) {
    const uint32_t l = c * V;
    T2* dp = dst + int64_t(rhs0) * a.N + HS_BCHK(global_of(l, m0, m1, sh) | base, a.N - (V - 1), BS_SWEEP_STATE);
    const T2* tp = tile + l;
    for (int q = 0; q < nrb; ++q, dp += a.N, tp += TS)
      *reinterpret_cast<uint4*>(dp) = *reinterpret_cast<const uint4*>(tp);
  }
  }  // units
}

// Shared-memory bytes of the slot, row-base and value tables of a sweep.
inline size_t meta_bytes(int n_mslot, int n_mtab, int n_vt = 0, size_t elem = 8) {
  return size_t(n_mslot) * 16 + size_t((n_mtab + 1) & ~1) * 8 + (size_t(n_vt) * elem + 15) / 16 * 16;
}

}  // namespace sweep
}  // namespace hs
