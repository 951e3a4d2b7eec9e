// Register-blocked tile sweep (see qsweep.h for the descriptor).
//
// One CTA evolves a tile of 2^T amplitudes of one state through every op of
// the sweep:
//   1. the tile is copied from HBM into shared memory with 16-byte cp.async
//      copies (chunk c of the tile lands at the swizzled chunk swz(c));
//   2. each thread reads its 2^B rows for the first register layout into
//      registers and applies the ops: a factor whose flips lie in the
//      register bits touches only registers; a LAYOUT op writes the rows back
//      and reads them again for the next set of register bits;
//   3. the rows go back through shared memory and out to HBM with coalesced
//      16-byte stores.
// With T = 13 and B = 5 the tile is 64 KiB, the CTA has 256 threads, and a
// step of the 24-qubit MaxCut instance (24 factors) takes two sweeps, each
// reading and writing the states once.
//
// PHASE ops generate a diagonal run's values from (z_j, theta_j): with the
// tile's fixed bits folded in, phi(r) = C0 + sum_m C_m chi_m(l), where m runs
// over the distinct local parts of the z_j, chi_m(l) = (-1)^popcount(m & l)
// and C_m sums +-theta_j (FP64, once per tile).  A thread's rows differ only
// in their register bits, so phi over its 2^B rows is the Walsh-Hadamard
// transform of the per-thread coefficients E[mu] = sum over classes with
// register part mu of +-C_m; each row then takes exp(-i phi) (sincospi in
// the bulk precision, with exp(-i C0) from an FP64 sincos per tile).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "counters.h"
#include "hs_internal.h"
#include "qsweep.h"
#include "sweep_core.cuh"

namespace hs {
namespace q {
namespace {

using sweep::C2;
using sweep::cp_async16;
using sweep::cp_async_commit;
using sweep::cp_async_wait;
using sweep::deposit_runs;
using sweep::global_of;
using sweep::grid_dependency_wait;
using sweep::grid_launch_dependents;
using sweep::pattern_fast;

__device__ __forceinline__ void sincospi_r(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_r(double x, double* s, double* c) { sincospi(x, s, c); }

__device__ __forceinline__ int parity(uint32_t v) { return __popc(v) & 1; }

__host__ __device__ constexpr int highest_bit(int v) {
  int h = 0;
  while (v >> (h + 1)) ++h;
  return v ? (1 << h) : 0;
}


// (re, im) * (c, s) helpers.
template <typename T2, typename R>
__device__ __forceinline__ T2 cmul(T2 a, R bx, R by) {
  return T2{fma(a.x, bx, -a.y * by), fma(a.x, by, a.y * bx)};
}

// ---------------------------------------------------------------------------
// ROT: x <- (cos I - i sin P_j) x for one term whose flips are the register
// coordinates KU.  Row k's partner is k ^ KU; the off-diagonal coefficient of
// row k is sin * i^q * (-1)^popcount(z & r_{k ^ KU}), r_k the global row.
//
// A term with y = 0 and z = 0 (P = X on the flipped qubits) takes the factor
// build's split exp(-i theta P) = cos(theta') (I - i t P) (-i P)^k, t =
// tan(theta'), |theta'| <= pi / 4: rot_tan applies I - i t P with two fused
// multiply-adds per amplitude, cos(theta') and (-i)^k go into the sweep's
// scale, and an odd k swaps the partner rows (flip_pairs) at the end of the
// op, so the rotation itself has no data-dependent branch.
// ---------------------------------------------------------------------------
template <typename R, int NR, int KU>
__device__ __forceinline__ void rot_tan(typename C2<R>::T (&x)[NR], R t) {
  using T2 = typename C2<R>::T;
  constexpr int HB = highest_bit(KU);
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    if (k & HB) continue;
    const int k2 = k ^ KU;
    const T2 b1 = x[k], b2 = x[k2];
    x[k] = T2{fma(t, b2.y, b1.x), fma(-t, b2.x, b1.y)};
    x[k2] = T2{fma(t, b1.y, b2.x), fma(-t, b1.x, b2.y)};
  }
}

template <typename R, int NR, int KU>
__device__ __forceinline__ void flip_pairs(typename C2<R>::T (&x)[NR]) {
  using T2 = typename C2<R>::T;
  constexpr int HB = highest_bit(KU);
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    if (k & HB) continue;
    const T2 b = x[k];
    x[k] = x[k ^ KU];
    x[k ^ KU] = b;
  }
}

template <typename R, int NR, int KU>
__device__ __forceinline__ void rot_ku(typename C2<R>::T (&x)[NR], R c, R s, bool fast, int q, uint32_t zk,
                                       int sb, bool flip) {
  using T2 = typename C2<R>::T;
  constexpr int HB = highest_bit(KU);
  if (fast) {
    rot_tan<R, NR, KU>(x, c);
    if (flip) flip_pairs<R, NR, KU>(x);
    return;
  }
  const R qx = (q == 0) ? s : (q == 2 ? -s : R(0));
  const R qy = (q == 1) ? s : (q == 3 ? -s : R(0));
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    if (k & HB) continue;
    const int k2 = k ^ KU;
    const T2 b1 = x[k], b2 = x[k2];
    // row k pairs with column k2 (sign of r_k2), row k2 with column k (sign of r_k)
    const R sk = (sb ^ parity(zk & uint32_t(k2))) ? R(-1) : R(1);
    const R sk2 = (sb ^ parity(zk & uint32_t(k))) ? R(-1) : R(1);
    const R ax = sk * qx, ay = sk * qy, bx = sk2 * qx, by = sk2 * qy;
    x[k] = T2{fma(ax, b2.x, fma(-ay, b2.y, c * b1.x)), fma(ax, b2.y, fma(ay, b2.x, c * b1.y))};
    x[k2] = T2{fma(bx, b1.x, fma(-by, b1.y, c * b2.x)), fma(bx, b1.y, fma(by, b1.x, c * b2.y))};
  }
}

// ---------------------------------------------------------------------------
// TAB: x[k] <- v(p_k, 0) x[k] + v(p_k, 1) x[k ^ KU] with p_k the pattern of
// row k's global index at the factor's support (p_k = pt ^ XOR of pr[i] over
// the set bits i of k: the pattern map is linear over XOR).
// ---------------------------------------------------------------------------
template <typename R, int NR, int B, int KU>
__device__ __forceinline__ void tab_ku(typename C2<R>::T (&x)[NR], const typename C2<R>::T* tb, int ns,
                                       uint32_t pt, const uint32_t (&pr)[B]) {
  using T2 = typename C2<R>::T;
  constexpr int HB = KU ? highest_bit(KU) : 0;
  // Pattern of register row k: pt ^ XOR of pr[i] over the set bits i of k.
  auto pat = [&](int k) {
    uint32_t p = pt;
#pragma unroll
    for (int i = 0; i < B; ++i)
      if ((k >> i) & 1) p ^= pr[i];
    return p;
  };
  if constexpr (KU == 0) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const T2 v0 = tb[pat(k) * uint32_t(ns)];
      x[k] = T2{fma(v0.x, x[k].x, -v0.y * x[k].y), fma(v0.x, x[k].y, v0.y * x[k].x)};
    }
  } else {
  // Two slots: a row's entries (r, r) and (r, r ^ u) sit side by side in the
  // table, one 2 * sizeof(T2)-byte load.
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    if (k & HB) continue;
    const int k2 = k ^ KU;
    T2 a0, a1, c0, c1;
    if constexpr (sizeof(T2) == 8) {
      const float4 va = *reinterpret_cast<const float4*>(tb + pat(k) * 2u);
      const float4 vc = *reinterpret_cast<const float4*>(tb + pat(k2) * 2u);
      a0 = T2{va.x, va.y};
      a1 = T2{va.z, va.w};
      c0 = T2{vc.x, vc.y};
      c1 = T2{vc.z, vc.w};
    } else {
      const T2* va = tb + pat(k) * 2u;
      const T2* vc = tb + pat(k2) * 2u;
      a0 = va[0];
      a1 = va[1];
      c0 = vc[0];
      c1 = vc[1];
    }
    const T2 b1 = x[k], b2 = x[k2];
    T2 r1, r2;
    r1.x = fma(a0.x, b1.x, fma(-a0.y, b1.y, fma(a1.x, b2.x, -a1.y * b2.y)));
    r1.y = fma(a0.x, b1.y, fma(a0.y, b1.x, fma(a1.x, b2.y, a1.y * b2.x)));
    r2.x = fma(c0.x, b2.x, fma(-c0.y, b2.y, fma(c1.x, b1.x, -c1.y * b1.y)));
    r2.y = fma(c0.x, b2.y, fma(c0.y, b2.x, fma(c1.x, b1.y, c1.y * b1.x)));
    x[k] = r1;
    x[k2] = r2;
  }
  }
}

// ROTN: commuting X rotations on distinct single register bits (tan form,
// see ROT), the slot of register bit i in byte i of (zthr, zrest).  The full
// run and the run without bit 0 are straight-line bodies; any other run tests
// its bits.  The odd-k swaps follow the whole run (every factor of the run is
// a function of its own X, so they commute).
__device__ __forceinline__ int rotn_slot(const Op& op, int i) {
  return int((i < 4 ? (op.zthr >> (8 * i)) : (op.zrest >> (8 * (i - 4)))) & 0xffu);
}

template <typename R, int NR, int B, int MASK, int I>
__device__ __forceinline__ void rotn_fixed(typename C2<R>::T (&x)[NR], const Op& op, const typename C2<R>::T* rcs) {
  if constexpr (I < B) {
    if constexpr (((MASK >> I) & 1) != 0) rot_tan<R, NR, (1 << I)>(x, rcs[rotn_slot(op, I)].x);
    rotn_fixed<R, NR, B, MASK, I + 1>(x, op, rcs);
  }
}

template <typename R, int NR, int B, int I>
__device__ __forceinline__ void rotn_any(typename C2<R>::T (&x)[NR], const Op& op, const typename C2<R>::T* rcs) {
  if constexpr (I < B) {
    if ((op.ku >> I) & 1) rot_tan<R, NR, (1 << I)>(x, rcs[rotn_slot(op, I)].x);
    rotn_any<R, NR, B, I + 1>(x, op, rcs);
  }
}

template <typename R, int NR, int B, int I>
__device__ __forceinline__ void flip_run(typename C2<R>::T (&x)[NR], uint32_t fl) {
  if constexpr (I < B) {
    if ((fl >> I) & 1) flip_pairs<R, NR, (1 << I)>(x);
    flip_run<R, NR, B, I + 1>(x, fl);
  }
}

template <typename R, int NR, int B>
__device__ __forceinline__ void rot_run(typename C2<R>::T (&x)[NR], const Op& op, const typename C2<R>::T* rcs,
                                        uint32_t fl) {
  constexpr int FULL = (1 << B) - 1;
  if (op.ku == FULL)
    rotn_fixed<R, NR, B, FULL, 0>(x, op, rcs);
  else if (op.ku == (FULL & ~1))
    rotn_fixed<R, NR, B, (FULL & ~1), 0>(x, op, rcs);
  else
    rotn_any<R, NR, B, 0>(x, op, rcs);
  if (fl) flip_run<R, NR, B, 0>(x, fl);
}

// DROT: x[k] <- (cos - i sin (-1)^popcount(z & r_k)) x[k], the rotation of one
// diagonal term; sb is the parity of z over the row's fixed bits.
template <typename R, int NR>
__device__ __forceinline__ void diag_rot(typename C2<R>::T (&x)[NR], R c, R s, uint32_t zk, int sb) {
  using T2 = typename C2<R>::T;
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const R ss = (sb ^ parity(zk & uint32_t(k))) ? -s : s;
    const T2 v = x[k];
    x[k] = T2{fma(ss, v.y, c * v.x), fma(-ss, v.x, c * v.y)};
  }
}

// Register flips the planner may emit: one or two register bits.
#define HS_Q_KU_LIST(X) \
  X(1) X(2) X(4) X(8) X(16) X(3) X(5) X(6) X(9) X(10) X(12) X(17) X(18) X(20) X(24)

template <typename R, int NR>
__device__ __forceinline__ void rot_dispatch(typename C2<R>::T (&x)[NR], int ku, R c, R s, bool fast, int q,
                                          uint32_t zk, int sb, bool flip) {
  switch (ku) {
#define HS_Q_ROT_CASE(K) \
  case K:                \
    if constexpr (K < NR) rot_ku<R, NR, K>(x, c, s, fast, q, zk, sb, flip); \
    break;
    HS_Q_KU_LIST(HS_Q_ROT_CASE)
#undef HS_Q_ROT_CASE
    default: break;
  }
}

template <typename R, int NR>
__device__ __forceinline__ void tan_dispatch(typename C2<R>::T (&x)[NR], int ku, R t, bool flip) {
  switch (ku) {
#define HS_Q_TAN_CASE(K)                  \
  case K:                                 \
    if constexpr (K < NR) {               \
      rot_tan<R, NR, K>(x, t);            \
      if (flip) flip_pairs<R, NR, K>(x);  \
    }                                     \
    break;
    HS_Q_KU_LIST(HS_Q_TAN_CASE)
#undef HS_Q_TAN_CASE
    default: break;
  }
}

template <typename R, int NR, int B>
__device__ __forceinline__ void tab_dispatch(typename C2<R>::T (&x)[NR], int ku, const typename C2<R>::T* tb, int ns,
                                          uint32_t pt, const uint32_t (&pr)[B]) {
  switch (ku) {
    case 0: tab_ku<R, NR, B, 0>(x, tb, ns, pt, pr); break;
#define HS_Q_TAB_CASE(K) \
  case K:                \
    if constexpr (K < NR) tab_ku<R, NR, B, K>(x, tb, ns, pt, pr); \
    break;
    HS_Q_KU_LIST(HS_Q_TAB_CASE)
#undef HS_Q_TAB_CASE
    default: break;
  }
}

// ---------------------------------------------------------------------------
// PHASE: x[k] <- exp(-i phi(r_k)) x[k].  With the tile's fixed bits folded
// into the per-tile class constants (units of pi) and the thread's bits into
// E[mu] = sum over the classes with register part mu of +-C_c, the phase of
// register row k is e0 * prod_mu exp(-i pi E[mu] chi_mu(k)), chi_mu(k) =
// (-1)^popcount(mu & k).  The factors of mu = 0 and of the single register
// bits are multiplied out in two small groups of bits (all rows' values from
// a few products); every other mu present multiplies each row by
// cos(pi E) -+ i sin(pi E).  One sincospi per present mu, not per row.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R class_sum(const PClass* cls, const R* Cs, int c0, int c1, uint32_t lt) {
  R e = R(0);
  for (int cc = c0; cc < c1; ++cc) {
    const R v = Cs[cc];
    e += parity(cls[cc].thr & lt) ? -v : v;
  }
  return e;
}

template <typename R, int NR, int B>
__device__ __forceinline__ void phase_apply(typename C2<R>::T (&x)[NR], const Phase& P, const PClass* cls,
                                            const R* Cs, typename C2<R>::T e0, uint32_t lt) {
  using T2 = typename C2<R>::T;
  constexpr int B1 = (B + 1) / 2, B2 = B - B1;  // the single-bit factors in two groups
  const int base = P.cls0;
  // mu = 0 (thread-dependent part of the constant) folded into e0.
  T2 g0 = e0;
  {
    const R e = class_sum<R>(cls, Cs, base + P.mu_beg[0], base + P.mu_beg[1], lt);
    R sn, cn;
    sincospi_r(e, &sn, &cn);
    g0 = T2{fma(g0.x, cn, g0.y * sn), fma(g0.y, cn, -g0.x * sn)};
  }
  // Single register bits: (cos, sin) of pi E[2^i].
  R cb[B], sb[B];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const int mu = 1 << i;
    const R e = class_sum<R>(cls, Cs, base + P.mu_beg[mu], base + P.mu_beg[mu + 1], lt);
    sincospi_r(e, &sb[i], &cb[i]);
  }
  // Group values, applied one group at a time (fewer live registers):
  // A[a] = g0 prod_{i < B1} f_i(bit i of a), then Bv[b] = prod_{i < B2}
  // f_{B1+i}(bit i of b); f_i(0) = cos - i sin, f_i(1) = cos + i sin.  A
  // pattern mu of two or more register bits within one group multiplies that
  // group's values; one that spans both groups multiplies every row.
  uint32_t rest = P.mu_mask;
#pragma unroll
  for (int i = 0; i <= B; ++i) rest &= ~(i == 0 ? 1u : (1u << (1 << (i - 1))));
  constexpr uint32_t GA = (1u << B1) - 1u;
  auto mu_factor = [&](int mu, R& cn, R& sn) {
    const R e = class_sum<R>(cls, Cs, base + P.mu_beg[mu], base + P.mu_beg[mu + 1], lt);
    sincospi_r(e, &sn, &cn);
  };
  {
    T2 A[1 << B1];
    A[0] = g0;
#pragma unroll
    for (int i = 0; i < B1; ++i)
#pragma unroll
      for (int k = 0; k < (1 << i); ++k) {
        const T2 p = A[k];
        const R ac = p.x * cb[i], bs = p.y * sb[i], bc = p.y * cb[i], as = p.x * sb[i];
        A[k] = T2{ac + bs, bc - as};
        A[k + (1 << i)] = T2{ac - bs, bc + as};
      }
    for (uint32_t r = rest & ((1u << (1u << B1)) - 1u); r; r &= r - 1u) {  // mu inside group A
      const int mu = __ffs(r) - 1;
      R cn, sn;
      mu_factor(mu, cn, sn);
#pragma unroll
      for (int k = 0; k < (1 << B1); ++k) A[k] = cmul<T2, R>(A[k], cn, parity(uint32_t(mu) & uint32_t(k)) ? sn : -sn);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) x[k] = cmul<T2, R>(x[k], A[k & GA].x, A[k & GA].y);
  }
  {
    T2 Bv[1 << B2];
    Bv[0] = T2{R(1), R(0)};
#pragma unroll
    for (int i = 0; i < B2; ++i)
#pragma unroll
      for (int k = 0; k < (1 << i); ++k) {
        const T2 p = Bv[k];
        const R c = cb[B1 + i], sn = sb[B1 + i];
        const R ac = p.x * c, bs = p.y * sn, bc = p.y * c, as = p.x * sn;
        Bv[k] = T2{ac + bs, bc - as};
        Bv[k + (1 << i)] = T2{ac - bs, bc + as};
      }
    for (uint32_t r = rest; r; r &= r - 1u) {  // mu inside group B
      const int mu = __ffs(r) - 1;
      if (uint32_t(mu) & GA) continue;
      R cn, sn;
      mu_factor(mu, cn, sn);
#pragma unroll
      for (int k = 0; k < (1 << B2); ++k)
        Bv[k] = cmul<T2, R>(Bv[k], cn, parity(uint32_t(mu >> B1) & uint32_t(k)) ? sn : -sn);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) x[k] = cmul<T2, R>(x[k], Bv[k >> B1].x, Bv[k >> B1].y);
  }
  for (uint32_t r = rest; r; r &= r - 1u) {  // mu across the two groups
    const int mu = __ffs(r) - 1;
    if (!(uint32_t(mu) & GA) || uint32_t(mu) <= GA) continue;
    R cn, sn;
    mu_factor(mu, cn, sn);
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const R ss = parity(uint32_t(mu) & uint32_t(k)) ? sn : -sn;
      x[k] = cmul<T2, R>(x[k], cn, ss);
    }
  }
}

// ---------------------------------------------------------------------------
// The sweep of units [u0, u1) of one descriptor (single launch: the kernel
// parameter; batched launch: a descriptor in global memory).  NT = 2^(T - B)
// threads; NR = 2^B rows per thread.
//
// A unit's tile moves HBM -> shared memory -> registers by warp-cooperative
// copies (each warp copies exactly the rows its threads hold in the first
// layout, in address order), so the first read needs only a warp barrier.
// Once a unit has read its last layout, the tile buffer is free: after one CTA
// barrier every warp starts copying its rows of the CTA's next unit, which
// land while the current unit finishes in registers and writes its rows
// straight back to HBM.
// ---------------------------------------------------------------------------
template <typename R, int B, bool FULL>
__device__ __forceinline__ void qsweep_core(const Args& a, uint32_t u0, uint32_t u1, unsigned char* smem_raw,
                                            bool pdl) {
  using T2 = typename C2<R>::T;
  constexpr int NR = 1 << B;
  constexpr int V = 16 / int(sizeof(T2));  // rows per 16-byte chunk (2 for complex64)
  constexpr int VB = V == 2 ? 1 : 0;       // register bits inside a chunk
  constexpr int NJ = NR / V;               // chunks per thread
  const int NT = blockDim.x;
  const uint32_t tid = threadIdx.x;
  const uint32_t TS = 1u << a.tile_bits;
  const uint32_t m0 = a.m0, m1 = a.m1;
  const int sh = a.sh;
  const int n_warps = NT >> 5;
  const int warp = tid >> 5, lane = tid & 31;

  // Shared memory: [tile][value tables][rotations][per-warp e0 per phase]
  // [per-warp class constants][ops][layouts][phase headers][classes][terms]
  // [term angles][scale partials]
  T2* tile = reinterpret_cast<T2*>(smem_raw);
  T2* vts = tile + TS;  // 16-byte aligned (the planner keeps n_vt and every table start even)
  T2* rcs = vts + a.n_vt;
  T2* e0s = rcs + a.n_rot + warp * a.n_phase;
  R* Cs = reinterpret_cast<R*>(rcs + a.n_rot + n_warps * a.n_phase) + warp * a.n_cls;
  unsigned char* meta = reinterpret_cast<unsigned char*>(
      reinterpret_cast<R*>(rcs + a.n_rot + n_warps * a.n_phase) + n_warps * a.n_cls);
  meta += (16 - reinterpret_cast<uintptr_t>(meta) % 16) % 16;
  Op* sops = reinterpret_cast<Op*>(meta);
  Layout* slay = reinterpret_cast<Layout*>(sops + a.n_ops);
  Phase* sph = reinterpret_cast<Phase*>(slay + a.n_lay);
  PClass* scls = reinterpret_cast<PClass*>(sph + a.n_phase);
  PTerm* spt = reinterpret_cast<PTerm*>(scls + a.n_cls);
  auto align16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15); };
  R* thpi = reinterpret_cast<R*>(align16(spt + a.n_pterm));
  double* mpart = reinterpret_cast<double*>(align16(thpi + a.n_pterm));
  int* kpart = reinterpret_cast<int*>(mpart + n_warps);
  uint8_t* flips = reinterpret_cast<uint8_t*>(kpart + n_warps);  // per op: register bits whose partners swap
  // Per layout: the local-row bits a lane index and a warp index deposit
  // (local row of a thread's register row 0 = dlane[lane] | dwarp[warp]).
  uint32_t* dlane = reinterpret_cast<uint32_t*>(align16(flips + a.n_ops));
  uint32_t* dwarp = dlane + 32 * a.n_lay;

  auto unit_base = [&](uint32_t unit) { return deposit_runs(unit & ((1u << a.n_tiles_log2) - 1u), a.rest); };
  auto unit_src = [&](uint32_t unit) {
    return reinterpret_cast<const T2*>(a.src) + HS_BCHK(unit >> a.n_tiles_log2, a.n_rhs, BS_REG_STATE) * a.N;
  };

  // Per-CTA tables (written by launches that completed before this grid began).
  {
    auto copy_words = [&](void* dst, const void* src, size_t bytes) {
      const uint32_t* s4 = static_cast<const uint32_t*>(src);
      uint32_t* d4 = static_cast<uint32_t*>(dst);
      for (uint32_t w = tid; w < bytes / 4; w += NT) d4[w] = s4[w];
    };
    copy_words(sops, a.ops, sizeof(Op) * a.n_ops);
    copy_words(slay, a.lay, sizeof(Layout) * a.n_lay);
    copy_words(sph, a.ph, sizeof(Phase) * a.n_phase);
    copy_words(scls, a.cls, sizeof(PClass) * a.n_cls);
    copy_words(spt, a.pt, sizeof(PTerm) * a.n_pterm);
  }
  for (int e = tid; e < 48 * a.n_lay; e += NT) {
    const int li = e / 48, j = e - 48 * li;
    const Layout& L = a.lay[li];
    uint32_t d = 0;
    if (j < 32) {
      for (int i = 0; i < 5 && i < L.n_thr; ++i) d |= uint32_t((j >> i) & 1) << L.thr[i];
      dlane[32 * li + j] = d;
    } else {
      for (int i = 5; i < L.n_thr; ++i) d |= uint32_t(((j - 32) >> (i - 5)) & 1) << L.thr[i];
      dwarp[16 * li + (j - 32)] = d;
    }
  }
  // Rotations: a fast rotation (y = 0, z = 0) as tan(theta') of the factor
  // build's record, with cos(theta') and its quarter turns k in the sweep's
  // scale (the warps' partial products and sums, combined where the scale is
  // applied) and an odd k as a swap of partners in its op; any other rotation
  // as (cos, sin).
  for (int i = tid; i < a.n_rot; i += NT) {
    const int e = a.rot[i].cs;
    if (a.rot[i].fast) {
      const double* q = a.rq + 4 * HS_BCHK(e, a.n_terms_g, BS_REG_TERM);
      rcs[i] = T2{R(q[0]), R(0)};
    } else {
      const double* p = a.cs + 2 * HS_BCHK(e, a.n_terms_g, BS_REG_TERM);
      rcs[i] = T2{R(p[0]), R(p[1])};
    }
  }
  {
    double m = 1.0;
    int kq = 0;
    auto take = [&](int rot) {
      const double* q = a.rq + 4 * HS_BCHK(a.rot[rot].cs, a.n_terms_g, BS_REG_TERM);
      m *= q[2];
      const int k = int(q[1]);
      kq += k;
      return k & 1;
    };
    for (int oi = tid; oi < a.n_ops; oi += NT) {
      const Op& op = a.ops[oi];
      uint32_t fl = 0;
      if (op.type == OP_ROT && (op.flags & 1)) {
        fl = uint32_t(take(op.idx));
      } else if (op.type == OP_ROTN) {
#pragma unroll
        for (int i = 0; i < B; ++i)
          if ((op.ku >> i) & 1) fl |= uint32_t(take(rotn_slot(op, i))) << i;
      }
      flips[oi] = uint8_t(fl);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m *= __shfl_xor_sync(0xffffffffu, m, o);
      kq += __shfl_xor_sync(0xffffffffu, kq, o);
    }
    if (lane == 0) {
      mpart[warp] = m;
      kpart[warp] = kq;
    }
  }
  for (int t = tid; t < a.n_pterm; t += NT) thpi[t] = R(a.rq[4 * HS_BCHK(a.pt[t].th, a.n_terms_g, BS_REG_TERM) + 3]);
  for (int t = 0; t < a.n_tab; ++t) {
    const T2* g = reinterpret_cast<const T2*>(a.vt) + a.tab[t].vt0;
    const int s0 = a.tab[t].s0, n = a.tab[t].n;
    for (int e = tid; e < n; e += NT) vts[s0 + e] = g[HS_BCHK(a.tab[t].vt0 + e, a.n_vt_g, BS_REG_VT) - a.tab[t].vt0];
  }
  const int n_ops = a.n_ops, n_cls = a.n_cls;

  // Index of the last layout op (the tile buffer is free after its reads).
  int last_lay = 0;
  for (int oi = 0; oi < n_ops; ++oi)
    if (a.ops[oi].type == OP_LAYOUT) last_lay = oi;

  // Warp-cooperative copy of this warp's rows of a unit in the first layout of
  // the sweep into the tile buffer: chunk mm of the thread lies at swizzled
  // chunk s0 ^ mswz(mm) and global row g0 ^ mglob(mm), both maps linear over
  // XOR, so four basis values each give all of them.
  constexpr int NJB = B - VB;  // log2 NJ
  uint32_t cin_s0, cin_g0;
  {
    const Layout& L = a.lay[a.ops[0].idx];
    uint32_t lc = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) lc |= uint32_t((lane >> k) & 1) << L.wlo[k];
    uint32_t wb = 0;
    for (int i = 5; i < L.n_thr; ++i) wb |= ((tid >> i) & 1u) << L.thr[i];
    const uint32_t c0 = lc | (wb >> VB);
    cin_s0 = swz(c0);
    cin_g0 = global_of(c0 * V, m0, m1, sh);
  }
  const Layout* L0 = slay + a.ops[0].idx;  // the first op is always a layout
  auto copy_in = [&](uint32_t base, const T2* src) {
    uint32_t ms[NJB], mg[NJB];
#pragma unroll
    for (int k = 0; k < NJB; ++k) {
      ms[k] = L0->mswz[1 << k];
      mg[k] = L0->mglob[1 << k];
    }
    const uint32_t g0 = cin_g0 | base;
#pragma unroll
    for (int mm = 0; mm < NJ; ++mm) {
      uint32_t sx = cin_s0, gx = g0;
#pragma unroll
      for (int k = 0; k < NJB; ++k)
        if ((mm >> k) & 1) {
          sx ^= ms[k];
          gx ^= mg[k];
        }
      cp_async16(tile + sx * V, src + HS_BCHK(gx, a.N - (V - 1), BS_REG_STATE));
    }
    cp_async_commit();
  };

  if (pdl) grid_dependency_wait();  // the state written by the previous launch is visible after this
  __syncthreads();                  // the tables are in shared memory
  if (u0 < u1) copy_in(unit_base(u0), unit_src(u0));
  // The sweep's rotation scale m (-i)^K (the same for every unit).
  R m_sweep;
  int k_sweep;
  {
    double md = 1.0;
    int kq = 0;
    for (int w = 0; w < n_warps; ++w) {
      md *= mpart[w];
      kq += kpart[w];
    }
    m_sweep = R(md);
    k_sweep = kq & 3;
  }
  if (pdl) grid_launch_dependents();  // the next sweep may load its tables meanwhile

  for (uint32_t unit = u0; unit < u1; ++unit) {
    const uint32_t base = unit_base(unit);
    T2* dst = reinterpret_cast<T2*>(a.dst) + HS_BCHK(unit >> a.n_tiles_log2, a.n_rhs, BS_REG_STATE) * a.N;
    // Per-tile phase constants, in this warp's copy: class sums of +-theta_j
    // (units of pi, each term reduced mod 2 in FP64 by the factor build) with
    // the signs of the tile's fixed bits, reduced mod 2 again; a constant class
    // becomes its phase op's e0.  (The warp barrier keeps a lane from writing
    // them while another lane still reads the previous unit's.)
    __syncwarp();
    for (int cc = lane; cc < n_cls; cc += 32) {
      const PClass C = scls[cc];
      R acc = R(0);
      for (int t = C.t0; t < C.t0 + C.nt; ++t) {
        const R v = thpi[t];
        acc += parity(spt[t].rest & base) ? -v : v;
      }
      const R ur = acc - R(2) * rint(R(0.5) * acc);
      if (C.c0p >= 0) {
        R sn, cn;
        sincospi_r(ur, &sn, &cn);
        e0s[C.c0p] = T2{cn, -sn};
        Cs[cc] = R(0);
      } else {
        Cs[cc] = ur;
      }
    }

    __syncwarp();
    T2 x[NR];
    uint32_t lt = 0, st = 0, gt = 0;  // row of register index 0: local, swizzled chunk, global
    const Layout* cur = nullptr;      // the register layout in effect

    for (int oi = 0; oi < n_ops; ++oi) {
      const Op op = sops[oi];
      if (op.type == OP_LAYOUT) {
        // A thread writes back only rows of its own warp (each warp owns the
        // rows with its warp-bit values), so a warp barrier orders those writes
        // after the warp's reads of the previous layout; the new layout reads
        // other warps' rows unless its warp bits are the previous ones (flag).
        if (cur) {
          __syncwarp();
          uint32_t q[B];
#pragma unroll
          for (int i = 0; i < B; ++i) q[i] = cur->qoff[i];
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            uint32_t pc = st;
#pragma unroll
            for (int i = 0; i < B - VB; ++i)
              if ((j >> i) & 1) pc ^= q[i + VB];
            if constexpr (V == 2) {
              *reinterpret_cast<float4*>(tile + pc * 2) =
                  make_float4(x[2 * j].x, x[2 * j].y, x[2 * j + 1].x, x[2 * j + 1].y);
            } else {
              tile[pc] = x[j];
            }
          }
          if (op.flags & 1)
            __syncwarp();
          else
            __syncthreads();
        } else {
          cp_async_wait(0);  // this unit's rows, copied by this warp
          __syncwarp();
        }
        const Layout* L = slay + op.idx;
        const uint32_t l = dlane[32 * op.idx + lane] | dwarp[16 * op.idx + warp];
        uint32_t q[B];
#pragma unroll
        for (int i = 0; i < B; ++i) q[i] = L->qoff[i];
        lt = l;
        st = swz(l >> VB);
        gt = global_of(l, m0, m1, sh) | base;
        cur = L;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          uint32_t pc = st;
#pragma unroll
          for (int i = 0; i < B - VB; ++i)
            if ((j >> i) & 1) pc ^= q[i + VB];
          if constexpr (V == 2) {
            const float4 w = *reinterpret_cast<const float4*>(tile + pc * 2);
            x[2 * j] = T2{w.x, w.y};
            x[2 * j + 1] = T2{w.z, w.w};
          } else {
            x[j] = tile[pc];
          }
        }
        if (oi == last_lay && unit + 1 < u1) {
          // The tile buffer is free once every warp has read its rows: start
          // copying the next unit's rows.
          __syncthreads();
          copy_in(unit_base(unit + 1), unit_src(unit + 1));
        }
      } else if (op.type == OP_ROTN) {
        rot_run<R, NR, B>(x, op, rcs, flips[oi]);
      } else if (op.type == OP_ROT) {
        const T2 cs = rcs[op.idx];
        if constexpr (FULL) {
          const bool fast = op.flags & 1;
          const int sbit = fast ? 0 : (parity(op.zrest & base) ^ parity(op.zthr & lt));
          rot_dispatch<R, NR>(x, op.ku, cs.x, cs.y, fast, (op.flags >> 1) & 3, op.zk, sbit, flips[oi] != 0);
        } else {
          tan_dispatch<R, NR>(x, op.ku, cs.x, flips[oi] != 0);  // the planner sends only tan-form rotations here
        }
      } else if (op.type == OP_DROT) {
        const T2 cs = rcs[op.idx];
        diag_rot<R, NR>(x, cs.x, cs.y, op.zk, parity(op.zrest & base) ^ parity(op.zthr & lt));
      } else if (op.type == OP_TAB) {
        if constexpr (FULL) {
          const Tab& tb = a.tab[op.idx];
          const uint32_t sm = tb.sm;
          const int tsh = tb.sh;
          uint32_t pr[B];
#pragma unroll
          for (int i = 0; i < B; ++i) pr[i] = pattern_fast(cur->goff[i], sm, tsh);
          tab_dispatch<R, NR, B>(x, op.ku, vts + tb.s0, tb.ns, pattern_fast(gt, sm, tsh), pr);
        }
      } else {
        phase_apply<R, NR, B>(x, sph[op.idx], scls, Cs, e0s[op.idx], lt);
      }
    }
    // The sweep's rotation scale m (-i)^K, then the rows straight to HBM:
    // register row 2j (and 2j + 1 in the same 16 bytes for complex64) sits at
    // global row gt ^ XOR of the layout's global offsets of the set bits of 2j.
    // (One store body per form of the scale, so no join follows it.)
    const R m = m_sweep;
    const int K = k_sweep;
    uint32_t go[B];
#pragma unroll
    for (int i = 0; i < B; ++i) go[i] = cur->goff[i];
    auto store_rows = [&](auto scale) {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        uint32_t g = gt;
#pragma unroll
        for (int i = 0; i < B - VB; ++i)
          if ((j >> i) & 1) g ^= go[i + VB];
        if constexpr (V == 2) {
          const T2 v0 = scale(x[2 * j]), v1 = scale(x[2 * j + 1]);
          *reinterpret_cast<float4*>(dst + HS_BCHK(g, a.N - 1, BS_REG_STATE)) = make_float4(v0.x, v0.y, v1.x, v1.y);
        } else {
          dst[HS_BCHK(g, a.N, BS_REG_STATE)] = scale(x[j]);
        }
      }
    };
    // When the two lowest register bits are local bits 0 and 1 (complex64;
    // for complex128 register bit 0 is local bit 0) and the tile keeps those
    // bits contiguous, a thread's registers 4q .. 4q + 3 (2q, 2q + 1) are 32
    // consecutive bytes: one 32-byte store fills a whole sector.
    constexpr int WB = V == 2 ? 2 : 1;  // register bits inside a 32-byte store
    auto store_wide = [&](auto scale) {
#pragma unroll
      for (int q = 0; q < (NR >> WB); ++q) {
        uint32_t g = gt;
#pragma unroll
        for (int i = WB; i < B; ++i)
          if (((q << WB) >> i) & 1) g ^= go[i];
        T2* p = dst + HS_BCHK(g, a.N - (1 << WB) + 1, BS_REG_STATE);
        if constexpr (V == 2) {
          const T2 v0 = scale(x[4 * q]), v1 = scale(x[4 * q + 1]), v2 = scale(x[4 * q + 2]), v3 = scale(x[4 * q + 3]);
          asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"l"(p), "f"(v0.x), "f"(v0.y),
                       "f"(v1.x), "f"(v1.y), "f"(v2.x), "f"(v2.y), "f"(v3.x), "f"(v3.y)
                       : "memory");
        } else {
          const T2 v0 = scale(x[2 * q]), v1 = scale(x[2 * q + 1]);
          asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};\n" ::"l"(p), "d"(v0.x), "d"(v0.y), "d"(v1.x), "d"(v1.y)
                       : "memory");
        }
      }
    };
    const uint32_t wide_bits = (1u << WB) - 1u;  // local bits that must be the lowest register bits
    const bool wide = (cur->reg & wide_bits) == wide_bits && (m0 & wide_bits) == wide_bits &&
                      (reinterpret_cast<uintptr_t>(a.dst) & 31u) == 0;  // (states may be only 16-byte aligned)
    if (K == 0) {
      auto sc = [&](T2 v) { return T2{v.x * m, v.y * m}; };
      if (wide) store_wide(sc); else store_rows(sc);
    } else {
      const R cr = K == 2 ? -m : R(0), ci = K == 1 ? -m : (K == 3 ? m : R(0));
      auto sc = [&](T2 v) { return T2{fma(v.x, cr, -v.y * ci), fma(v.x, ci, v.y * cr)}; };
      if (wide) store_wide(sc); else store_rows(sc);
    }
  }
}

// FULL: the kernel with the TAB and general-rotation paths; sweeps without
// them run the lighter instantiation (fewer live registers, no spills).  NT:
// threads per CTA the instantiation is built for (2^(tile_bits - B); 512 for
// 2^14-row complex64 tiles with five register bits, one CTA per SM).
template <typename R, int B, bool FULL, int NT = (B == 5 ? 256 : 512)>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) qsweep_kernel(const __grid_constant__ Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t u0 = blockIdx.x * uint32_t(a.units_per_cta);
  const uint32_t u1 = min(uint32_t(a.n_units), u0 + uint32_t(a.units_per_cta));
  qsweep_core<R, B, FULL>(a, u0, u1, smem_raw, true);
}

template <typename R, int B, bool FULL>
__global__ void __launch_bounds__(B == 5 ? 256 : 512, B == 5 ? 2 : 1) qlevel_kernel(const __grid_constant__ LevelArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* pref = reinterpret_cast<int*>(smem_raw + p.prefix_smem);
  for (int i = threadIdx.x; i < p.count; i += blockDim.x) pref[i] = p.lvl_prefix[p.off + i];
  __syncthreads();
  int lo = 0, hi = p.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= int(blockIdx.x)) lo = mid; else hi = mid - 1;
  }
  const Args& a = p.descs[p.lvl_desc[p.off + lo]];
  const uint32_t u = uint32_t(HS_BCHK(blockIdx.x - uint32_t(pref[lo]), a.n_units, BS_BATCH_JOB));
  qsweep_core<R, B, FULL>(a, u, u + 1, smem_raw, true);
}

using LFn = void (*)(LevelArgs);

using QFn = void (*)(Args);

// The instantiation for (precision, register bits, tile bits): 2^(T - B)
// threads, at most 256 for five register bits (512 with T = 14), at most 512
// for four; nullptr otherwise.
template <bool FULL>
QFn qsweep_fn_t(hs_dtype dt, int B, int tile_bits) {
  const int tb = tile_bits - B;
  if (tb < 5) return nullptr;
  if (dt == HS_C64 && B == 5)
    return tb <= 8 ? qsweep_kernel<float, 5, FULL> : (tb == 9 ? qsweep_kernel<float, 5, FULL, 512> : nullptr);
  if (B == 4 && tb <= 9) return dt == HS_C64 ? qsweep_kernel<float, 4, FULL> : qsweep_kernel<double, 4, FULL>;
  return nullptr;
}
QFn qsweep_fn(hs_dtype dt, int B, bool full, int tile_bits) {
  return full ? qsweep_fn_t<true>(dt, B, tile_bits) : qsweep_fn_t<false>(dt, B, tile_bits);
}

template <bool FULL>
LFn qlevel_fn_t(hs_dtype dt, int B) {
  if (dt == HS_C64)
    return B == 5 ? qlevel_kernel<float, 5, FULL> : (B == 4 ? qlevel_kernel<float, 4, FULL> : nullptr);
  return B == 4 ? qlevel_kernel<double, 4, FULL> : nullptr;
}
LFn qlevel_fn(hs_dtype dt, int B, bool full) { return full ? qlevel_fn_t<true>(dt, B) : qlevel_fn_t<false>(dt, B); }

}  // namespace

cudaError_t prepare_qsweep() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && done[dev]) return cudaSuccess;
  const hs_dtype dts[3] = {HS_C64, HS_C64, HS_C128};
  const int Bs[3] = {5, 4, 4};
  for (int v = 0; v < 3; ++v)
    for (bool full : {false, true}) {
      e = cudaFuncSetAttribute((const void*)qsweep_fn(dts[v], Bs[v], full, Bs[v] + 8),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSweepSmemMax));
      if (e == cudaSuccess && v == 0)
        e = cudaFuncSetAttribute((const void*)qsweep_fn(dts[v], Bs[v], full, 14),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSweepSmemMax));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)qlevel_fn(dts[v], Bs[v], full),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSweepSmemMax));
      if (e != cudaSuccess) return e;
    }
  if (dev < 64) done[dev] = true;
  return cudaSuccess;
}

size_t qsweep_smem_bytes(const Args& a, hs_dtype dt, int B) {
  const size_t e = elem_bytes(dt), r = e / 2;
  const size_t warps = size_t(1) << (a.tile_bits - B - 5);
  const size_t head =
      ((size_t(1) << a.tile_bits) + a.n_rot + a.n_vt + warps * a.n_phase) * e + warps * size_t(a.n_cls) * r;
  return (head + 15) / 16 * 16 + sizeof(Op) * a.n_ops + sizeof(Layout) * a.n_lay + sizeof(Phase) * a.n_phase +
         sizeof(PClass) * a.n_cls + sizeof(PTerm) * a.n_pterm + 16 + r * a.n_pterm + 16 + 12 * warps + a.n_ops + 16 +
         192 * size_t(a.n_lay);
}

void fill_job(const hs_factors* f, Args& a, void* psi, int n_rhs) {
  const Plan& p = f->plan;
  a.src = psi;
  a.dst = psi;
  a.cs = f->bin.cs;
  a.th = f->bin.th;
  a.rq = f->bin.rq;
  a.vt = f->d_vt;
  a.N = p.N;
  a.n_vt_g = p.total_vt;
  a.n_terms_g = int(p.x.size()) * p.n_kinds;
  a.n_rhs = n_rhs;
  a.n_tiles_log2 = p.n_qubits - a.tile_bits;
  a.n_units = (1 << a.n_tiles_log2) * n_rhs;
}

cudaError_t launch_qlevel(hs_dtype dt, int B, bool full, int tile_bits, const LevelArgs& L, int64_t ctas, size_t smem,
                          cudaStream_t s) {
  LFn fn = qlevel_fn(dt, B, full);
  if (!fn || tile_bits - B < 5 || smem > kSweepSmemMax || ctas <= 0 || ctas >= (int64_t(1) << 31))
    return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(ctas), 1u, 1u);
  cfg.blockDim = dim3(unsigned(1u << (tile_bits - B)), 1u, 1u);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fn, L);
  if (e == cudaSuccess) note_launches();
  return e;
}

cudaError_t launch_qsweep(const hs_factors* f, Args& a, const void* src, void* dst, int n_rhs, int B, bool pdl,
                          cudaStream_t s, const double* rq, const double* cs, int n_terms) {
  const Plan& p = f->plan;
  QFn fn = qsweep_fn(f->dtype, B, a.full != 0, a.tile_bits);
  if (!fn || a.tile_bits - B < 5 || a.tile_bits > p.n_qubits) return cudaErrorInvalidValue;
  fill_job(f, a, const_cast<void*>(src), n_rhs);
  a.dst = dst;
  if (rq) {
    a.rq = rq;
    a.cs = cs;
    a.n_terms_g = n_terms;
  }
  // Several tiles per CTA once the grid is large (the per-CTA tables are then
  // loaded once for them), up to eight, keeping at least four waves of two
  // CTAs per SM (eight units per CTA measured 2.7% faster than four on the
  // 24-qubit, 16-state MaxCut sweeps).
  if (a.units_per_cta < 1) a.units_per_cta = std::max(1, std::min(8, a.n_units / (152 * 2 * 4)));
  const size_t smem = qsweep_smem_bytes(a, f->dtype, B);
  if (smem > kSweepSmemMax) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned((a.n_units + a.units_per_cta - 1) / a.units_per_cta), 1u, 1u);
  cfg.blockDim = dim3(unsigned(1u << (a.tile_bits - B)), 1u, 1u);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fn, a);
  if (e == cudaSuccess) note_launches();
  return e;
}

}  // namespace q
}  // namespace hs
