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
// ---------------------------------------------------------------------------
template <typename R, int NR, int KU>
__device__ __forceinline__ void rot_ku(typename C2<R>::T (&x)[NR], R c, R s, bool fast, int q, uint32_t zk,
                                       int sb) {
  using T2 = typename C2<R>::T;
  constexpr int HB = highest_bit(KU);
  if (fast) {
    // y = 0, z = 0: coefficient -i sin on every row.
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      if (k & HB) continue;
      const int k2 = k ^ KU;
      const T2 b1 = x[k], b2 = x[k2];
      x[k] = T2{fma(s, b2.y, c * b1.x), fma(-s, b2.x, c * b1.y)};
      x[k2] = T2{fma(s, b1.y, c * b2.x), fma(-s, b1.x, c * b2.y)};
    }
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
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    if (KU && (k & HB)) continue;
    uint32_t p = pt;
#pragma unroll
    for (int i = 0; i < B; ++i)
      if ((k >> i) & 1) p ^= pr[i];
    const T2* v = tb + p * uint32_t(ns);
    if (KU == 0) {
      const T2 v0 = v[0];
      x[k] = T2{fma(v0.x, x[k].x, -v0.y * x[k].y), fma(v0.x, x[k].y, v0.y * x[k].x)};
    } else {
      const int k2 = k ^ KU;
      uint32_t p2 = pt;
#pragma unroll
      for (int i = 0; i < B; ++i)
        if ((k2 >> i) & 1) p2 ^= pr[i];
      const T2* w = tb + p2 * uint32_t(ns);
      const T2 a0 = v[0], a1 = v[1], c0 = w[0], c1 = w[1];
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

// Register flips the planner may emit: one or two register bits.
#define HS_Q_KU_LIST(X) \
  X(1) X(2) X(4) X(8) X(16) X(3) X(5) X(6) X(9) X(10) X(12) X(17) X(18) X(20) X(24)

template <typename R, int NR>
__device__ __forceinline__ void rot_dispatch(typename C2<R>::T (&x)[NR], int ku, R c, R s, bool fast, int q,
                                          uint32_t zk, int sb) {
  switch (ku) {
#define HS_Q_ROT_CASE(K) \
  case K:                \
    if constexpr (K < NR) rot_ku<R, NR, K>(x, c, s, fast, q, zk, sb); \
    break;
    HS_Q_KU_LIST(HS_Q_ROT_CASE)
#undef HS_Q_ROT_CASE
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
// PHASE: x[k] <- e0 exp(-i pi phi_k) x[k], phi = WHT(E) over the register bits.
// ---------------------------------------------------------------------------
template <typename R, int NR>
__device__ __forceinline__ void phase_apply(typename C2<R>::T (&x)[NR], const Args& a, int pi, const R* Cs,
                                         typename C2<R>::T e0, uint32_t lt) {
  using T2 = typename C2<R>::T;
  const Phase& P = a.ph[pi];
  R E[NR];
#pragma unroll
  for (int mu = 0; mu < NR; ++mu) {
    R e = R(0);
    if ((P.mu_mask >> mu) & 1u) {
      const int c1 = P.cls0 + P.mu_beg[mu + 1];
      for (int cc = P.cls0 + P.mu_beg[mu]; cc < c1; ++cc) {
        const R v = Cs[cc];
        e += parity(a.cls[cc].thr & lt) ? -v : v;
      }
    }
    E[mu] = e;
  }
#pragma unroll
  for (int h = 1; h < NR; h <<= 1)
#pragma unroll
    for (int k = 0; k < NR; ++k)
      if (!(k & h)) {
        const R u = E[k], v = E[k | h];
        E[k] = u + v;
        E[k | h] = u - v;
      }
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    R sn, cn;
    sincospi_r(E[k], &sn, &cn);
    // e0 * (cn - i sn)
    const R px = fma(e0.x, cn, e0.y * sn), py = fma(e0.y, cn, -e0.x * sn);
    x[k] = cmul<T2, R>(x[k], px, py);
  }
}

// ---------------------------------------------------------------------------
// The kernel.  NT = 2^(T - B) threads; NR = 2^B rows per thread.
// ---------------------------------------------------------------------------
template <typename R, int B>
__global__ void __launch_bounds__(B == 5 ? 256 : 512, B == 5 ? 2 : 1) qsweep_kernel(const __grid_constant__ Args a) {
  using T2 = typename C2<R>::T;
  constexpr int NR = 1 << B;
  constexpr int V = 16 / int(sizeof(T2));  // rows per 16-byte chunk (2 for complex64)
  constexpr int VB = V == 2 ? 1 : 0;       // register bits inside a chunk
  constexpr int NJ = NR / V;               // chunks per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  const uint32_t tid = threadIdx.x;
  const uint32_t TS = 1u << a.tile_bits;
  const uint32_t n_chunks = TS / V;
  const uint32_t m0 = a.m0, m1 = a.m1;
  const int sh = a.sh;

  // Shared memory: [tile][rotation (cos, sin)][value tables][e0 per phase][class constants]
  T2* tile = reinterpret_cast<T2*>(smem_raw);
  T2* rcs = tile + TS;
  T2* vts = rcs + a.n_rot;
  T2* e0s = vts + a.n_vt;
  R* Cs = reinterpret_cast<R*>(e0s + a.n_phase);

  // Per-CTA tables (written by launches that completed before this grid began).
  for (int i = tid; i < a.n_rot; i += NT) {
    const double* p = a.cs + 2 * int64_t(a.rot[i].cs);
    rcs[i] = T2{R(p[0]), R(p[1])};
  }
  for (int t = 0; t < a.n_tab; ++t) {
    const Tab& tb = a.tab[t];
    const T2* g = reinterpret_cast<const T2*>(a.vt) + tb.vt0;
    for (int e = tid; e < tb.n; e += NT) vts[tb.s0 + e] = g[e];
  }

  const uint32_t u0 = blockIdx.x * uint32_t(a.units_per_cta);
  const uint32_t u1 = min(uint32_t(a.n_units), u0 + uint32_t(a.units_per_cta));
  for (uint32_t unit = u0; unit < u1; ++unit) {
    const uint32_t tile_id = unit & ((1u << a.n_tiles_log2) - 1u);
    const int rhs = int(unit >> a.n_tiles_log2);
    const uint32_t base = deposit_runs(tile_id, a.rest);
    const T2* src = reinterpret_cast<const T2*>(a.src) + int64_t(rhs) * a.N;
    T2* dst = reinterpret_cast<T2*>(a.dst) + int64_t(rhs) * a.N;
    __syncthreads();  // the previous unit is done with the tile and the per-tile constants
    if (unit == u0) {
      // The state written by the previous launch is visible only after this;
      // the next sweep may start its table loads meanwhile.
      grid_dependency_wait();
      grid_launch_dependents();
    }
    for (uint32_t c = tid; c < n_chunks; c += NT)
      cp_async16(tile + swz(c) * V, src + (global_of(c * V, m0, m1, sh) | base));
    cp_async_commit();
    // Per-tile phase constants: class sums of +-theta_j in FP64 with the signs
    // of the tile's fixed bits; a constant class becomes its phase op's e0.
    for (int cc = tid; cc < a.n_cls; cc += NT) {
      const PClass& C = a.cls[cc];
      double acc = 0.0;
      for (int t = C.t0; t < C.t0 + C.nt; ++t) {
        const PTerm& pt = a.pt[t];
        const double th = a.th[pt.th];
        acc += parity(pt.rest & base) ? -th : th;
      }
      if (C.c0p >= 0) {
        double sn, cn;
        sincos(acc, &sn, &cn);
        e0s[C.c0p] = T2{R(cn), R(-sn)};
      }
      Cs[cc] = R(acc * 0.318309886183790671537767526745);  // in units of pi
    }
    cp_async_wait(0);

    T2 x[NR];
    int cur = -1;
    uint32_t lt = 0, st = 0, gt = 0;  // row of register index 0: local, swizzled chunk, global
    auto chunk_of = [&](int j) -> uint32_t {
      const Layout& L = a.lay[cur];
      uint32_t pc = st;
#pragma unroll
      for (int i = 0; i < B - VB; ++i)
        if ((j >> i) & 1) pc ^= L.qoff[i + VB];
      return pc;
    };
    auto load_rows = [&]() {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const uint32_t pc = chunk_of(j);
        if constexpr (V == 2) {
          const float4 w = *reinterpret_cast<const float4*>(tile + pc * 2);
          x[2 * j] = T2{w.x, w.y};
          x[2 * j + 1] = T2{w.z, w.w};
        } else {
          x[j] = tile[pc];
        }
      }
    };
    auto store_rows = [&]() {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const uint32_t pc = chunk_of(j);
        if constexpr (V == 2) {
          *reinterpret_cast<float4*>(tile + pc * 2) = make_float4(x[2 * j].x, x[2 * j].y, x[2 * j + 1].x,
                                                                  x[2 * j + 1].y);
        } else {
          tile[pc] = x[j];
        }
      }
    };

    for (int oi = 0; oi < a.n_ops; ++oi) {
      const Op op = a.ops[oi];
      if (op.type == OP_LAYOUT) {
        __syncthreads();  // every thread is done reading the previous layout (or the copies have landed)
        if (cur >= 0) {
          store_rows();
          __syncthreads();
        }
        const Layout& L = a.lay[op.idx];
        uint32_t l = 0;
        for (int i = 0; i < L.n_thr; ++i) l |= ((tid >> i) & 1u) << L.thr[i];
        lt = l;
        st = swz(l >> VB);
        gt = global_of(l, m0, m1, sh) | base;
        cur = op.idx;
        load_rows();
      } else if (op.type == OP_ROT) {
        const T2 cs = rcs[op.idx];
        const bool fast = op.flags & 1;
        const int sb = fast ? 0 : (parity(op.zrest & base) ^ parity(op.zthr & lt));
        rot_dispatch<R, NR>(x, op.ku, cs.x, cs.y, fast, (op.flags >> 1) & 3, op.zk, sb);
      } else if (op.type == OP_TAB) {
        const Tab& tb = a.tab[op.idx];
        const Layout& L = a.lay[cur];
        uint32_t pr[B];
#pragma unroll
        for (int i = 0; i < B; ++i) pr[i] = pattern_fast(L.goff[i], tb.sm, tb.sh);
        tab_dispatch<R, NR, B>(x, op.ku, vts + tb.s0, tb.ns, pattern_fast(gt, tb.sm, tb.sh), pr);
      } else {
        phase_apply<R, NR>(x, a, op.idx, Cs, e0s[op.idx], lt);
      }
    }
    __syncthreads();
    store_rows();
    __syncthreads();
    for (uint32_t c = tid; c < n_chunks; c += NT)
      *reinterpret_cast<uint4*>(dst + (global_of(c * V, m0, m1, sh) | base)) =
          *reinterpret_cast<const uint4*>(tile + swz(c) * V);
  }
}

using QFn = void (*)(Args);

QFn qsweep_fn(hs_dtype dt, int B) {
  if (dt == HS_C64) return B == 5 ? qsweep_kernel<float, 5> : (B == 4 ? qsweep_kernel<float, 4> : nullptr);
  return B == 4 ? qsweep_kernel<double, 4> : nullptr;
}

}  // namespace

cudaError_t prepare_qsweep() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && done[dev]) return cudaSuccess;
  const QFn fns[3] = {qsweep_kernel<float, 5>, qsweep_kernel<float, 4>, qsweep_kernel<double, 4>};
  for (QFn fn : fns) {
    e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSweepSmemMax));
    if (e != cudaSuccess) return e;
  }
  if (dev < 64) done[dev] = true;
  return cudaSuccess;
}

size_t qsweep_smem_bytes(const Args& a, hs_dtype dt) {
  const size_t e = elem_bytes(dt), r = e / 2;
  return ((size_t(1) << a.tile_bits) + a.n_rot + a.n_vt + a.n_phase) * e + size_t(a.n_cls) * r;
}

cudaError_t launch_qsweep(const hs_factors* f, Args& a, const void* src, void* dst, int n_rhs, int B, bool pdl,
                          cudaStream_t s) {
  const Plan& p = f->plan;
  QFn fn = qsweep_fn(f->dtype, B);
  if (!fn || a.tile_bits - B < 5 || a.tile_bits > p.n_qubits) return cudaErrorInvalidValue;
  a.src = src;
  a.dst = dst;
  a.cs = f->bin.cs;
  a.th = f->bin.th;
  a.vt = f->d_vt;
  a.N = p.N;
  a.n_rhs = n_rhs;
  a.n_tiles_log2 = p.n_qubits - a.tile_bits;
  a.n_units = (1 << a.n_tiles_log2) * n_rhs;
  if (a.units_per_cta < 1) a.units_per_cta = 1;
  const size_t smem = qsweep_smem_bytes(a, f->dtype);
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
