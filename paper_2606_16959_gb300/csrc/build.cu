// Factor construction on the GPU in FP64 (Eq. 4 factors, Eq. 6 layout).
//
// Each factor is F_g = R_last ... R_first with R_j = cos(theta_j) I -
// i sin(theta_j) P_j.  One thread computes one ROW r of F_g: the row is the
// conjugate of F_g^dagger e_r, and F_g^dagger e_r = R_first^dagger ... R_last^dagger e_r
// is a vector supported on r xor X, where X (the group's x-mask space) has
// 2^xdim elements.  It is kept as 2^xdim FP64 complex slots indexed by GF(2)
// coordinates in the group's reduced echelon basis.  The thread then writes
// row r's entry on every structural diagonal of the factor (zero where
// r xor (r+d) is not in X), so writes are coalesced along each diagonal and
// no separate clearing pass is needed.  Values are rounded once to float2
// for complex64 storage.
#include <cuda_runtime.h>

#include <cstdint>

#include "counters.h"
#include "bounds.cuh"
#include "hs_internal.h"

namespace hs {
namespace {

struct BuildArgs {
  void* vals;
  const int64_t* offs;
  const int64_t* rowbase;
  const int* fac_D;
  const int* fac_diag0;
  const double* cs;  // (cos, sin) per term
  const double* th;  // theta per term (same indexing as cs / 2)
  const uint64_t* x;
  const uint64_t* z;
  const uint32_t* cx;
  const int* gfirst;
  const int* glast;
  const uint64_t* basis;  // kMaxXDim per group
  const int* xdim;
  const int* pivot;       // kMaxXDim per group
  int64_t N;
  const uint32_t* smask;  // per group: support mask of its value table
  const int* vt0;         // per group: first value-table entry, -1 if none
  const void* vt;         // value tables (filled before the diagonals)
  const int* kind;        // per group: angle kind (cs holds m (cos, sin) pairs per kind)
  const int* dir;         // per group: +1 terms first..last act in order, -1 reversed
  int m;                  // number of terms
  const int* glist;       // groups of grid row blockIdx.y (NULL: group blockIdx.y)
  int64_t n_vals, n_vt;   // extents of vals and vt (index checks only)
};

__device__ __forceinline__ int group_of(const BuildArgs& a) {
  return a.glist ? a.glist[blockIdx.y] : int(blockIdx.y);
}

__device__ __forceinline__ double2 mul_ipow(double2 v, int k) {
  switch (k & 3) {
    case 0: return v;
    case 1: return make_double2(-v.y, v.x);
    case 2: return make_double2(-v.x, -v.y);
    default: return make_double2(v.y, -v.x);
  }
}

__device__ __forceinline__ void store_val(void* vals, int64_t idx, double2 v, bool c64) {
  if (c64)
    reinterpret_cast<float2*>(vals)[idx] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  else
    reinterpret_cast<double2*>(vals)[idx] = v;
}

// Group g's basis, pivots, slot x-masks and term range, read once per thread.
template <int MAXS>
struct GroupRows {
  int xd, S, first, last, dir;
  const double* cs;  // this group's angle kind
  const double* th;
  uint64_t bas[kMaxXDim];
  int piv[kMaxXDim];
  uint64_t u[MAXS];
  __device__ __forceinline__ void load(const BuildArgs& a, int g) {
    xd = a.xdim[g];
    S = 1 << xd;
#pragma unroll
    for (int i = 0; i < kMaxXDim; ++i) {
      bas[i] = (i < xd) ? a.basis[g * kMaxXDim + i] : 0;
      piv[i] = (i < xd) ? a.pivot[g * kMaxXDim + i] : 0;
    }
    first = a.gfirst[g];
    last = a.glast[g];
    dir = a.dir[g];
    cs = a.cs + size_t(2) * a.m * a.kind[g];
    th = a.th + size_t(a.m) * a.kind[g];
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
      uint64_t m = 0;
#pragma unroll
      for (int i = 0; i < kMaxXDim; ++i)
        if (i < xd && ((s >> i) & 1)) m ^= bas[i];
      u[s] = m;
    }
  }
  // w[s] = slot s of F_g^dagger e_r (the conjugate of row r of F_g at column
  // r ^ u_s), by applying R_j^dagger = cos I + i sin P_j in the reverse of the
  // order in which F_g applies the R_j: j = last-1 .. first for a forward
  // factor (F_g = R_last ... R_first), j = first .. last-1 for a reversed one.
  // A run of consecutive diagonal terms (x_j = 0) commutes and multiplies each
  // slot by a phase: R_j^dagger scales basis state b by exp(+i theta_j
  // (-1)^popcount(z_j & b)), so the run's angles are summed per slot and
  // applied with one FP64 sincos per slot when the run ends.
  __device__ __forceinline__ void row(const BuildArgs& a, uint64_t r, double2 (&w)[MAXS]) const {
    double2 nw[MAXS];
    double phi[MAXS];
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
      w[s] = make_double2(s == 0 ? 1.0 : 0.0, 0.0);
      phi[s] = 0.0;
    }
    bool pending = false;
    const int n_t = last - first;
    for (int q = 0; q <= n_t; ++q) {
      const int j = dir > 0 ? last - 1 - q : first + q;
      const uint64_t xj = q < n_t ? a.x[j] : 1;
      if (q < n_t && xj == 0) {
        const double t = th[j];
        const uint64_t zj = a.z[j];
#pragma unroll
        for (int s = 0; s < MAXS; ++s)
          if (s < S) phi[s] += (__popcll(zj & (r ^ u[s])) & 1) ? -t : t;
        pending = true;
        continue;
      }
      if (pending) {
#pragma unroll
        for (int s = 0; s < MAXS; ++s)
          if (s < S) {
            double sn, c;
            sincos(phi[s], &sn, &c);
            w[s] = make_double2(c * w[s].x - sn * w[s].y, c * w[s].y + sn * w[s].x);
            phi[s] = 0.0;
          }
        pending = false;
      }
      if (q == n_t) break;
      const double c = cs[2 * j], sn = cs[2 * j + 1];
      const uint64_t zj = a.z[j];
      const int y = __popcll(xj & zj);
      const uint32_t cxj = a.cx[j];
#pragma unroll
      for (int s = 0; s < MAXS; ++s) {
        if (s < S) {
          const int src = s ^ int(cxj);
          // P_j maps slot src (basis state r ^ u[src]) to slot s with phase
          // i^y (-1)^popcount(z & (r ^ u[src])); times i sin.
          const int par = __popcll(zj & (r ^ u[src])) & 1;
          double2 p = mul_ipow(w[src], y + 1 + 2 * par);
          nw[s] = make_double2(fma(c, w[s].x, sn * p.x), fma(c, w[s].y, sn * p.y));
        }
      }
#pragma unroll
      for (int s = 0; s < MAXS; ++s)
        if (s < S) w[s] = nw[s];
    }
  }

  // Rows r and r ^ u_1 of a factor with a two-element x-mask set {0, u_1}, r
  // without the pivot bit: the slots of both rows are the basis states r and
  // r ^ u_1, so a diagonal run's phases are formed once for the pair.  With
  // s_j(b) = (-1)^popcount(z_j & b), s_j(r ^ u_1) = s_j(r) (-1)^popcount(z_j & u_1):
  // the run's angles s_j(r) theta_j sum to A over terms with an even overlap
  // with u_1 and to B over the others, and phi(r) = A + B, phi(r ^ u_1) = A - B.
  __device__ __forceinline__ void row_pair(const BuildArgs& a, uint64_t r, double2 (&w0)[2], double2 (&w1)[2]) const {
    const uint64_t u1 = bas[0];
    const uint64_t r1 = r ^ u1;
    w0[0] = make_double2(1.0, 0.0);
    w0[1] = make_double2(0.0, 0.0);
    w1[0] = w0[0];
    w1[1] = w0[1];
    double A = 0.0, B = 0.0;
    bool pending = false;
    const int n_t = last - first;
    for (int q = 0; q <= n_t; ++q) {
      const int j = dir > 0 ? last - 1 - q : first + q;
      const uint64_t xj = q < n_t ? a.x[j] : 1;
      if (q < n_t && xj == 0) {
        const double t = th[j];
        const uint64_t zj = a.z[j];
        const double st = (__popcll(zj & r) & 1) ? -t : t;
        if (__popcll(zj & u1) & 1) B += st;
        else A += st;
        pending = true;
        continue;
      }
      if (pending) {
        double s0, c0, s1, c1;
        sincos(A + B, &s0, &c0);  // basis state r
        sincos(A - B, &s1, &c1);  // basis state r ^ u_1
        auto mulp = [](double2& v, double c, double sn) {
          v = make_double2(c * v.x - sn * v.y, c * v.y + sn * v.x);
        };
        mulp(w0[0], c0, s0);  // row r, slot 0: state r
        mulp(w0[1], c1, s1);  // row r, slot 1: state r ^ u_1
        mulp(w1[0], c1, s1);  // row r ^ u_1, slot 0: state r ^ u_1
        mulp(w1[1], c0, s0);  // row r ^ u_1, slot 1: state r
        A = B = 0.0;
        pending = false;
      }
      if (q == n_t) break;
      const double c = cs[2 * j], sn = cs[2 * j + 1];
      const uint64_t zj = a.z[j];
      const int y = __popcll(xj & zj);
      const int cxj = int(a.cx[j]);
      auto rot = [&](uint64_t rr, double2 (&w)[2]) {
        double2 nw[2];
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
          const int src = s2 ^ cxj;
          const int par = __popcll(zj & (rr ^ (src ? u1 : 0ull))) & 1;
          const double2 p = mul_ipow(src ? w[1] : w[0], y + 1 + 2 * par);
          const double2 ws = s2 ? w[1] : w[0];
          nw[s2] = make_double2(fma(c, ws.x, sn * p.x), fma(c, ws.y, sn * p.y));
        }
        w[0] = nw[0];
        w[1] = nw[1];
      };
      rot(r, w0);
      rot(r1, w1);
    }
  }
};

// Row r of F on every structural diagonal: F[r, c] = conj(w[coord(r ^ c)])
// when r ^ c lies in X, an exact zero otherwise.
template <int NS, int MAXS>
__device__ __forceinline__ void write_row(const BuildArgs& a, const GroupRows<MAXS>& G, int D, int d0, int64_t r,
                                          const double2 (&w)[NS], bool c64) {
  for (int k = 0; k < D; ++k) {
    const int64_t d = a.offs[d0 + k];
    const int64_t col = r + d;
    if (col < 0 || col >= a.N) continue;
    const uint64_t uu = uint64_t(r) ^ uint64_t(col);
    int cc = 0;
    uint64_t rec = 0;
#pragma unroll
    for (int i = 0; i < kMaxXDim; ++i)
      if (i < G.xd && ((uu >> G.piv[i]) & 1ull)) {
        cc |= 1 << i;
        rec ^= G.bas[i];
      }
    double2 v = make_double2(0.0, 0.0);
    if (rec == uu) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (s == cc) v = make_double2(w[s].x, -w[s].y);
    }
    store_val(a.vals, HS_BCHK(a.rowbase[d0 + k] + r, a.n_vals, BS_BUILD_VAL), v, c64);
  }
}

// Rows of a factor with a value table: the entry of row r on diagonal d_k is
// table entry pattern(r) * S + cc, cc the coordinates of r ^ (r + d_k) in the
// factor's basis (an exact zero when that mask is outside the x-mask set).
// The table holds the stored values already rounded to the storage type, so
// they are copied in that type with no FP64 arithmetic.
template <typename T2, typename Grp>
__device__ __forceinline__ void copy_rows(const BuildArgs& a, const Grp& G, int D, int d0, int vt0, uint32_t sm) {
  const T2* __restrict__ vt = reinterpret_cast<const T2*>(a.vt);
  T2* __restrict__ vals = reinterpret_cast<T2*>(a.vals);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < a.N; r += stride) {
    uint32_t pat = 0;
    int q = 0;
    for (uint32_t t = sm; t; t &= t - 1u, ++q) pat |= uint32_t((uint64_t(r) >> (__ffs(t) - 1)) & 1u) << q;
    const int64_t e0 = int64_t(vt0) + int64_t(pat) * G.S;
    for (int k = 0; k < D; ++k) {
      const int64_t col = r + a.offs[d0 + k];
      if (col < 0 || col >= a.N) continue;
      const uint64_t uu = uint64_t(r) ^ uint64_t(col);
      int cc = 0;
      uint64_t rec = 0;
#pragma unroll
      for (int i = 0; i < kMaxXDim; ++i)
        if (i < G.xd && ((uu >> G.piv[i]) & 1ull)) {
          cc |= 1 << i;
          rec ^= G.bas[i];
        }
      T2 v;
      v.x = 0;
      v.y = 0;
      if (rec == uu) v = vt[HS_BCHK(e0 + cc, a.n_vt, BS_BUILD_VT)];
      vals[HS_BCHK(a.rowbase[d0 + k] + r, a.n_vals, BS_BUILD_VAL)] = v;
    }
  }
}

// A factor's x-mask basis and pivots (all that copying from its value table needs).
struct GroupBasis {
  int xd, S;
  uint64_t bas[kMaxXDim];
  int piv[kMaxXDim];
  __device__ __forceinline__ void load(const BuildArgs& a, int g) {
    xd = a.xdim[g];
    S = 1 << xd;
#pragma unroll
    for (int i = 0; i < kMaxXDim; ++i) {
      bas[i] = (i < xd) ? a.basis[g * kMaxXDim + i] : 0;
      piv[i] = (i < xd) ? a.pivot[g * kMaxXDim + i] : 0;
    }
  }
};

// The stored diagonals of factors with value tables, one diagonal at a time
// (its offset, row base and x-mask coordinates fixed for the whole pass), two
// consecutive rows per thread and one 2 x sizeof(T2) store: a streaming write
// with a few integer operations per element.  Row r's entry on diagonal d is
// table entry pattern(r) * S + cc when r ^ (r + d) = u_cc lies in the x-mask
// set, an exact zero otherwise.
static_assert(HS_MAX_QUBITS <= 30, "copy_diagonals keeps row indices and offsets in 32 bits");

template <typename T2>
__device__ __forceinline__ void copy_diagonals(const BuildArgs& a, const GroupBasis& G, int D, int d0, int vt0,
                                               uint32_t sm) {
  // Row and column indices fit in 32 bits (at most 2^30 rows), and so do the
  // x-mask basis and the offsets.
  const T2* __restrict__ vt = reinterpret_cast<const T2*>(a.vt);
  T2* __restrict__ vals = reinterpret_cast<T2*>(a.vals);
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t N = uint32_t(a.N);
  uint32_t bas[kMaxXDim];
#pragma unroll
  for (int i = 0; i < kMaxXDim; ++i) bas[i] = uint32_t(G.bas[i]);
  // pattern(r): r's bits at smask, packed; a window of consecutive bits is a
  // shift and a mask.
  const int sm_lo = sm ? __ffs(sm) - 1 : 0;
  const bool sm_window = ((sm >> sm_lo) & ((sm >> sm_lo) + 1u)) == 0u;
  auto pattern = [&](uint32_t r) -> uint32_t {
    if (sm_window) return (r & sm) >> sm_lo;
    uint32_t p = 0;
    int q = 0;
    for (uint32_t t = sm; t; t &= t - 1u, ++q) p |= ((r >> (__ffs(t) - 1)) & 1u) << q;
    return p;
  };
  for (int k = 0; k < D; ++k) {
    const int32_t d = int32_t(a.offs[d0 + k]);
    const int64_t rb = a.rowbase[d0 + k];
    auto value = [&](uint32_t r) -> T2 {
      const uint32_t uu = r ^ uint32_t(int32_t(r) + d);
      int cc = 0;
      uint32_t rec = 0;
#pragma unroll
      for (int i = 0; i < kMaxXDim; ++i)
        if (i < G.xd && ((uu >> G.piv[i]) & 1u)) {
          cc |= 1 << i;
          rec ^= bas[i];
        }
      T2 v;
      v.x = 0;
      v.y = 0;
      if (rec == uu) v = vt[HS_BCHK(int64_t(vt0) + int64_t(pattern(r)) * G.S + cc, a.n_vt, BS_BUILD_VT)];
      return v;
    };
    // Only the rows whose column is in range own an element of the diagonal
    // (the others lie in neighbouring diagonals' storage). Rows r0, r0 + 1
    // with r0 even: element rb + r0 is 16-byte aligned (the row base is a
    // multiple of 32 bytes), so a pair inside the range is one vector store.
    const uint32_t lo = d < 0 ? uint32_t(-d) : 0u, hi = d > 0 ? N - uint32_t(d) : N;
    for (uint32_t pr = (lo >> 1) + blockIdx.x * blockDim.x + threadIdx.x; pr < (hi + 1u) >> 1; pr += stride) {
      const uint32_t r0 = 2u * pr;
      const bool in0 = r0 >= lo && r0 < hi, in1 = r0 + 1u >= lo && r0 + 1u < hi;
      if (in0 && in1) {
        const T2 v0 = value(r0), v1 = value(r0 + 1u);
        if constexpr (sizeof(T2) == 8) {
          *reinterpret_cast<float4*>(vals + HS_BCHK(rb + r0, a.n_vals - 1, BS_BUILD_VAL)) =
              make_float4(v0.x, v0.y, v1.x, v1.y);
        } else {
          vals[HS_BCHK(rb + r0, a.n_vals, BS_BUILD_VAL)] = v0;
          vals[HS_BCHK(rb + r0 + 1, a.n_vals, BS_BUILD_VAL)] = v1;
        }
      } else {
        if (in0) vals[HS_BCHK(rb + r0, a.n_vals, BS_BUILD_VAL)] = value(r0);
        if (in1) vals[HS_BCHK(rb + r0 + 1, a.n_vals, BS_BUILD_VAL)] = value(r0 + 1u);
      }
    }
  }
}

// The stored diagonals of factors with value tables (few registers, so the
// copy runs at full occupancy whatever the widest factor of the set).
__global__ void __launch_bounds__(256) copy_kernel(BuildArgs a, bool c64) {
  const int g = group_of(a);
  const int vt0 = a.vt0[g];
  if (vt0 < 0) return;
  GroupBasis G;
  G.load(a, g);
  if (c64)
    copy_diagonals<float2>(a, G, a.fac_D[g], a.fac_diag0[g], vt0, a.smask[g]);
  else
    copy_diagonals<double2>(a, G, a.fac_D[g], a.fac_diag0[g], vt0, a.smask[g]);
}

template <int MAXS>
__global__ void __launch_bounds__(256) build_kernel(BuildArgs a, bool c64) {
  const int g = group_of(a);
  GroupRows<MAXS> G;
  G.load(a, g);
  const int D = a.fac_D[g], d0 = a.fac_diag0[g];
  const int vt0 = a.vt0[g];
  const uint32_t sm = a.smask[g];
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;

  if (vt0 >= 0) {
    if (c64)
      copy_rows<float2>(a, G, D, d0, vt0, sm);
    else
      copy_rows<double2>(a, G, D, d0, vt0, sm);
    return;
  }
  if (MAXS >= 2 && G.xd == 1) {
    // Two-element x-mask set: one thread per pair of rows (r, r ^ u_1).
    const int p = G.piv[0];
    const uint64_t lowm = (1ull << p) - 1ull;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < (a.N >> 1); k += stride) {
      const uint64_t r = ((uint64_t(k) >> p) << (p + 1)) | (uint64_t(k) & lowm);
      double2 w0[2], w1[2];
      G.row_pair(a, r, w0, w1);
      write_row(a, G, D, d0, int64_t(r), w0, c64);
      write_row(a, G, D, d0, int64_t(r ^ G.bas[0]), w1, c64);
    }
    return;
  }
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < a.N; r += stride) {
    double2 w[MAXS];
    G.row(a, uint64_t(r), w);
    write_row(a, G, D, d0, r, w, c64);
  }
}

// Value tables: for a factor with one, pattern p of the bits at smask stands
// for every row r with those bits; row r = the pattern deposited at smask (the
// other bits do not enter the row's values), entry p * nslot + s = F[r, r ^ u_s]
// = conj(w[s]), computed by the same arithmetic as the row's stored values.
template <int MAXS>
__global__ void __launch_bounds__(256) value_table_kernel(BuildArgs a, const uint32_t* smask, const int* vt0,
                                                          void* vt, bool c64) {
  const int g = group_of(a);
  if (vt0[g] < 0) return;
  const uint32_t sm = smask[g];
  const int bits = __popc(sm);
  const int p = int(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= (1 << bits)) return;
  GroupRows<MAXS> G;
  G.load(a, g);
  uint64_t r = 0;
  int q = 0;
  for (uint32_t t = sm; t; t &= t - 1u, ++q) r |= uint64_t((p >> q) & 1) << (__ffs(t) - 1);
  double2 w[MAXS];
  G.row(a, r, w);
#pragma unroll
  for (int s = 0; s < MAXS; ++s)
    if (s < G.S)
      store_val(vt, HS_BCHK(int64_t(vt0[g]) + int64_t(p) * G.S + s, a.n_vt, BS_BUILD_VT), make_double2(w[s].x, -w[s].y),
                c64);
}

// cs[2 (k n + j) + {0, 1}] = (cos, sin)(c_j * h[k]) for kind k, with c_j =
// coeff[j], or coeff[j] + f coeff1[j] (f = *fval, the product rounded before
// the sum, no fused multiply-add) for a time-dependent set.
// rq[4 (k n + j) + {0..3}]: what a register sweep needs of the rotation
// exp(-i theta P) = cos(theta') (I - i tan(theta') P) (-i P)^k, theta = theta'
// + k pi / 2 with |theta'| <= pi / 4: tan(theta'), k mod 4, cos(theta') and
// theta / pi reduced to [-1, 1].
// The records of term j at angle kind k: theta = c_j h_k with c_j = a_j, or
// a_j + f b_j (the product rounded before the sum, no fused multiply-add).
__device__ __forceinline__ void term_records(const double* coeff, const double* coeff1, double fv, const double* h,
                                             int k, int j, double* th, double* cs, double* rq) {
  double c = coeff[j];
  if (coeff1) c = __dadd_rn(c, __dmul_rn(fv, coeff1[j]));
  const double theta = c * h[k];
  if (th) *th = theta;
  double s, co;
  sincos(theta, &s, &co);
  cs[0] = co;
  cs[1] = s;
  // theta = pi u (mod 2 pi), u in [-1, 1]; u = v + k / 2 with k = rint(2 u)
  // and |v| <= 1/4 (an exact subtraction), so that
  // exp(-i theta P) = cos(pi v) (I - i tan(pi v) P) (-i P)^k.
  const double u0 = theta * 0.318309886183790671537767526745;
  const double u = u0 - 2.0 * rint(0.5 * u0);
  const double kh = rint(2.0 * u);
  const double v = u - 0.5 * kh;
  double sv, cv;
  sincospi(v, &sv, &cv);
  rq[0] = sv / cv;
  rq[1] = double(int(kh) & 3);
  rq[2] = cv;
  rq[3] = u;
}

__global__ void sincos_kernel(const double* coeff, const double* coeff1, const double* fval, const double* h,
                              int n_kinds, double* cs, double* th, double* rq, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n * n_kinds) {
    const int k = e / n, j = e - k * n;
    term_records(coeff, coeff1, fval ? *fval : 0.0, h, k, j, th + e, cs + 2 * e, rq + 4 * e);
  }
}

// One set of records per drive sample: step blockIdx.y at offsets of
// n * n_kinds records.
__global__ void sincos_steps_kernel(const double* coeff, const double* coeff1, const double* fval, const double* h,
                                    int n_kinds, double* cs, double* rq, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int st = blockIdx.y;
  if (e < n * n_kinds) {
    const int k = e / n, j = e - k * n;
    const size_t r = size_t(st) * n * n_kinds + e;
    term_records(coeff, coeff1, fval[st], h, k, j, nullptr, cs + 2 * r, rq + 4 * r);
  }
}

BuildArgs build_args(const hs_factors* f, const int* glist) {
  const hs_build_inputs& b = f->bin;
  return BuildArgs{f->d_vals, f->d_offs, f->d_rowbase, f->d_fac_D, f->d_fac_diag0, b.cs, b.th, b.x, b.z, b.cx,
                   b.gfirst, b.glast, b.basis, b.xdim, b.pivot, f->plan.N, b.smask, b.vt0, f->d_vt, b.kind,
                   b.dir, int(f->plan.x.size()), glist, f->plan.total_elems, f->plan.total_vt};
}

}  // namespace

cudaError_t launch_sincos(const hs_factors* f, const double* d_fval, cudaStream_t s) {
  const hs_build_inputs& b = f->bin;
  const int n = int(f->plan.x.size());
  sincos_kernel<<<(n * b.n_kinds + 127) / 128, 128, 0, s>>>(b.coeff, b.coeff1, d_fval, b.h, b.n_kinds, b.cs, b.th,
                                                            b.rq, n);
  note_launches();
  return cudaGetLastError();
}

namespace {
cudaError_t launch_rows(const hs_factors* f, const int* d_groups, int n_groups, int maxdim, cudaStream_t s);
}

cudaError_t launch_sincos_steps(const hs_factors* f, const double* d_fval, int n_steps, double* cs_out,
                                double* rq_out, cudaStream_t s) {
  const hs_build_inputs& b = f->bin;
  const int n = int(f->plan.x.size());
  if (n_steps <= 0 || n_steps > 65535) return cudaErrorInvalidValue;
  sincos_steps_kernel<<<dim3((n * b.n_kinds + 127) / 128, n_steps), 128, 0, s>>>(b.coeff, b.coeff1, d_fval, b.h,
                                                                                b.n_kinds, cs_out, rq_out, n);
  note_launches();
  return cudaGetLastError();
}

cudaError_t launch_build(const hs_factors* f, const int* d_groups, int n_groups, cudaStream_t s) {
  const Plan& p = f->plan;
  const int G = d_groups ? n_groups : int(p.groups.size());
  if (G <= 0) return cudaSuccess;
  int maxdim = 0;
  for (const Group& g : p.groups) maxdim = g.xdim > maxdim ? g.xdim : maxdim;
  return launch_rows(f, d_groups, G, maxdim, s);
}

namespace {
cudaError_t launch_rows(const hs_factors* f, const int* d_groups, int G, int maxdim, cudaStream_t s) {
  const Plan& p = f->plan;
  const BuildArgs a = build_args(f, d_groups);
  const bool c64 = f->dtype == HS_C64;
  const int threads = 256;
  int64_t blocks_x = (p.N + threads - 1) / threads;
  if (blocks_x > 4096) blocks_x = 4096;
  const dim3 grid{unsigned(blocks_x), unsigned(G), 1u};
  switch (maxdim) {
    case 0: build_kernel<1><<<grid, threads, 0, s>>>(a, c64); break;
    case 1: build_kernel<2><<<grid, threads, 0, s>>>(a, c64); break;
    case 2: build_kernel<4><<<grid, threads, 0, s>>>(a, c64); break;
    case 3: build_kernel<8><<<grid, threads, 0, s>>>(a, c64); break;
    case 4: build_kernel<16><<<grid, threads, 0, s>>>(a, c64); break;
    case 5: build_kernel<32><<<grid, threads, 0, s>>>(a, c64); break;
    default: build_kernel<64><<<grid, threads, 0, s>>>(a, c64); break;
  }
  note_launches();
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_build_split(const hs_factors* f, const int* d_vt_groups, int n_vt, const int* d_row_groups,
                               int n_rows, cudaStream_t s) {
  const Plan& p = f->plan;
  const bool c64 = f->dtype == HS_C64;
  const int threads = 256;
  int64_t blocks_x = (p.N + threads - 1) / threads;
  if (blocks_x > 4096) blocks_x = 4096;
  if (n_vt > 0) {
    const BuildArgs a = build_args(f, d_vt_groups);
    copy_kernel<<<dim3{unsigned(blocks_x), unsigned(n_vt), 1u}, threads, 0, s>>>(a, c64);
    note_launches();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (n_rows > 0) {
    int maxdim = 0;
    for (const Group& g : p.groups)
      if (g.vt0 < 0) maxdim = g.xdim > maxdim ? g.xdim : maxdim;
    return launch_rows(f, d_row_groups, n_rows, maxdim, s);
  }
  return cudaSuccess;
}

cudaError_t launch_value_tables(const hs_factors* f, const int* d_groups, int n_groups, cudaStream_t s) {
  const Plan& p = f->plan;
  if (p.total_vt == 0) return cudaSuccess;
  const int G = d_groups ? n_groups : int(p.groups.size());
  if (G <= 0) return cudaSuccess;
  int maxdim = 0, maxbits = 0;
  for (const Group& g : p.groups)
    if (g.vt0 >= 0) {
      maxdim = g.xdim > maxdim ? g.xdim : maxdim;
      maxbits = __builtin_popcount(g.smask) > maxbits ? __builtin_popcount(g.smask) : maxbits;
    }
  const BuildArgs a = build_args(f, d_groups);
  const bool c64 = f->dtype == HS_C64;
  const hs_build_inputs& b = f->bin;
  const dim3 grid{unsigned(((1 << maxbits) + 255) / 256), unsigned(G), 1u};
  switch (maxdim) {
    case 0: value_table_kernel<1><<<grid, 256, 0, s>>>(a, b.smask, b.vt0, f->d_vt, c64); break;
    case 1: value_table_kernel<2><<<grid, 256, 0, s>>>(a, b.smask, b.vt0, f->d_vt, c64); break;
    case 2: value_table_kernel<4><<<grid, 256, 0, s>>>(a, b.smask, b.vt0, f->d_vt, c64); break;
    case 3: value_table_kernel<8><<<grid, 256, 0, s>>>(a, b.smask, b.vt0, f->d_vt, c64); break;
    case 4: value_table_kernel<16><<<grid, 256, 0, s>>>(a, b.smask, b.vt0, f->d_vt, c64); break;
    default: value_table_kernel<32><<<grid, 256, 0, s>>>(a, b.smask, b.vt0, f->d_vt, c64); break;
  }
  note_launches();
  return cudaGetLastError();
}

}  // namespace hs
