// Register-blocked tile sweep ("q-sweep"): launch descriptor shared by the
// host planner (qplan.cpp) and the kernel (qsweep.cu).
//
// A CTA holds a tile of 2^T amplitudes of ONE state (the rows whose bits
// outside the tile's local bit set are fixed by the CTA index, as in the
// staged sweep) in shared memory, and each thread keeps 2^B of the tile's
// rows in registers: the rows l = l_t | pdep(k, reg) for k = 0 .. 2^B - 1,
// where `reg` is a set of B local bits (the register bits) and l_t places the
// thread index on the other local bits.  A factor whose flips lie in the
// register bits is applied in registers with no exchange; a LAYOUT op changes
// the register bits by one pass through shared memory.
//
// A factor of the sweep becomes a short list of ops:
//   TAB    a factor with a value table and at most two slots (x-mask set
//          {0, u}): row r's entries F[r, r] and F[r, r ^ u] are read from the
//          table at the pattern of r's bits on the factor's support;
//   ROT    one non-diagonal term of a factor without such a table: its exact
//          rotation cos(theta) I - i sin(theta) P_j, from the FP64 (cos, sin)
//          of the factor build; an X-type term (y = 0, z = 0) in the form
//          cos(theta') (I - i tan(theta') P_j) (-i P_j)^k, theta = theta' +
//          k pi / 2, |theta'| <= pi / 4: two fused multiply-adds per
//          amplitude, cos(theta') and (-i)^k in one scale per sweep, an odd
//          k a swap of partner rows;
//   ROTN   a run of consecutive X-type single-qubit rotations on distinct
//          register bits (they commute), applied back to back in that form;
//   DROT   a single diagonal term between non-diagonal ones: its rotation
//          exp(-i theta (-1)^popcount(z & r)) from the build's FP64 (cos, sin);
//   PHASE  a run of consecutive diagonal terms (x = 0) of such a factor: the
//          phase exp(-i sum_j theta_j (-1)^popcount(z_j & r)) computed for
//          each row from (z_j, theta_j) -- the factor values are generated
//          inside the sweep instead of being read from stored diagonals.
// Terms of a factor are applied in the factor's order, so a factor's ops
// multiply out to the factor itself (F_g = R_last ... R_first).
#pragma once

#include <cstdint>
#include <memory>
#include <utility>

#include "hs_internal.h"

namespace hs {
namespace q {

constexpr int kMaxOps = 160;
constexpr int kMaxLayouts = 40;
constexpr int kMaxRot = 96;
constexpr int kMaxTab = 24;
constexpr int kMaxPhase = 12;
constexpr int kMaxPTerms = 320;
constexpr int kMaxClasses = 256;
constexpr int kMaxVt = 2048;   // value-table entries held in shared memory
constexpr int kMaxB = 5;       // register bits per thread

enum : uint8_t { OP_ROT = 0, OP_TAB = 1, OP_PHASE = 2, OP_LAYOUT = 3, OP_ROTN = 4, OP_DROT = 5 };

struct Op {
  uint8_t type;
  uint8_t ku;     // ROT, TAB: the flip in register coordinates (TAB: 0 for a one-slot factor)
  uint8_t zk;     // ROT: the register coordinates of z's bits in the tile
  uint8_t flags;  // ROT: bit 0 = fast path (y = 0 and z = 0); bits 1-2 = q with -i i^y = i^q
  int16_t idx;    // ROT: rotation slot; TAB: table slot; PHASE: phase slot; LAYOUT: layout slot
  int16_t pad;
  uint32_t zthr;  // ROT: z's bits in the tile on thread positions (local-index mask)
  uint32_t zrest; // ROT: z's bits outside the tile (global mask)
  // ROTN (a run of consecutive rotations exp(-i theta X_q) on distinct single
  // register bits, which commute): ku is the mask of those register bits and
  // byte i of (zthr, zrest) the rotation slot of register bit i.
};

struct Layout {
  uint32_t reg;        // local-index mask of the register bits (register bit i = i-th lowest set bit)
  uint32_t qoff[kMaxB];  // per register bit: XOR offset of the physical 16-byte chunk index
  uint32_t goff[kMaxB];  // per register bit: global row offset (global image of the local bit)
  int8_t thr[28];      // local positions of the thread-index bits, thread bit 0 first
  int32_t n_thr;
  // A warp's rows (fixed warp bits, all register and lane bits) copied in
  // address order: chunk e = lane + 32 m of the warp's set lies at chunk
  // pdep(lane, wlo) ^ pdep(32 m, W) ^ (the warp's fixed chunk bits), W the
  // warp's chunk bits; mswz / mglob hold the swizzled chunk and global row
  // of pdep(32 m, W).
  int8_t wlo[5];       // the five lowest chunk bits of W
  int8_t pad[3];
  uint32_t mswz[1 << (kMaxB - 1)];
  uint32_t mglob[1 << (kMaxB - 1)];
};

struct Rot {
  int32_t cs;    // index of the term's (cos, sin) pair in the factor set's angle table
  int32_t fast;  // y = 0 and z = 0: kept as a ratio with its larger factor in the sweep's scale
};

struct Tab {
  int32_t vt0;  // first entry in the factor set's value tables
  int32_t s0;   // first entry in shared memory
  int32_t n;    // entries
  uint32_t sm;  // support mask (global bits); the pattern of row r indexes the table
  int8_t sh;    // lowest bit of sm when its bits are consecutive, else -1
  int8_t ns;    // slots (1 or 2)
  int16_t pad;
};

struct Phase {
  int16_t cls0, ncls;  // classes [cls0, cls0 + ncls); class cls0 has the empty local part
  uint32_t mu_mask;    // register patterns mu that have at least one class besides cls0
  int16_t mu_beg[(1 << kMaxB) + 1];  // per mu: first class (relative to cls0; mu = 0 starts
                                     // after the constant class), sentinel last
};

struct PClass {
  uint32_t thr;   // local part on thread positions (local-index mask)
  int16_t t0, nt; // terms [t0, t0 + nt) of the phase term list
  int16_t c0p;    // the phase op whose constant class (empty local part) this is, else -1
  int16_t mu;     // register part (register coordinates)
};

struct PTerm {
  int32_t th;     // index of theta_j in the factor set's angle table
  uint32_t rest;  // z_j's bits outside the tile (global mask)
};

struct Args {
  const void* src;
  void* dst;
  const double* cs;  // (cos, sin) per kind and term (FP64)
  const double* th;  // theta per kind and term (FP64)
  const double* rq;  // register-sweep record per kind and term (FP64, see the factor build)
  const void* vt;    // value tables (storage type)
  int64_t N;
  int64_t n_vt_g;    // extents of vt and of the per-term records (index checks only)
  int n_terms_g;
  int n_rhs;
  int tile_bits;
  int n_tiles_log2;
  int n_units;
  int units_per_cta;
  uint32_t m0, m1;  // local index of global row r: (r & m0) | ((r >> sh) & m1)
  int sh;
  Runs rest;
  int n_ops, n_lay, n_rot, n_tab, n_phase, n_cls, n_pterm, n_vt;
  int full;          // 1 if a TAB op or a rotation other than tan form occurs (the larger kernel)
  Op ops[kMaxOps];
  Layout lay[kMaxLayouts];
  Rot rot[kMaxRot];
  Tab tab[kMaxTab];
  Phase ph[kMaxPhase];
  PClass cls[kMaxClasses];
  PTerm pt[kMaxPTerms];
};

// Physical 16-byte chunk of natural chunk c in the shared-memory tile: the
// XOR fold of c's higher bit triples into its lowest three bits spreads the
// chunks a quarter-warp touches over distinct 16-byte bank groups.
__host__ __device__ __forceinline__ uint32_t swz(uint32_t c) {
  return c ^ (((c >> 3) ^ (c >> 6) ^ (c >> 9) ^ (c >> 12) ^ (c >> 15)) & 7u);
}

// Host planner: the ops of a fused sweep (factors in order, two-run local mask)
// for tiles of T bits and B register bits.  Returns false (with a reason) when
// a factor cannot be expressed as register ops or a limit is exceeded.
// steps (optional): the step of each factor application, for a sweep that
// spans steps of a time-dependent set whose terms have one record per step:
// a term record is then addressed (step - steps[0]) * step_stride + kind * m
// + term, relative to the records of the sweep's first step.
bool plan_qsweep(const hs_factors* f, const std::vector<int>& factors, uint32_t local_mask, int T, int B,
                 Args& a, std::string* why, const std::vector<int>* steps = nullptr, int step_stride = 0);

// The same for a run of factors that may exceed a descriptor's limits: the
// run is split into consecutive shorter runs (same local mask) until each
// fits.  Returns false if a single factor cannot be expressed.
bool plan_qsweep_runs(const hs_factors* f, const std::vector<int>& factors, uint32_t local_mask, int T, int B,
                      std::vector<std::pair<std::vector<int>, std::shared_ptr<Args>>>& out, std::string* why,
                      const std::vector<int>* steps = nullptr, int step_stride = 0);

size_t qsweep_smem_bytes(const Args& a, hs_dtype dt, int B);

// The job-dependent fields of a descriptor: state (evolved in place), the
// factor set's angle records and value tables, and the unit count (tiles of
// the planned local mask times n_rhs states).
void fill_job(const hs_factors* f, Args& a, void* psi, int n_rhs);

// One level of a batch of register sweeps: CTA c runs unit c - prefix[e] of
// descriptor lvl_desc[off + e], e the last entry with prefix[off + e] <= c.
struct LevelArgs {
  const Args* descs;
  const int* lvl_desc;
  const int* lvl_prefix;
  int off, count;
  uint32_t prefix_smem;  // byte offset of the level's prefix table in shared memory
};
cudaError_t launch_qlevel(hs_dtype dt, int B, bool full, int tile_bits, const LevelArgs& L, int64_t ctas, size_t smem,
                          cudaStream_t s);
// rq, cs (optional): term records to use instead of the factor set's own
// (n_terms of them), for a sweep over steps of a time-dependent set.
cudaError_t launch_qsweep(const hs_factors* f, Args& a, const void* src, void* dst, int n_rhs, int B,
                          bool pdl, cudaStream_t s, const double* rq = nullptr, const double* cs = nullptr,
                          int n_terms = 0);
cudaError_t prepare_qsweep();

}  // namespace q
}  // namespace hs
