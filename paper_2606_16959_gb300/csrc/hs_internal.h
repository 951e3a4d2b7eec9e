// Internal declarations shared by the translation units of libhs.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hs.h"

namespace hs {

constexpr int kMaxDiags = 4096;     // diagonals per factor
constexpr int kMaxXDim = 6;         // log2 of the x-mask set size per factor
constexpr int kMaxRuns = 6;         // contiguous bit runs describing a tile's local bits
constexpr int kMaxSweepFactors = 64;
constexpr int kMaxFusedDiags = 32;                 // factors with more diagonals use the plain kernel
constexpr size_t kSweepSmemMax = 227 * 1024;       // opt-in shared memory per CTA
constexpr size_t kSweepSmemDefault = 112 * 1024;   // two sweep CTAs per SM
constexpr int kMaxVtBits = 8;       // qubits a factor's terms may touch for a value table
constexpr int kMaxVtSweep = 2048;   // value-table entries one sweep holds in shared memory

// Storage alignment of each diagonal's row-indexed base, in elements (32 bytes).
inline int64_t align_elems(hs_dtype dt) { return dt == HS_C64 ? 4 : 2; }
inline size_t elem_bytes(hs_dtype dt) { return dt == HS_C64 ? 8 : 16; }

// One grouped factor (a contiguous range of terms).
struct Group {
  int first = 0, last = 0;   // term range [first, last)
  int D = 0;                 // number of diagonals
  int diag0 = 0;             // index of its first diagonal in the global diagonal arrays
  int64_t S = 0;             // stored elements without padding (sum of N - |d|)
  uint64_t span = 0;         // OR of the x masks: the qubits the factor flips
  int xdim = 0;              // dimension of the x-mask space over GF(2)
  uint64_t basis[kMaxXDim];  // reduced echelon basis of the x-mask space
  int pivot[kMaxXDim];       // pivot bit of each basis vector
  // Slot tables (only for factors with at most kMaxFusedDiags diagonals):
  // slot s is the x-mask u_s = XOR of basis[i] over the set bits i of s; row r's
  // entry in column r ^ u_s lies on diagonal (r ^ u_s) - r, whose row-indexed
  // base is tab_rb[slot_tab[slot0 + s] + p] with p the bits of r at the set
  // bits of u_s (lowest bit of u_s -> bit 0 of p).
  int slot0 = 0;             // first slot in the global slot arrays
  int nslot = 0;             // 2^xdim, or 0 if the factor has no slot tables
  // Value table (factors with slot tables whose terms touch at most kMaxVtBits
  // qubits): entry (r, r ^ u_s) of the factor depends on r only through r's
  // bits at the union of its terms' x and z masks, so the values sit in a
  // table indexed p * nslot + s, p = r's bits at smask packed (lowest bit
  // first).  smask is that union, or the window of consecutive bits covering
  // it (then p = (r & smask) >> lowest bit, and rows differing only at the
  // window's other bits share values).
  uint32_t smask = 0;
  int vt0 = -1;              // first entry in the factor set's value tables, -1 if none
  int vt_n = 0;              // nslot << popcount(smask)
  // Product formula stage this factor belongs to: angle kind (which multiple
  // of the step its rotations use) and direction (+1: terms first..last act in
  // order, -1: last..first).
  int kind = 0;
  int dir = 1;
};

// Result of planning a factor set on the host.
struct Plan {
  int n_qubits = 0;
  int64_t N = 0;
  std::vector<uint64_t> x, z;
  std::vector<double> coeff;
  std::vector<Group> groups;
  std::vector<int64_t> offs;      // all diagonals, factor after factor, canonical order
  std::vector<int64_t> dstart;    // element index (padded storage) of element 0 of each diagonal
  std::vector<int64_t> rowbase;   // value(row r) of diagonal k sits at element rowbase[k] + r
  std::vector<uint32_t> term_cx;  // per term: coordinates of its x mask in its factor's basis
  int64_t total_elems = 0;        // padded storage size in elements
  int64_t total_vt = 0;           // value-table entries (stored after the diagonals)
  int order = 1;                  // product formula: 1, 2 (Strang) or 4 (Suzuki)
  int n_kinds = 1;                // distinct angle multiples of the step
  std::vector<int> step_seq;      // factors one step applies, in order
  std::vector<uint32_t> slot_u;   // per slot: its x-mask
  std::vector<int32_t> slot_tab;  // per slot: first entry in tab_rb (one sentinel at the end)
  std::vector<int64_t> tab_rb;    // per (slot, row pattern): row-indexed base of the diagonal
  int g0 = 0;                     // groups of the first-order grouping (factor g holds group g mod g0)
  std::vector<char> commute;      // g0 x g0: the groups' terms commute pairwise (empty above
                                  // kMaxCommuteGroups groups)
};

// Largest grouping for which the plan records which groups commute.
constexpr int kMaxCommuteGroups = 2048;

// Parse labels into masks.  Returns HS_OK or HS_EINVAL (message in *err).
int parse_labels(const char* const* labels, size_t n, std::vector<uint64_t>& x, std::vector<uint64_t>& z,
                 int& n_qubits, std::string* err);

// Group, order offsets and lay out storage.  Returns HS_OK or HS_EINVAL.
// order 2 / 4 lays out each group twice per angle kind (forward and reversed
// term order) and sets step_seq to the formula's sequence of factors.
int make_plan(const uint64_t* x, const uint64_t* z, const double* coeff, size_t n, int n_qubits, int budget,
              hs_dtype dt, Plan& plan, std::string* err, int order = 1);

// Angle multiples of the step dt for each kind of a product formula of the given order.
std::vector<double> kind_steps(int order, double dt);

// A tile partition: `local` bits (held by one CTA) and the rest (enumerated by the grid).
struct Runs {
  int n = 0;
  int8_t pos[kMaxRuns + 2];
  int8_t len[kMaxRuns + 2];
};

// One launch of the evolution schedule.
struct Sweep {
  bool fused = true;         // tile sweep (true) or plain diagonal-times-vector (false)
  uint32_t local_mask = 0;   // fused: bits held by a tile
  std::vector<int> factors;  // fused: factor ids in order; plain: exactly one
  std::vector<int> steps;    // the step of each factor application (for a planned register
                             // sweep: one entry, the step its descriptor's term records start at)
};

// Plan the launches for n_steps steps with tiles of tile_bits local bits.
// Factors with more than max_fused_diags diagonals, or whose flip span does not
// fit a tile, get plain launches.
std::vector<Sweep> plan_sweeps(const Plan& p, int n_steps, int tile_bits, int min_low_bits, bool fused,
                               int max_fused_diags = kMaxFusedDiags, int max_fuse = kMaxSweepFactors);
// As plan_sweeps with fused = true, but a sweep may also take later factor
// applications that commute with every application they pass over (up to two
// steps past the last one it takes), so the product is the formula's up to the
// order of commuting factors; the in-order schedule where that has no more
// sweeps. The steps of a sweep's applications are nondecreasing.
std::vector<Sweep> plan_sweeps_commuting(const Plan& p, int n_steps, int tile_bits, int min_low_bits,
                                         int max_fused_diags = kMaxFusedDiags, int max_fuse = kMaxSweepFactors);

// Decompose a bit mask into runs of consecutive set bits (low to high).
Runs runs_of(uint64_t mask, int n_bits);

// A tile's local bits [0, a) U [h, h + T - a) with a >= low_bits that cover
// `used` (the window is placed at the lowest used bit above a, moved down to
// fit below n); 0 if no such mask exists.  T >= n gives all n bits.
uint64_t two_run_mask(uint64_t used, int n, int T, int low_bits);

}  // namespace hs

// Device-resident inputs of a factor build (inside hs_factors::d_tables), kept
// so that the values can be rebuilt for new coefficients on the same structure.
struct hs_build_inputs {
  const uint64_t* x = nullptr;
  const uint64_t* z = nullptr;
  const double* coeff = nullptr;   // a_j (the only coefficients of a static set)
  const double* coeff1 = nullptr;  // b_j of H(t) = H0 + f(t) H1; NULL for a static set
  const uint32_t* cx = nullptr;
  const int* gfirst = nullptr;
  const int* glast = nullptr;
  const uint64_t* basis = nullptr;
  const int* xdim = nullptr;
  const int* pivot = nullptr;
  const uint32_t* smask = nullptr;
  const int* vt0 = nullptr;
  const int* kind = nullptr;
  const int* dir = nullptr;
  const double* h = nullptr;       // angle multiple of each kind
  double* cs = nullptr;            // (cos, sin) per kind and term, written on the device
  double* th = nullptr;            // the angle per kind and term, written on the device
  double* rq = nullptr;            // register-sweep record per kind and term (4 doubles), written on the device
  double* fval = nullptr;          // one drive value (hs_factors_set_drive)
  int n_kinds = 1;
  // Groups holding a term with b_j != 0: all of them, those without a value
  // table, those with one.
  const int* dep_all = nullptr;
  const int* dep_notab = nullptr;
  const int* dep_tab = nullptr;
  int n_dep_all = 0, n_dep_notab = 0, n_dep_tab = 0;
  // Every group with a value table, and every one without.
  const int* tab_groups = nullptr;
  const int* row_groups = nullptr;
  int n_tab_groups = 0, n_row_groups = 0;
};

// Opaque object behind the C ABI.
struct hs_factors {
  hs::Plan plan;
  hs_dtype dtype = HS_C64;
  int n_steps = 0;
  double t = 0.0;
  int device = 0;
  void* d_vals = nullptr;        // padded factor values (float2 / double2), then the value tables
  void* d_vt = nullptr;          // value tables (inside the d_vals allocation)
  void* d_tables = nullptr;      // one allocation holding every table below (and the build inputs)
  int64_t* d_offs = nullptr;     // per diagonal offset
  int64_t* d_rowbase = nullptr;  // per diagonal row-indexed base
  int* d_fac_D = nullptr;        // per factor diagonal count
  int* d_fac_diag0 = nullptr;    // per factor first diagonal index
  uint32_t* d_slot_u = nullptr;  // slot tables (see Group)
  int32_t* d_slot_tab = nullptr;
  int64_t* d_tab_rb = nullptr;
  hs_build_inputs bin;           // build inputs (device pointers into d_tables)
  double* d_drive = nullptr;     // drive samples of hs_evolve_td (library-owned)
  int drive_cap = 0;
  // HS_BUILD_DEFER_DIAGONALS: the stored diagonals are built by the first call
  // that needs them (hs::ensure_diagonals).
  mutable bool diag_pending = false;
  mutable std::mutex diag_mu;
  double* d_steprec = nullptr;   // per-step term records of register sweeps spanning steps (hs_evolve_td)
  size_t steprec_cap = 0;        // doubles
  // cached CUDA graphs of evolve launch sequences
  struct GraphKey {
    void* psi;
    int n_rhs, n_steps, method, tile_bits, rhs_block;
    cudaStream_t stream;
    int variant;  // 0: hs_evolve_ex, 1: hs_evolve_td
    bool operator<(const GraphKey& o) const;
  };
  mutable std::mutex graph_mu;
  mutable std::map<GraphKey, cudaGraphExec_t> graphs;
};

namespace hs {

// Kernel launchers (defined in the .cu files).
// (cos, sin) of c_j * h_k for every term j and angle kind k, kind-major, into
// f->bin.cs; c_j = a_j, or a_j + f b_j with f read from d_fval when the set is
// time-dependent (d_fval NULL: f = 0).
cudaError_t launch_sincos(const hs_factors* f, const double* d_fval, cudaStream_t s);
// The same per-term records for n_steps drive samples d_fval[0 .. n_steps),
// step k's (cos, sin) at cs_out + 2 k r and register-sweep records at
// rq_out + 4 k r, r = terms x angle kinds (one launch).
cudaError_t launch_sincos_steps(const hs_factors* f, const double* d_fval, int n_steps, double* cs_out,
                                double* rq_out, cudaStream_t s);
// Value tables of the listed groups (d_groups NULL: every group with a table).
cudaError_t launch_value_tables(const hs_factors* f, const int* d_groups, int n_groups, cudaStream_t s);
// Factor values of the listed groups (d_groups NULL: all); groups with a value
// table copy it, so their tables must be current (launch_value_tables first).
cudaError_t launch_build(const hs_factors* f, const int* d_groups, int n_groups, cudaStream_t s);
// The same with the groups split: those with value tables (copied from the
// tables) and those without (built row by row in FP64).
cudaError_t launch_build_split(const hs_factors* f, const int* d_vt_groups, int n_vt, const int* d_row_groups,
                               int n_rows, cudaStream_t s);

cudaError_t launch_apply_plain(const hs_factors* f, int g, const void* x, void* y, int n_rhs, cudaStream_t s);

struct SweepLaunch {
  const void* src;
  void* dst;
  int n_rhs;
  int rhs_block;
  int tile_bits;
  uint32_t local_mask;  // two-run local bit set (see two_run_mask)
  Runs rest;            // the other bits
  int n_factors;
  int factors[kMaxSweepFactors];
  size_t smem_budget;  // shared memory the launch may use (sets the number of factor stages)
  bool pdl;            // launch with programmatic dependent launch
  bool value_tables;   // read factors that have value tables from them instead of staging planes
};
cudaError_t launch_sweep(const hs_factors* f, const SweepLaunch& L, cudaStream_t s);
size_t sweep_smem_bytes(hs_dtype dt, int rhs_block, int tile_bits, int stage_diags, int n_stages);
int max_tile_bits(hs_dtype dt, int rhs_block, int stage_diags, size_t budget);
int max_rows_per_thread(hs_dtype dt, int rhs_block);
cudaError_t prepare_kernels();

cudaError_t launch_inner(const void* a, const void* b, int64_t N, hs_dtype dt, double* d_out4, cudaStream_t s);

// Stream-ordered allocation from the library's memory pool (api.cpp).
cudaError_t pool_malloc(void** ptr, size_t bytes, cudaStream_t s);

// Build the stored diagonals of a set built with HS_BUILD_DEFER_DIAGONALS, on
// stream s, if they are not built yet (api.cpp).
cudaError_t ensure_diagonals(const hs_factors* f, cudaStream_t s);

// Autotuner cache (tune.cpp).
bool tuned_opts(const hs_factors* f, int n_rhs, hs_evolve_opts* out);

}  // namespace hs
