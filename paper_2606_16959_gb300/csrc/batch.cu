// Batched evolution of many independent jobs of uneven size.
//
// Every job (its own factor set, states and step count) is planned into its
// sweep schedule exactly as hs_evolve_ex would plan it.  Launch k ("level k")
// then applies the k-th sweep of every job that has one: its grid is the union
// of those jobs' tiles, and each CTA finds its job by a binary search over the
// level's prefix table, rebuilds the sweep's arguments in shared memory from
// device tables, and runs the same tile code as the per-sweep kernel.  Levels
// are chained with programmatic dependent launch and the whole launch sequence
// is captured once into a CUDA graph, so a batch is one graph launch.  A job's
// schedule is eventually periodic, so only its distinct sweeps are stored.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "counters.h"
#include "hs_internal.h"
#include "qsweep.h"
#include "sweep_core.cuh"

namespace hs {
int report_error(int code, const std::string& msg);
}

namespace {

using hs::sweep::SweepArgs;

struct BJob {
  void* psi;
  const void* vals;
  const void* vt;
  const uint32_t* slot_u;
  const int32_t* slot_tab;
  const int64_t* tab_rb;
  int64_t N;
  int64_t n_vals, n_vt_g;  // extents (index checks only)
  int n_slot_g, n_tab_g;
  int n_qubits;
  int n_rhs;
};

struct BFac {
  int slot0, tab_g;
  int16_t nslot, mslot, tab_s, tab_n;
  int vt;          // first global value-table entry, -1: staged from the diagonals
  int16_t vts;     // first shared value-table entry (running prefix)
  int8_t sh;       // pattern shift of sm (see pattern_fast)
  uint32_t sm;     // the factor's value-table index mask
};

struct BSweep {
  int job;
  int fac_off, n_factors;
  int n_stages, stage_planes, n_mslot, n_mtab, n_vt;
  int all_tables;     // register path (see SweepArgs)
  uint64_t flane;
  uint32_t m0, m1;
  int sh;
  hs::Runs rest;
};

struct LevelArgs {
  const BJob* jobs;
  const BSweep* sweeps;
  const BFac* facs;
  const int* lvl_sweep;   // per entry of the level: distinct-sweep id
  const int* lvl_prefix;  // per entry: first CTA of the entry within the level
  int off, count;         // the level's entries
  int tile_bits;
  int tiles_per_cta;      // units (tile, state) one CTA runs back to back
};

constexpr int kBatchThreads = 512;  // at most; a tile of 2^T rows gets min(2^T, 512) threads
constexpr size_t kArgsBytes = (sizeof(SweepArgs) + 15) / 16 * 16;

template <typename R, int ROWS>
__global__ void __launch_bounds__(kBatchThreads) batch_level_kernel(const __grid_constant__ LevelArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  SweepArgs* sa = reinterpret_cast<SweepArgs*>(smem);
  int* pref = reinterpret_cast<int*>(smem + kArgsBytes);
  for (int i = threadIdx.x; i < p.count; i += blockDim.x) pref[i] = p.lvl_prefix[p.off + i];
  __syncthreads();
  // Entry of this CTA: the last one whose first CTA is <= blockIdx.x.
  int lo = 0, hi = p.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= int(blockIdx.x)) lo = mid; else hi = mid - 1;
  }
  const int local = int(blockIdx.x) - pref[lo];
  const BSweep& bs = p.sweeps[p.lvl_sweep[p.off + lo]];
  const BJob& bj = p.jobs[bs.job];
  if (threadIdx.x == 0) {
    sa->src = bj.psi;
    sa->dst = bj.psi;
    sa->vals = bj.vals;
    sa->vt = bj.vt;
    sa->slot_u = bj.slot_u;
    sa->slot_tab = bj.slot_tab;
    sa->tab_rb = bj.tab_rb;
    sa->N = bj.N;
    sa->n_vals = bj.n_vals;
    sa->n_vt_g = bj.n_vt_g;
    sa->n_slot_g = bj.n_slot_g;
    sa->n_tab_g = bj.n_tab_g;
    sa->n_rhs = bj.n_rhs;
    sa->rhs_block = 1;
    sa->tile_bits = p.tile_bits;
    sa->n_tiles_log2 = bj.n_qubits - p.tile_bits;
    sa->n_stages = bs.n_stages;
    sa->stage_planes = bs.stage_planes;
    sa->n_mslot = bs.n_mslot;
    sa->n_mtab = bs.n_mtab;
    sa->n_vt = bs.n_vt;
    sa->all_tables = bs.all_tables;
    sa->tiles_per_cta = 1;
    sa->n_units = 0;
    sa->flane = bs.flane;
    sa->m0 = bs.m0;
    sa->m1 = bs.m1;
    sa->sh = bs.sh;
    sa->rest = bs.rest;
    sa->n_factors = bs.n_factors;
  }
  for (int i = threadIdx.x; i < bs.n_factors; i += blockDim.x) {
    const BFac fe = p.facs[bs.fac_off + i];
    sa->fslot0[i] = fe.slot0;
    sa->ftab_g[i] = fe.tab_g;
    sa->fnslot[i] = fe.nslot;
    sa->fmslot[i] = fe.mslot;
    sa->ftab_s[i] = fe.tab_s;
    sa->ftab_n[i] = fe.tab_n;
    sa->fvt[i] = fe.vt;
    sa->fvts[i] = fe.vts;
    sa->fsm[i] = fe.sm;
    sa->fsh[i] = fe.sh;
  }
  __syncthreads();
  const uint32_t units = (1u << (bj.n_qubits - p.tile_bits)) * uint32_t(bj.n_rhs);
  const uint32_t u0 = uint32_t(local) * uint32_t(p.tiles_per_cta);
  const uint32_t u1 = min(units, u0 + uint32_t(p.tiles_per_cta));
  hs::sweep::sweep_tiles<R, ROWS, 1>(*sa, u0, u1, smem + kArgsBytes + size_t((p.count + 3) & ~3) * sizeof(int));
}

using LevelFn = void (*)(LevelArgs);

template <typename R>
LevelFn level_fn(int rows) {
  switch (rows) {
    case 1: return batch_level_kernel<R, 1>;
    case 2: return batch_level_kernel<R, 2>;
    case 4: return batch_level_kernel<R, 4>;
    case 8: return sizeof(R) == 4 ? batch_level_kernel<R, 8> : nullptr;
    default: return nullptr;
  }
}

}  // namespace

struct hs_batch {
  std::vector<const hs_factors*> diag_users;  // factor sets whose stored diagonals the batch reads
  uint64_t graph_kernels = 0;  // kernels one replay of the captured graph launches
  bool value_tables = true;    // read small-support factors from their value tables
  int tiles_per_cta = 1;       // units one CTA runs back to back (tables loaded once)
  hs_dtype dtype = HS_C64;
  int tile_bits = 0, low_bits = 0, rows = 1;
  bool use_graph = true;
  size_t smem = 0;
  struct Sep {
    const hs_factors* f;
    void* psi;
    int n_rhs, n_steps;
  };
  std::vector<Sep> separate;  // jobs evolved with their own launches
  struct Level {
    int off, count;
    int64_t ctas;
    bool full = false;  // register sweeps: some descriptor of the level needs the full kernel
  };
  std::vector<Level> levels;
  int max_count = 0;
  BJob* d_jobs = nullptr;
  BSweep* d_sweeps = nullptr;
  BFac* d_facs = nullptr;
  int* d_lvl_sweep = nullptr;
  int* d_lvl_prefix = nullptr;
  bool uploaded = false;
  // host copies of the device tables (uploaded on the first launch's stream)
  std::vector<BJob> hjobs;
  std::vector<BSweep> hsweeps;
  std::vector<BFac> hfacs;
  std::vector<int> hlvl_sweep, hlvl_prefix;
  cudaGraphExec_t graph = nullptr;
  int64_t updates = 0;
  int64_t ctas = 0;
  int64_t n_batched = 0;
  // Register-blocked batches: one descriptor per distinct sweep of every
  // batched job, and per tile size a sequence of levels over them.
  bool reg = false;
  int reg_bits = 0;
  struct QGroup {
    int tile_bits = 0;
    size_t smem = 0, prefix_smem = 0;
    std::vector<Level> levels;
    std::vector<int> lvl_desc, lvl_prefix;
    int* d_lvl_desc = nullptr;
    int* d_lvl_prefix = nullptr;
  };
  std::vector<hs::q::Args> qdescs;
  hs::q::Args* d_qdescs = nullptr;
  std::vector<QGroup> qgroups;
};

namespace {

void batch_release(hs_batch* b, cudaStream_t s) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  void* bufs[] = {b->d_jobs, b->d_sweeps, b->d_facs, b->d_lvl_sweep, b->d_lvl_prefix, b->d_qdescs};
  for (void* p : bufs)
    if (p) cudaFreeAsync(p, s);
  for (auto& g : b->qgroups) {
    if (g.d_lvl_desc) cudaFreeAsync(g.d_lvl_desc, s);
    if (g.d_lvl_prefix) cudaFreeAsync(g.d_lvl_prefix, s);
  }
  delete b;
}

template <typename T>
cudaError_t upload(T** dptr, const std::vector<T>& v, cudaStream_t s) {
  cudaError_t e = hs::pool_malloc(reinterpret_cast<void**>(dptr), std::max<size_t>(1, v.size()) * sizeof(T), s);
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpyAsync(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

// Upload the tables in stream order on s (once).
int upload_tables(hs_batch* b, cudaStream_t s) {
  if (b->uploaded) return HS_OK;
  cudaError_t e;
  if (b->reg) {
    e = upload(&b->d_qdescs, b->qdescs, s);
    for (auto& g : b->qgroups)
      if (e == cudaSuccess && (e = upload(&g.d_lvl_desc, g.lvl_desc, s)) == cudaSuccess)
        e = upload(&g.d_lvl_prefix, g.lvl_prefix, s);
    if (e != cudaSuccess)
      return hs::report_error(e == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA,
                              std::string("batch tables: ") + cudaGetErrorString(e));
    b->uploaded = true;
    return HS_OK;
  }
  if ((e = upload(&b->d_jobs, b->hjobs, s)) != cudaSuccess || (e = upload(&b->d_sweeps, b->hsweeps, s)) != cudaSuccess ||
      (e = upload(&b->d_facs, b->hfacs, s)) != cudaSuccess || (e = upload(&b->d_lvl_sweep, b->hlvl_sweep, s)) != cudaSuccess ||
      (e = upload(&b->d_lvl_prefix, b->hlvl_prefix, s)) != cudaSuccess)
    return hs::report_error(e == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA,
                            std::string("batch tables: ") + cudaGetErrorString(e));
  b->uploaded = true;
  return HS_OK;
}

int enqueue_batch(hs_batch* b, cudaStream_t s) {
  for (const hs_batch::Sep& j : b->separate) {
    hs_evolve_opts o{HS_METHOD_AUTO, 0, 0, 0, 0, 0, 0, 0};
    int rc = hs_evolve_ex(j.f, j.psi, j.n_rhs, j.n_steps, &o, s);
    if (rc != HS_OK) return rc;
  }
  if (b->reg) {
    for (const hs_batch::QGroup& g : b->qgroups)
      for (const hs_batch::Level& L : g.levels) {
        hs::q::LevelArgs a{b->d_qdescs, g.d_lvl_desc, g.d_lvl_prefix, L.off, L.count, uint32_t(g.prefix_smem)};
        cudaError_t e = hs::q::launch_qlevel(b->dtype, b->reg_bits, L.full, g.tile_bits, a, L.ctas, g.smem, s);
        if (e != cudaSuccess)
          return hs::report_error(HS_ECUDA, std::string("batch level launch: ") + cudaGetErrorString(e));
      }
    return HS_OK;
  }
  LevelFn fn = b->dtype == HS_C64 ? level_fn<float>(b->rows) : level_fn<double>(b->rows);
  if (!fn) return hs::report_error(HS_EINVAL, "internal: no batch kernel for this tile size");
  for (const hs_batch::Level& L : b->levels) {
    LevelArgs a{b->d_jobs, b->d_sweeps, b->d_facs, b->d_lvl_sweep, b->d_lvl_prefix, L.off, L.count, b->tile_bits,
                b->tiles_per_cta};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(L.ctas), 1u, 1u);
    cfg.blockDim = dim3(unsigned((1 << b->tile_bits) / b->rows), 1u, 1u);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, fn, a);
    if (e != cudaSuccess) return hs::report_error(HS_ECUDA, std::string("batch level launch: ") + cudaGetErrorString(e));
    hs::note_launches();
  }
  return HS_OK;
}

}  // namespace

namespace {

// Plan a batch of register-blocked sweeps: every job is scheduled as
// hs_evolve_ex's REG method schedules it (same sweeps, same ops, so results
// are bitwise those of evolving each job alone with the same options), with
// tiles of min(tile_bits, n) qubits; jobs are grouped by tile size, and level
// k of a group runs the k-th sweep of each of its jobs.
int create_reg_batch(const hs_batch_job* jobs, size_t n_jobs, const hs_batch_opts& o, hs_batch** out) {
  std::unique_ptr<hs_batch> b(new hs_batch());
  b->reg = true;
  b->dtype = jobs[0].factors ? jobs[0].factors->dtype : HS_C64;
  const hs_dtype dt = b->dtype;
  const bool c64 = dt == HS_C64;
  const int B = o.reg_bits > 0 ? o.reg_bits : (c64 ? 5 : 4);
  if (B != 4 && B != 5) return hs::report_error(HS_EINVAL, "reg_bits must be 0, 4 or 5");
  if (!c64 && B != 4) return hs::report_error(HS_EINVAL, "complex128 register sweeps use reg_bits 4");
  const int T = o.tile_bits > 0 ? o.tile_bits : (c64 ? 13 : 12);
  if (T < B + 5 || T > 13) return hs::report_error(HS_EINVAL, "register batches take tile_bits reg_bits + 5 .. 13");
  b->reg_bits = B;
  b->tile_bits = T;
  b->low_bits = o.low_bits > 0 ? o.low_bits : (c64 ? 2 : 1);
  b->use_graph = o.use_graph != 0;
  struct GJob { std::vector<int> descs; int64_t units; };
  std::map<int, std::vector<GJob>> by_tile;
  for (size_t j = 0; j < n_jobs; ++j) {
    const hs_batch_job& J = jobs[j];
    if (!J.factors || !J.psi) return hs::report_error(HS_EINVAL, "job " + std::to_string(j) + ": null factors or psi");
    if (J.factors->dtype != dt) return hs::report_error(HS_EDTYPE, "jobs differ in dtype");
    if (J.n_rhs < 1 || J.n_steps < 0) return hs::report_error(HS_EINVAL, "job " + std::to_string(j) + ": bad n_rhs/n_steps");
    if (reinterpret_cast<uintptr_t>(J.psi) % 16) return hs::report_error(HS_EINVAL, "psi must be 16-byte aligned");
  }
  // Per job (independent, planned on host threads): its sweeps as descriptor
  // pieces (a sweep seen before reuses its pieces), the order in which its
  // levels use them, or "separate" when some sweep has no register form.
  struct JobPlan {
    bool ok = false;
    int Tj = 0;
    std::vector<std::shared_ptr<hs::q::Args>> pieces;
    std::vector<int> order;  // indices into pieces, one per level
  };
  std::vector<JobPlan> plans(n_jobs);
  const int lb = b->low_bits;
  auto plan_job = [&](size_t j) {
    const hs_batch_job& J = jobs[j];
    JobPlan& P = plans[j];
    const hs::Plan& p = J.factors->plan;
    if (J.n_steps == 0) return;
    const int n = p.n_qubits;
    P.Tj = std::min(T, n);
    bool ok = n >= B + 5;
    std::vector<hs::Sweep> sw;
    if (ok) sw = hs::plan_sweeps_commuting(p, J.n_steps, P.Tj, lb);
    for (const hs::Sweep& w : sw) ok = ok && w.fused;
    std::map<std::pair<uint32_t, std::vector<int>>, std::vector<int>> memo;  // sweep -> its pieces
    for (size_t k = 0; ok && k < sw.size(); ++k) {
      const auto key = std::make_pair(sw[k].local_mask, sw[k].factors);
      auto it = memo.find(key);
      if (it != memo.end()) {
        P.order.insert(P.order.end(), it->second.begin(), it->second.end());
        continue;
      }
      std::vector<std::pair<std::vector<int>, std::shared_ptr<hs::q::Args>>> pieces;
      std::string why;
      if (!hs::q::plan_qsweep_runs(J.factors, sw[k].factors, sw[k].local_mask, P.Tj, B, pieces, &why)) {
        ok = false;
        break;
      }
      std::vector<int> ids;
      for (auto& pc : pieces) {
        hs::q::fill_job(J.factors, *pc.second, J.psi, J.n_rhs);
        pc.second->units_per_cta = 1;
        ids.push_back(int(P.pieces.size()));
        P.pieces.push_back(std::move(pc.second));
      }
      P.order.insert(P.order.end(), ids.begin(), ids.end());
      memo[key] = std::move(ids);
    }
    P.ok = ok;
  };
  {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t n_thr = std::min<size_t>(std::min<size_t>(hw, 16), (n_jobs + 7) / 8);
    std::atomic<size_t> next{0};
    auto worker = [&]() {
      for (size_t j; (j = next.fetch_add(1)) < n_jobs;) plan_job(j);
    };
    std::vector<std::thread> pool;
    for (size_t t = 1; t < n_thr; ++t) pool.emplace_back(worker);
    worker();
    for (std::thread& t : pool) t.join();
  }
  for (size_t j = 0; j < n_jobs; ++j) {
    const hs_batch_job& J = jobs[j];
    const hs::Plan& p = J.factors->plan;
    b->updates += int64_t(J.n_steps) * int64_t(p.step_seq.size()) * p.N * J.n_rhs;
    if (J.n_steps == 0) continue;
    JobPlan& P = plans[j];
    if (!P.ok) {
      b->separate.push_back(hs_batch::Sep{J.factors, J.psi, J.n_rhs, J.n_steps});
      b->diag_users.push_back(J.factors);  // its own (plain or staged) evolution reads the diagonals
      continue;
    }
    const int first = int(b->qdescs.size());
    for (auto& a : P.pieces) b->qdescs.push_back(*a);
    GJob gj;
    gj.descs.reserve(P.order.size());
    for (int i : P.order) gj.descs.push_back(first + i);
    gj.units = (int64_t(1) << (p.n_qubits - P.Tj)) * J.n_rhs;
    by_tile[P.Tj].push_back(std::move(gj));
    ++b->n_batched;
  }
  for (auto& kv : by_tile) {
    hs_batch::QGroup g;
    g.tile_bits = kv.first;
    size_t smem = 0, max_levels = 0;
    for (const GJob& gj : kv.second) {
      max_levels = std::max(max_levels, gj.descs.size());
      for (int d : gj.descs) smem = std::max(smem, hs::q::qsweep_smem_bytes(b->qdescs[d], dt, B));
    }
    int max_count = 0;
    for (size_t k = 0; k < max_levels; ++k) {
      hs_batch::Level L{int(g.lvl_desc.size()), 0, 0};
      for (const GJob& gj : kv.second) {
        if (k >= gj.descs.size()) continue;
        g.lvl_desc.push_back(gj.descs[k]);
        g.lvl_prefix.push_back(int(L.ctas));
        L.full = L.full || b->qdescs[gj.descs[k]].full != 0;
        L.ctas += gj.units;
        ++L.count;
      }
      if (L.ctas >= (int64_t(1) << 31)) return hs::report_error(HS_EINVAL, "batch level exceeds 2^31 CTAs");
      max_count = std::max(max_count, L.count);
      b->ctas += L.ctas;
      g.levels.push_back(L);
    }
    g.prefix_smem = (smem + 15) / 16 * 16;
    g.smem = g.prefix_smem + size_t(max_count) * sizeof(int);
    if (g.smem > hs::kSweepSmemMax) return hs::report_error(HS_EINVAL, "batch needs more shared memory than a CTA has");
    b->levels.insert(b->levels.end(), g.levels.begin(), g.levels.end());  // for hs_batch_info
    b->qgroups.push_back(std::move(g));
  }
  *out = b.release();
  return HS_OK;
}

}  // namespace

extern "C" int hs_batch_create(const hs_batch_job* jobs, size_t n_jobs, const hs_batch_opts* opts, hs_batch** out) {
  if (!out) return hs::report_error(HS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!jobs || n_jobs == 0) return hs::report_error(HS_EINVAL, "no jobs");
  hs_batch_opts o{0, 0, 1, 0, 0, 0, 0, 0};
  if (opts) o = *opts;
  if (o.method == HS_METHOD_REG) return create_reg_batch(jobs, n_jobs, o, out);
  std::unique_ptr<hs_batch> b(new hs_batch());
  b->dtype = jobs[0].factors ? jobs[0].factors->dtype : HS_C64;
  int min_n = 64;
  for (size_t j = 0; j < n_jobs; ++j) {
    const hs_batch_job& J = jobs[j];
    if (!J.factors || !J.psi) return hs::report_error(HS_EINVAL, "job " + std::to_string(j) + ": null factors or psi");
    if (J.factors->dtype != b->dtype) return hs::report_error(HS_EDTYPE, "jobs differ in dtype");
    if (J.n_rhs < 1 || J.n_steps < 0) return hs::report_error(HS_EINVAL, "job " + std::to_string(j) + ": bad n_rhs/n_steps");
    if (reinterpret_cast<uintptr_t>(J.psi) % 16) return hs::report_error(HS_EINVAL, "psi must be 16-byte aligned");
    min_n = std::min(min_n, J.factors->plan.n_qubits);
  }
  const hs_dtype dt = b->dtype;
  // Defaults measured on the 256-instance TFIM/Heisenberg batch (complex64,
  // value tables and the register path on): tiles of 2^10 rows with 24 KiB per
  // CTA ran it in 561 ms, against 576 ms with 40 KiB, 584 ms with 64 KiB,
  // 652 ms for 2^11 rows and 747 ms for 2^9.
  b->tile_bits = o.tile_bits > 0 ? o.tile_bits : 10;
  b->low_bits = o.low_bits > 0 ? o.low_bits : (dt == HS_C64 ? 2 : 1);
  b->use_graph = o.use_graph != 0;
  b->value_tables = o.no_tables == 0;
  if (o.tiles_per_cta < 0 || o.tiles_per_cta > 64) return hs::report_error(HS_EINVAL, "tiles_per_cta must be 0..64");
  // 8 measured best on the 256-instance batch (458 ms against 574 ms for 1).
  b->tiles_per_cta = o.tiles_per_cta > 0 ? o.tiles_per_cta : 8;
  if (b->tile_bits < 8 || b->tile_bits > 11) return hs::report_error(HS_EINVAL, "batch tile_bits must be 8..11");
  b->rows = (1 << b->tile_bits) > kBatchThreads ? (1 << b->tile_bits) / kBatchThreads : 1;
  if ((dt == HS_C64 ? level_fn<float>(b->rows) : level_fn<double>(b->rows)) == nullptr)
    return hs::report_error(HS_EINVAL, "batch tile_bits too large for complex128");
  const int T = b->tile_bits;
  if (o.smem_kb < 0 || size_t(o.smem_kb) * 1024 > hs::kSweepSmemMax)
    return hs::report_error(HS_EINVAL, "batch smem_kb must be 0..227");
  const size_t budget = size_t(o.smem_kb > 0 ? o.smem_kb : 24) * 1024;

  std::vector<BJob> hjobs;
  std::vector<BSweep> hsweeps;
  std::vector<BFac> hfacs;
  std::vector<std::vector<int>> job_levels;  // per batched job: distinct-sweep id of each level
  std::vector<int64_t> job_ctas;
  size_t need_smem = 0;
  for (size_t j = 0; j < n_jobs; ++j) {
    const hs_batch_job& J = jobs[j];
    const hs::Plan& p = J.factors->plan;
    b->updates += int64_t(J.n_steps) * int64_t(p.step_seq.size()) * p.N * J.n_rhs;
    if (J.n_steps == 0) continue;
    std::vector<hs::Sweep> sw = p.n_qubits >= T ? hs::plan_sweeps(p, J.n_steps, T, b->low_bits, true)
                                                : std::vector<hs::Sweep>{};
    bool ok = !sw.empty();
    for (const hs::Sweep& w : sw) ok = ok && w.fused;
    b->diag_users.push_back(J.factors);  // staged sweeps and separate evolutions read the diagonals
    if (!ok) {
      b->separate.push_back(hs_batch::Sep{J.factors, J.psi, J.n_rhs, J.n_steps});
      continue;
    }
    const int jid = int(hjobs.size());
    const hs_factors* f = J.factors;
    hjobs.push_back(BJob{J.psi, f->d_vals, f->d_vt, f->d_slot_u, f->d_slot_tab, f->d_tab_rb, p.N, p.total_elems,
                         p.total_vt, int(p.slot_u.size()), int(p.tab_rb.size()), p.n_qubits, J.n_rhs});
    const int64_t units = (int64_t(1) << (p.n_qubits - T)) * J.n_rhs;
    job_ctas.push_back((units + b->tiles_per_cta - 1) / b->tiles_per_cta);
    std::map<std::pair<uint32_t, std::vector<int>>, int> uniq;
    std::vector<int> lv;
    const uint64_t all = (1ull << p.n_qubits) - 1;
    for (const hs::Sweep& w : sw) {
      auto key = std::make_pair(w.local_mask, w.factors);
      auto it = uniq.find(key);
      if (it != uniq.end()) { lv.push_back(it->second); continue; }
      BSweep bs{};
      bs.job = jid;
      bs.fac_off = int(hfacs.size());
      bs.n_factors = int(w.factors.size());
      const uint32_t lm = w.local_mask;
      int lo = 0;
      while (lo < 32 && ((lm >> lo) & 1u)) ++lo;
      const uint32_t hi = lm & ~((1u << lo) - 1u);
      const int wd = __builtin_popcount(hi);
      const int h = hi ? __builtin_ctz(hi) : lo;
      bs.m0 = (1u << lo) - 1u;
      bs.m1 = ((1u << wd) - 1u) << lo;
      bs.sh = h - lo;
      bs.rest = hs::runs_of(~uint64_t(lm) & all, p.n_qubits);
      int planes = 1, n_mslot = 0, n_mtab = 0, n_vt = 0;
      for (int g : w.factors) {
        const hs::Group& G = p.groups[g];
        const int t0 = p.slot_tab[G.slot0], t1 = p.slot_tab[G.slot0 + G.nslot];
        const bool table = b->value_tables && G.vt0 >= 0 && n_vt + G.vt_n <= hs::kMaxVtSweep;
        hfacs.push_back(BFac{G.slot0, t0, int16_t(G.nslot), int16_t(n_mslot), int16_t(n_mtab), int16_t(t1 - t0),
                             table ? G.vt0 : -1, int16_t(n_vt),
                             hs::sweep::pattern_shift(table ? G.smask : 0u), table ? G.smask : 0u});
        n_mslot += G.nslot;
        n_mtab += t1 - t0;
        if (table) n_vt += G.vt_n;
        else planes = std::max(planes, G.nslot);
      }
      bs.n_mslot = n_mslot;
      bs.n_mtab = n_mtab;
      bs.n_vt = n_vt;
      bs.stage_planes = planes;
      bs.all_tables = 0;
      bs.flane = 0;
      {
        const uint32_t thr_mask = uint32_t((1 << T) / b->rows - 1);
        bool all = n_vt > 0;
        for (size_t i = 0; i < w.factors.size(); ++i) {
          const hs::Group& G = p.groups[w.factors[i]];
          if (hfacs[bs.fac_off + i].vt < 0) all = false;
          bool lane = true;
          for (int sl = 0; sl < G.nslot; ++sl) {
            const uint32_t u = p.slot_u[G.slot0 + sl];
            if ((((u & bs.m0) | ((u >> bs.sh) & bs.m1)) & thr_mask) >= 32u) lane = false;
          }
          if (lane) bs.flane |= 1ull << i;
        }
        bs.all_tables = all ? 1 : 0;
      }
      const size_t mb = hs::sweep::meta_bytes(n_mslot, n_mtab, n_vt, hs::elem_bytes(dt));
      int S = 1;
      while (S < 8 && S < bs.n_factors && mb + hs::sweep_smem_bytes(dt, 1, T, planes, S + 1) <= budget) ++S;
      bs.n_stages = S;
      need_smem = std::max(need_smem, mb + hs::sweep_smem_bytes(dt, 1, T, planes, S));
      const int id = int(hsweeps.size());
      hsweeps.push_back(bs);
      uniq[key] = id;
      lv.push_back(id);
    }
    job_levels.push_back(std::move(lv));
  }
  // Level tables.
  std::vector<int> lvl_sweep, lvl_prefix;
  size_t max_levels = 0;
  for (const auto& lv : job_levels) max_levels = std::max(max_levels, lv.size());
  for (size_t k = 0; k < max_levels; ++k) {
    hs_batch::Level L{int(lvl_sweep.size()), 0, 0};
    for (size_t j = 0; j < job_levels.size(); ++j) {
      if (k >= job_levels[j].size()) continue;
      lvl_sweep.push_back(job_levels[j][k]);
      lvl_prefix.push_back(int(L.ctas));
      L.ctas += job_ctas[j];
      ++L.count;
    }
    if (L.ctas >= (int64_t(1) << 31)) return hs::report_error(HS_EINVAL, "batch level exceeds 2^31 CTAs");
    b->max_count = std::max(b->max_count, L.count);
    b->ctas += L.ctas;
    b->levels.push_back(L);
  }
  b->n_batched = int64_t(hjobs.size());
  b->smem = kArgsBytes + size_t((b->max_count + 3) & ~3) * sizeof(int) + need_smem;
  if (b->smem > hs::kSweepSmemMax) return hs::report_error(HS_EINVAL, "batch needs more shared memory than a CTA has");
  b->hjobs = std::move(hjobs);
  b->hsweeps = std::move(hsweeps);
  b->hfacs = std::move(hfacs);
  b->hlvl_sweep = std::move(lvl_sweep);
  b->hlvl_prefix = std::move(lvl_prefix);
  *out = b.release();
  return HS_OK;
}

extern "C" int hs_batch_launch(hs_batch* b, void* cuda_stream) {
  if (!b) return hs::report_error(HS_EINVAL, "batch is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = hs::prepare_kernels();
  if (e != cudaSuccess) return hs::report_error(HS_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
  if (b->reg) {
    e = hs::q::prepare_qsweep();
    if (e != cudaSuccess) return hs::report_error(HS_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
  }
  static std::mutex attr_mu;
  static bool attr_done[2][9] = {};
  if (!b->reg) {
    std::lock_guard<std::mutex> lk(attr_mu);
    bool& done = attr_done[b->dtype == HS_C64 ? 0 : 1][b->rows];
    if (!done) {
      LevelFn fn = b->dtype == HS_C64 ? level_fn<float>(b->rows) : level_fn<double>(b->rows);
      e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(hs::kSweepSmemMax));
      if (e != cudaSuccess) return hs::report_error(HS_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
      done = true;
    }
  }
  // Sets built with deferred diagonals: build them before any launch (and
  // outside a capture) for the jobs that read them.
  for (const hs_factors* f : b->diag_users) {
    e = hs::ensure_diagonals(f, s);
    if (e != cudaSuccess) return hs::report_error(HS_ECUDA, std::string("factor build: ") + cudaGetErrorString(e));
  }
  if (!b->uploaded) {
    int rc = upload_tables(b, s);
    if (rc != HS_OK) return rc;
    // A captured graph may later be launched on another stream.
    if (b->use_graph && cudaStreamSynchronize(s) != cudaSuccess) return hs::report_error(HS_ECUDA, "table upload");
  }
  if (!b->use_graph) return enqueue_batch(b, s);
  if (!b->graph) {
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return hs::report_error(HS_ECUDA, "cudaStreamCreate");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); return hs::report_error(HS_ECUDA, "cudaStreamBeginCapture"); }
    hs::begin_capture_count();
    int rc = enqueue_batch(b, cs);
    b->graph_kernels = hs::end_capture_count();
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc != HS_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return hs::report_error(HS_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return hs::report_error(HS_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  e = cudaGraphLaunch(b->graph, s);
  if (e == cudaSuccess) hs::note_launches(b->graph_kernels);
  return e == cudaSuccess ? HS_OK : hs::report_error(HS_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
}

extern "C" int hs_batch_info(const hs_batch* b, int* n_levels, int64_t* n_ctas, int64_t* n_updates, int* n_separate) {
  if (!b) return hs::report_error(HS_EINVAL, "batch is NULL");
  if (n_levels) *n_levels = int(b->levels.size());
  if (n_ctas) *n_ctas = b->ctas;
  if (n_updates) *n_updates = b->updates;
  if (n_separate) *n_separate = int(b->separate.size());
  return HS_OK;
}

extern "C" void hs_batch_free(hs_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_release(b, nullptr);
  cudaDeviceSynchronize();
}

extern "C" int hs_batch_free_async(hs_batch* b, void* cuda_stream) {
  if (b) batch_release(b, reinterpret_cast<cudaStream_t>(cuda_stream));
  return HS_OK;
}

extern "C" int hs_evolve_batch(const hs_factors* const* f, void* const* psi, const int* n_rhs, const int* n_steps,
                               size_t n_jobs, void* cuda_stream) {
  if (!f || !psi || !n_rhs || !n_steps || n_jobs == 0) return hs::report_error(HS_EINVAL, "null job arrays or no jobs");
  std::vector<hs_batch_job> jobs(n_jobs);
  for (size_t k = 0; k < n_jobs; ++k) jobs[k] = hs_batch_job{f[k], psi[k], n_rhs[k], n_steps[k]};
  hs_batch_opts o{0, 0, 0, 0, 0, 0, HS_METHOD_REG, 0};  // register-blocked sweeps, other options the library's
  hs_batch* b = nullptr;
  int rc = hs_batch_create(jobs.data(), n_jobs, &o, &b);
  if (rc != HS_OK) return rc;
  rc = hs_batch_launch(b, cuda_stream);
  hs_batch_free_async(b, cuda_stream);
  return rc;
}
