// C ABI of libhs (declared in include/hs.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <list>
#include <map>
#include <unordered_map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "counters.h"
#include "hs_internal.h"
#include "qsweep.h"

namespace hs {
size_t inner_scratch_bytes();
cudaError_t launch_inner_scratch(const void* a, const void* b, int64_t N, hs_dtype dt, double* d_out4, void* scratch,
                                 cudaStream_t s);
}  // namespace hs

namespace {

thread_local std::string g_err;

// Kernels per instantiated evolution graph (added to the launch count on replay).
std::mutex g_graph_mu;
std::map<cudaGraphExec_t, uint64_t> g_graph_kernels;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA,
              std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

bool valid_dtype(hs_dtype d) { return d == HS_C64 || d == HS_C128; }

// Default number of contiguous low bits in a tile: every access along a
// diagonal or the state then covers whole 32-byte sectors.
int min_low_bits(hs_dtype dt) { return dt == HS_C64 ? 2 : 1; }

// Free a factor set's device memory in stream order on s (stream-ordered
// allocations) and delete the object.
void release(hs_factors* f, cudaStream_t s) {
  if (!f) return;
  {
    std::lock_guard<std::mutex> lk(f->graph_mu);
    for (auto& kv : f->graphs) cudaGraphExecDestroy(kv.second);
    f->graphs.clear();
  }
  if (f->d_vals) cudaFreeAsync(f->d_vals, s);
  if (f->d_tables) cudaFreeAsync(f->d_tables, s);
  if (f->d_drive) cudaFreeAsync(f->d_drive, s);
  if (f->d_steprec) cudaFreeAsync(f->d_steprec, s);
  delete f;
}

// Register-blocked launches of a schedule: one descriptor per fused sweep
// (shared by the sweeps that repeat), or null where the sweep is launched
// otherwise.
using QPlans = std::vector<std::shared_ptr<hs::q::Args>>;

// Enqueue the launches of one evolution on stream s.
// StepRecords: per-step term records of a time-dependent set (register sweeps
// that span steps address them from their first step).
struct StepRecords {
  const double* rq = nullptr;  // 4 doubles per record
  const double* cs = nullptr;  // 2 doubles per record
  int stride = 0;              // records per step
  int n_steps = 0;
};

int enqueue_evolve(const hs_factors* f, const std::vector<hs::Sweep>& sw, void* psi, int n_rhs, int tile_bits,
                   int rhs_block, size_t smem_budget, bool value_tables, void* scratch, cudaStream_t s,
                   const QPlans* qp = nullptr, int reg_bits = 0, const StepRecords* rec = nullptr) {
  const hs::Plan& p = f->plan;
  void* cur = psi;
  void* other = scratch;
  const uint64_t all = (1ull << p.n_qubits) - 1;
  for (size_t wi = 0; wi < sw.size(); ++wi) {
    const hs::Sweep& w = sw[wi];
    cudaError_t e;
    if (qp && (*qp)[wi] && rec) {
      const int st = w.steps.empty() ? 0 : w.steps[0];
      e = hs::q::launch_qsweep(f, *(*qp)[wi], cur, cur, n_rhs, reg_bits, true, s, rec->rq + size_t(4) * st * rec->stride,
                               rec->cs + size_t(2) * st * rec->stride, (rec->n_steps - st) * rec->stride);
    } else if (qp && (*qp)[wi]) {
      e = hs::q::launch_qsweep(f, *(*qp)[wi], cur, cur, n_rhs, reg_bits, true, s);
    } else if (w.fused) {
      hs::SweepLaunch L;
      L.src = cur;
      L.dst = cur;
      L.n_rhs = n_rhs;
      L.rhs_block = rhs_block;
      L.tile_bits = std::min(tile_bits, p.n_qubits);
      L.local_mask = w.local_mask;
      L.rest = hs::runs_of(~uint64_t(w.local_mask) & all, p.n_qubits);
      L.n_factors = int(w.factors.size());
      for (int i = 0; i < L.n_factors; ++i) L.factors[i] = w.factors[i];
      L.smem_budget = smem_budget;
      L.pdl = true;
      L.value_tables = value_tables;
      e = hs::launch_sweep(f, L, s);
    } else {
      if (!other) return fail(HS_EINVAL, "internal: plain application without scratch");
      e = hs::launch_apply_plain(f, w.factors[0], cur, other, n_rhs, s);
      std::swap(cur, other);
    }
    if (e != cudaSuccess) return cuda_fail(e, "launch");
  }
  if (cur != psi) {
    cudaError_t e = cudaMemcpyAsync(psi, cur, size_t(n_rhs) * size_t(p.N) * hs::elem_bytes(f->dtype),
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  }
  return HS_OK;
}

// The launch schedule of n_steps steps: register sweeps may take commuting
// factor applications out of order (hs::plan_sweeps_commuting); the other
// methods apply the factors in the formula's order.
std::vector<hs::Sweep> schedule(const hs_factors* f, int n_steps, const hs_evolve_opts& o, int tb) {
  if (o.method == HS_METHOD_REG)
    return hs::plan_sweeps_commuting(f->plan, n_steps, tb, o.low_bits, hs::kMaxFusedDiags, o.max_fuse);
  return hs::plan_sweeps(f->plan, n_steps, tb, o.low_bits, o.method != HS_METHOD_PLAIN, hs::kMaxFusedDiags,
                         o.max_fuse);
}

bool has_plain(const std::vector<hs::Sweep>& sw) {
  for (const hs::Sweep& w : sw)
    if (!w.fused) return true;
  return false;
}

// Register-blocked descriptors for the fused sweeps of sw (method REG): each
// distinct sweep is planned once; a sweep that cannot be expressed as register
// ops is replaced by plain launches of its factors.
// step_stride > 0: the sweeps span steps of a time-dependent set whose term
// records are kept per step (step_stride records each); a planned sweep's
// steps become one entry, the step its records start at.
void plan_reg(const hs_factors* f, std::vector<hs::Sweep>& sw, int tile_bits, int reg_bits, QPlans& qp,
              int step_stride = 0) {
  using Pieces = std::vector<std::pair<std::vector<int>, std::shared_ptr<hs::q::Args>>>;
  std::map<std::tuple<uint32_t, std::vector<int>, std::vector<int>>, std::pair<bool, Pieces>> memo;
  std::vector<hs::Sweep> out;
  QPlans plans;
  for (hs::Sweep& w : sw) {
    if (!w.fused) {
      out.push_back(std::move(w));
      plans.push_back(nullptr);
      continue;
    }
    std::vector<int> rel;
    if (step_stride > 0)
      for (int st : w.steps) rel.push_back(st - w.steps[0]);
    const auto key = std::make_tuple(w.local_mask, w.factors, rel);
    auto it = memo.find(key);
    if (it == memo.end()) {
      Pieces pieces;
      std::string why;
      const bool ok = hs::q::plan_qsweep_runs(f, w.factors, w.local_mask, tile_bits, reg_bits, pieces, &why,
                                               step_stride > 0 ? &rel : nullptr, step_stride);
      it = memo.emplace(key, std::make_pair(ok, std::move(pieces))).first;
    }
    if (it->second.first) {
      size_t pos = 0;
      for (const auto& pc : it->second.second) {
        hs::Sweep s2;
        s2.fused = true;
        s2.local_mask = w.local_mask;
        s2.factors = pc.first;
        s2.steps.assign(1, pos < w.steps.size() ? w.steps[pos] : 0);
        pos += pc.first.size();
        out.push_back(std::move(s2));
        plans.push_back(pc.second);
      }
    } else {
      for (size_t i = 0; i < w.factors.size(); ++i) {
        hs::Sweep pl;
        pl.fused = false;
        pl.factors.push_back(w.factors[i]);
        if (i < w.steps.size()) pl.steps.push_back(w.steps[i]);
        out.push_back(std::move(pl));
        plans.push_back(nullptr);
      }
    }
  }
  sw = std::move(out);
  qp = std::move(plans);
}

// Largest number of staged planes (slots) among the factors a sweep may hold.
int fused_dmax(const hs_factors* f) {
  int d = 1;
  for (const hs::Group& g : f->plan.groups)
    if (g.nslot > d) d = g.nslot;
  return d;
}

int pick_rhs_block(hs_dtype dt, int n_rhs) {
  int rb = 1;
  const int cap = dt == HS_C64 ? 16 : 8;
  while (rb * 2 <= n_rhs && rb * 2 <= cap) rb *= 2;
  return rb;
}

int pick_tile_bits(const hs_factors* f, int rhs_block) {
  const int n = f->plan.n_qubits;
  int t = hs::max_tile_bits(f->dtype, rhs_block, fused_dmax(f), hs::kSweepSmemDefault);
  // keep at least ~128 tiles when the state allows it
  int cap = n - 7;
  if (cap < min_low_bits(f->dtype) + 4) cap = min_low_bits(f->dtype) + 4;
  if (t > cap) t = cap;
  if (t > n) t = n;
  return t;
}

// Plans depend only on the flip masks, the qubit count, the budget and the
// dtype (not on coefficients or the time step), so rebuilding a factor set for
// the same structure reuses the planned grouping, layout and slot tables.
struct PlanCache {
  std::mutex mu;
  std::list<std::string> lru;
  std::unordered_map<std::string, std::pair<hs::Plan, std::list<std::string>::iterator>> map;
  static constexpr size_t kCap = 64;
};
PlanCache& plan_cache() {
  static PlanCache c;
  return c;
}
// The z masks are part of the key: a factor's value table is indexed by the
// qubits its terms touch through x or z.
std::string plan_key(const uint64_t* x, const uint64_t* z, size_t n, int n_qubits, int budget, hs_dtype dt,
                     int order) {
  std::string k(reinterpret_cast<const char*>(x), n * sizeof(uint64_t));
  k.append(reinterpret_cast<const char*>(z), n * sizeof(uint64_t));
  k.append(reinterpret_cast<const char*>(&order), sizeof(int));
  k.append(reinterpret_cast<const char*>(&n_qubits), sizeof(int));
  k.append(reinterpret_cast<const char*>(&budget), sizeof(int));
  const int d = int(dt);
  k.append(reinterpret_cast<const char*>(&d), sizeof(int));
  return k;
}
int cached_plan(const uint64_t* x, const uint64_t* z, const double* coeff, size_t n, int n_qubits, int budget,
                hs_dtype dt, int order, hs::Plan& plan, std::string* err) {
  const std::string key = plan_key(x, z, n, n_qubits, budget, dt, order);
  PlanCache& c = plan_cache();
  {
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.map.find(key);
    if (it != c.map.end()) {
      c.lru.splice(c.lru.begin(), c.lru, it->second.second);
      plan = it->second.first;
    } else {
      plan = hs::Plan();
    }
  }
  if (plan.n_qubits == 0) {
    int rc = hs::make_plan(x, z, coeff, n, n_qubits, budget, dt, plan, err, order);
    if (rc != HS_OK) return rc;
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.map.find(key) == c.map.end()) {
      c.lru.push_front(key);
      c.map.emplace(key, std::make_pair(plan, c.lru.begin()));
      if (c.lru.size() > PlanCache::kCap) {
        c.map.erase(c.lru.back());
        c.lru.pop_back();
      }
    }
    return HS_OK;
  }
  // Same structure: take this call's phase masks and coefficients.
  for (size_t j = 0; j < n; ++j) {
    if (coeff && !std::isfinite(coeff[j])) { *err = "non-finite coefficient at term " + std::to_string(j); return HS_EINVAL; }
    if (z[j] >= (1ull << n_qubits)) { *err = "mask of term " + std::to_string(j) + " exceeds n_qubits"; return HS_EINVAL; }
  }
  plan.z.assign(z, z + n);
  plan.coeff.assign(coeff, coeff + n);
  return HS_OK;
}

}  // namespace

namespace hs {
std::atomic<uint64_t> g_launches{0};
namespace {
thread_local bool t_capturing = false;
thread_local uint64_t t_captured = 0;
}  // namespace

void note_launches(uint64_t n) {
  if (t_capturing) t_captured += n;
  else g_launches.fetch_add(n, std::memory_order_relaxed);
}
void begin_capture_count() {
  t_capturing = true;
  t_captured = 0;
}
uint64_t end_capture_count() {
  t_capturing = false;
  return t_captured;
}

// Readers of the translation units' bounds words (HS_DEBUG_BOUNDS build).
using BoundsReader = int (*)(uint64_t* out4, bool reset);
static std::vector<BoundsReader>& bounds_readers() {
  static std::vector<BoundsReader> r;
  return r;
}
void register_bounds_reader(BoundsReader r) { bounds_readers().push_back(r); }

// The library's stream-ordered memory pool on the current device: memory freed
// by hs_free_factors_async / hs_batch_free_async stays in the pool (release
// threshold unlimited) so that the next factor build reuses it without mapping
// new memory.  Falls back to the device's default pool if creation fails.
cudaMemPool_t library_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      if (cudaDeviceGetDefaultMemPool(&p, dev) != cudaSuccess) return nullptr;
    }
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    pools[dev] = p;
  }
  return pools[dev];
}

cudaError_t ensure_diagonals(const hs_factors* f, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(f->diag_mu);
  if (!f->diag_pending) return cudaSuccess;
  const hs_build_inputs& b = f->bin;
  const cudaError_t e = launch_build_split(f, b.tab_groups, b.n_tab_groups, b.row_groups, b.n_row_groups, s);
  if (e == cudaSuccess) f->diag_pending = false;
  return e;
}

cudaError_t pool_malloc(void** ptr, size_t bytes, cudaStream_t s) {
  cudaMemPool_t p = library_pool();
  if (!p) return cudaMallocAsync(ptr, bytes, s);
  return cudaMallocFromPoolAsync(ptr, bytes, p, s);
}
}  // namespace hs

namespace {

// Pinned host staging for table uploads: a small ring of buffers, each reused
// only after the copy that last read it has completed.
struct Staging {
  void* buf = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
};
int stage_upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static Staging ring[8];
  static int next = 0;
  std::lock_guard<std::mutex> lk(mu);
  Staging& st = ring[next];
  next = (next + 1) % 8;
  if (st.ev) cudaEventSynchronize(st.ev);
  if (st.cap < bytes) {
    if (st.buf) cudaFreeHost(st.buf);
    st.buf = nullptr;
    st.cap = 0;
    size_t cap = std::max<size_t>(bytes, 64 << 10);
    if (cudaHostAlloc(&st.buf, cap, cudaHostAllocDefault) != cudaSuccess) {
      st.buf = nullptr;
      cudaGetLastError();
      return int(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));  // pageable fallback
    }
    st.cap = cap;
  }
  if (!st.ev && cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming) != cudaSuccess) {
    st.ev = nullptr;
    return int(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
  }
  std::memcpy(st.buf, src, bytes);
  cudaError_t e = cudaMemcpyAsync(dst, st.buf, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(st.ev, s);
  return int(e);
}

}  // namespace

namespace hs {
int report_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace hs

bool hs_factors::GraphKey::operator<(const GraphKey& o) const {
  return std::tie(psi, n_rhs, n_steps, method, tile_bits, rhs_block, stream, variant) <
         std::tie(o.psi, o.n_rhs, o.n_steps, o.method, o.tile_bits, o.rhs_block, o.stream, o.variant);
}

namespace {

// Build a factor set; coeffs1 non-NULL makes it time-dependent (H0 + f(t) H1,
// values built for f = 0).
int build_impl(const uint64_t* x, const uint64_t* z, const double* coeffs, const double* coeffs1, size_t n_terms,
               int n_qubits, double t, int n_steps, int diag_budget, int order, hs_dtype dtype, void* cuda_stream,
               hs_factors** out, int flags = 0) {
  if (!out) return fail(HS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!x || !z || !coeffs) return fail(HS_EINVAL, "null term arrays");
  if (!valid_dtype(dtype)) return fail(HS_EDTYPE, "dtype must be HS_C64 or HS_C128");
  if (!(std::isfinite(t) && t > 0)) return fail(HS_EINVAL, "t must be finite and > 0");
  if (n_steps < 1) return fail(HS_EINVAL, "n_steps must be >= 1");
  if (diag_budget < 1) return fail(HS_EINVAL, "diag_budget must be >= 1");
  if (order != 1 && order != 2 && order != 4) return fail(HS_EINVAL, "order must be 1, 2 or 4");
  if (coeffs1)
    for (size_t j = 0; j < n_terms; ++j)
      if (!std::isfinite(coeffs1[j])) return fail(HS_EINVAL, "non-finite H1 coefficient at term " + std::to_string(j));
  std::unique_ptr<hs_factors> f(new hs_factors());
  std::string err;
  int rc = cached_plan(x, z, coeffs, n_terms, n_qubits, diag_budget, dtype, order, f->plan, &err);
  if (rc != HS_OK) return fail(rc, err);
  f->dtype = dtype;
  f->n_steps = n_steps;
  f->t = t;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&f->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");

  const hs::Plan& p = f->plan;
  const int G = int(p.groups.size());
  const int nd = int(p.offs.size());
  const size_t vbytes = size_t(p.total_elems + p.total_vt) * hs::elem_bytes(dtype);
  hs_factors* fp = f.get();
  auto guard = [&](cudaError_t e2, const char* what) -> int { return e2 == cudaSuccess ? HS_OK : cuda_fail(e2, what); };
  // Stream-ordered allocations (building, using and freeing a factor set never
  // synchronises the device): one for the values and one for every table --
  // the persistent per-diagonal / per-factor / slot tables and the term tables
  // the values are built from -- filled by a single host-to-device copy.
  if ((rc = guard(hs::pool_malloc(&fp->d_vals, vbytes, s), "cudaMallocAsync(values)"))) {
    release(f.release(), s);
    return rc;
  }
  fp->d_vt = static_cast<unsigned char*>(fp->d_vals) + size_t(p.total_elems) * hs::elem_bytes(dtype);
  const size_t m = n_terms;
  std::vector<int> fD(G), fd0(G), gfirst(G), glast(G), xdim(G), pivot(G * hs::kMaxXDim, 0), vt0(G), gkind(G),
      gdir(G), dep_all, dep_notab, dep_tab, tab_groups, row_groups;
  std::vector<uint32_t> smask(G);
  std::vector<uint64_t> basis(G * hs::kMaxXDim, 0);
  for (int g = 0; g < G; ++g) {
    const hs::Group& gr = p.groups[g];
    fD[g] = gr.D;
    fd0[g] = gr.diag0;
    gfirst[g] = gr.first;
    glast[g] = gr.last;
    xdim[g] = gr.xdim;
    smask[g] = gr.smask;
    vt0[g] = gr.vt0;
    gkind[g] = gr.kind;
    gdir[g] = gr.dir;
    for (int i = 0; i < gr.xdim; ++i) {
      basis[g * hs::kMaxXDim + i] = gr.basis[i];
      pivot[g * hs::kMaxXDim + i] = gr.pivot[i];
    }
    (gr.vt0 >= 0 ? tab_groups : row_groups).push_back(g);
    bool dep = false;
    for (int j = gr.first; coeffs1 && j < gr.last; ++j) dep = dep || coeffs1[j] != 0.0;
    if (dep) {
      dep_all.push_back(g);
      (gr.vt0 >= 0 ? dep_tab : dep_notab).push_back(g);
    }
  }
  std::vector<unsigned char> blob;
  auto put = [&](const void* src, size_t bytes) {
    size_t off = (blob.size() + 15) / 16 * 16;
    blob.resize(off + std::max<size_t>(bytes, 16));
    if (src && bytes) std::memcpy(blob.data() + off, src, bytes);
    return off;
  };
  const size_t o_offs = put(p.offs.data(), nd * 8), o_rb = put(p.rowbase.data(), nd * 8);
  const size_t o_fD = put(fD.data(), G * 4), o_fd0 = put(fd0.data(), G * 4);
  const size_t o_su = put(p.slot_u.data(), p.slot_u.size() * 4), o_st = put(p.slot_tab.data(), p.slot_tab.size() * 4);
  const size_t o_tab = put(p.tab_rb.data(), p.tab_rb.size() * 8);
  const size_t o_x = put(p.x.data(), m * 8), o_z = put(p.z.data(), m * 8), o_c = put(p.coeff.data(), m * 8);
  const size_t o_c1 = coeffs1 ? put(coeffs1, m * 8) : 0;
  const size_t o_cx = put(p.term_cx.data(), m * 4), o_gf = put(gfirst.data(), G * 4), o_gl = put(glast.data(), G * 4);
  const size_t o_b = put(basis.data(), basis.size() * 8), o_xd = put(xdim.data(), G * 4);
  const size_t o_pv = put(pivot.data(), pivot.size() * 4);
  const size_t o_sm = put(smask.data(), G * 4), o_vt0 = put(vt0.data(), G * 4);
  const size_t o_kind = put(gkind.data(), G * 4), o_dir = put(gdir.data(), G * 4);
  const size_t o_da = put(dep_all.data(), dep_all.size() * 4), o_dn = put(dep_notab.data(), dep_notab.size() * 4);
  const size_t o_dt = put(dep_tab.data(), dep_tab.size() * 4);
  const size_t o_tg = put(tab_groups.data(), tab_groups.size() * 4), o_rg = put(row_groups.data(), row_groups.size() * 4);
  const std::vector<double> hk = hs::kind_steps(p.order, t / double(n_steps));
  const size_t o_h = put(hk.data(), hk.size() * 8);
  const size_t o_fv = put(nullptr, 8);                   // drive value of hs_factors_set_drive
  const size_t o_cs = put(nullptr, m * 16 * hk.size());  // (cos, sin) per term and angle kind, written on the device
  const size_t o_th = put(nullptr, m * 8 * hk.size());   // the angles themselves
  const size_t o_rq = put(nullptr, m * 32 * hk.size());  // register-sweep record per term and angle kind
  unsigned char* d_blob = nullptr;
  if ((rc = guard(hs::pool_malloc((void**)&d_blob, blob.size(), s), "cudaMallocAsync(tables)"))) {
    release(f.release(), s);
    return rc;
  }
  fp->d_tables = d_blob;
  fp->d_offs = reinterpret_cast<int64_t*>(d_blob + o_offs);
  fp->d_rowbase = reinterpret_cast<int64_t*>(d_blob + o_rb);
  fp->d_fac_D = reinterpret_cast<int*>(d_blob + o_fD);
  fp->d_fac_diag0 = reinterpret_cast<int*>(d_blob + o_fd0);
  fp->d_slot_u = reinterpret_cast<uint32_t*>(d_blob + o_su);
  fp->d_slot_tab = reinterpret_cast<int32_t*>(d_blob + o_st);
  fp->d_tab_rb = reinterpret_cast<int64_t*>(d_blob + o_tab);
  hs_build_inputs& bi = fp->bin;
  bi.x = reinterpret_cast<const uint64_t*>(d_blob + o_x);
  bi.z = reinterpret_cast<const uint64_t*>(d_blob + o_z);
  bi.coeff = reinterpret_cast<const double*>(d_blob + o_c);
  bi.coeff1 = coeffs1 ? reinterpret_cast<const double*>(d_blob + o_c1) : nullptr;
  bi.cx = reinterpret_cast<const uint32_t*>(d_blob + o_cx);
  bi.gfirst = reinterpret_cast<const int*>(d_blob + o_gf);
  bi.glast = reinterpret_cast<const int*>(d_blob + o_gl);
  bi.basis = reinterpret_cast<const uint64_t*>(d_blob + o_b);
  bi.xdim = reinterpret_cast<const int*>(d_blob + o_xd);
  bi.pivot = reinterpret_cast<const int*>(d_blob + o_pv);
  bi.smask = reinterpret_cast<const uint32_t*>(d_blob + o_sm);
  bi.vt0 = reinterpret_cast<const int*>(d_blob + o_vt0);
  bi.kind = reinterpret_cast<const int*>(d_blob + o_kind);
  bi.dir = reinterpret_cast<const int*>(d_blob + o_dir);
  bi.h = reinterpret_cast<const double*>(d_blob + o_h);
  bi.cs = reinterpret_cast<double*>(d_blob + o_cs);
  bi.th = reinterpret_cast<double*>(d_blob + o_th);
  bi.rq = reinterpret_cast<double*>(d_blob + o_rq);
  bi.fval = reinterpret_cast<double*>(d_blob + o_fv);
  bi.n_kinds = int(hk.size());
  bi.dep_all = reinterpret_cast<const int*>(d_blob + o_da);
  bi.dep_notab = reinterpret_cast<const int*>(d_blob + o_dn);
  bi.dep_tab = reinterpret_cast<const int*>(d_blob + o_dt);
  bi.n_dep_all = int(dep_all.size());
  bi.n_dep_notab = int(dep_notab.size());
  bi.n_dep_tab = int(dep_tab.size());
  bi.tab_groups = reinterpret_cast<const int*>(d_blob + o_tg);
  bi.row_groups = reinterpret_cast<const int*>(d_blob + o_rg);
  bi.n_tab_groups = int(tab_groups.size());
  bi.n_row_groups = int(row_groups.size());
  if ((rc = guard(cudaError_t(stage_upload(d_blob, blob.data(), o_fv, s)), "table upload"))) {
    cudaStreamSynchronize(s);
    release(f.release(), s);
    return rc;
  }
  e = hs::launch_sincos(fp, nullptr, s);
  if (e == cudaSuccess) e = hs::launch_value_tables(fp, nullptr, 0, s);
  if (e == cudaSuccess && (flags & HS_BUILD_DEFER_DIAGONALS) && !coeffs1)
    fp->diag_pending = true;
  else if (e == cudaSuccess)
    e = hs::launch_build_split(fp, bi.tab_groups, bi.n_tab_groups, bi.row_groups, bi.n_row_groups, s);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);
    release(f.release(), s);
    return cuda_fail(e, "factor build launch");
  }
  *out = f.release();
  return HS_OK;
}

}  // namespace

extern "C" {

const char* hs_last_error(void) { return g_err.c_str(); }

uint64_t hs_kernel_launches(void) { return hs::g_launches.load(std::memory_order_relaxed); }

int hs_debug_bounds(uint64_t* out4, int reset) {
  if (!out4) return hs::report_error(HS_EINVAL, "null argument");
  out4[0] = out4[1] = out4[2] = out4[3] = 0;
#ifdef HS_DEBUG_BOUNDS
  for (hs::BoundsReader r : hs::bounds_readers()) {
    uint64_t w[4];
    if (r(w, reset != 0) != 0) return hs::report_error(HS_ECUDA, "reading a bounds word failed");
    if (w[0] && !out4[0]) { out4[1] = w[1]; out4[2] = w[2]; out4[3] = w[3]; }
    out4[0] += w[0];
  }
  return 1;
#else
  (void)reset;
  return 0;
#endif
}

int hs_build_factors_ex(const uint64_t* x, const uint64_t* z, const double* coeffs, size_t n_terms, int n_qubits,
                        double t, int n_steps, int diag_budget, int order, hs_dtype dtype, void* cuda_stream,
                        hs_factors** out) {
  return build_impl(x, z, coeffs, nullptr, n_terms, n_qubits, t, n_steps, diag_budget, order, dtype, cuda_stream,
                    out);
}

int hs_build_factors_flags(const uint64_t* x, const uint64_t* z, const double* coeffs, size_t n_terms, int n_qubits,
                           double t, int n_steps, int diag_budget, int order, hs_dtype dtype, int flags,
                           void* cuda_stream, hs_factors** out) {
  if (flags & ~int(HS_BUILD_DEFER_DIAGONALS)) {
    if (out) *out = nullptr;
    return fail(HS_EINVAL, "unknown build flag");
  }
  return build_impl(x, z, coeffs, nullptr, n_terms, n_qubits, t, n_steps, diag_budget, order, dtype, cuda_stream,
                    out, flags);
}

int hs_build_factors_td(const uint64_t* x, const uint64_t* z, const double* coeffs0, const double* coeffs1,
                        size_t n_terms, int n_qubits, double t, int n_steps, int diag_budget, int order,
                        hs_dtype dtype, void* cuda_stream, hs_factors** out) {
  if (!coeffs1) {
    if (out) *out = nullptr;
    return fail(HS_EINVAL, "coeffs1 is NULL");
  }
  return build_impl(x, z, coeffs0, coeffs1, n_terms, n_qubits, t, n_steps, diag_budget, order, dtype, cuda_stream,
                    out);
}

int hs_build_factors_masks(const uint64_t* x, const uint64_t* z, const double* coeffs, size_t n_terms, int n_qubits,
                           double t, int n_steps, int diag_budget, hs_dtype dtype, void* cuda_stream,
                           hs_factors** out) {
  return hs_build_factors_ex(x, z, coeffs, n_terms, n_qubits, t, n_steps, diag_budget, 1, dtype, cuda_stream, out);
}

int hs_factors_sequence(const hs_factors* f, int* order, int* seq, int capacity, int* seq_len) {
  if (!f) return fail(HS_EINVAL, "factors is NULL");
  const std::vector<int>& q = f->plan.step_seq;
  if (order) *order = f->plan.order;
  if (seq_len) *seq_len = int(q.size());
  if (seq) {
    if (capacity < int(q.size())) return fail(HS_EINVAL, "seq capacity too small");
    for (size_t k = 0; k < q.size(); ++k) seq[k] = q[k];
  }
  return HS_OK;
}

int hs_parse_terms(const char* const* labels, size_t n_terms, uint64_t* x, uint64_t* z, int* n_qubits) {
  if (!x || !z || !n_qubits) return fail(HS_EINVAL, "null output array");
  std::vector<uint64_t> xv, zv;
  int nq = 0;
  std::string err;
  int rc = hs::parse_labels(labels, n_terms, xv, zv, nq, &err);
  if (rc != HS_OK) return fail(rc, err);
  std::copy(xv.begin(), xv.end(), x);
  std::copy(zv.begin(), zv.end(), z);
  *n_qubits = nq;
  return HS_OK;
}

int hs_build_factors(const char* const* pauli_terms, const double* coeffs, size_t n_terms, double t, int n_steps,
                     int diag_budget, hs_dtype dtype, void* cuda_stream, hs_factors** out) {
  if (!out) return fail(HS_EINVAL, "out is NULL");
  *out = nullptr;
  std::vector<uint64_t> x, z;
  int nq = 0;
  std::string err;
  int rc = hs::parse_labels(pauli_terms, n_terms, x, z, nq, &err);
  if (rc != HS_OK) return fail(rc, err);
  return hs_build_factors_masks(x.data(), z.data(), coeffs, n_terms, nq, t, n_steps, diag_budget, dtype, cuda_stream,
                                out);
}

int hs_plan_factors(const uint64_t* x, const uint64_t* z, size_t n_terms, int n_qubits, int diag_budget,
                    hs_dtype dtype, int* n_factors, int* n_offsets, int* group_first, int* group_last, int* n_diags,
                    int64_t* offsets, int64_t* value_bytes, int capacity_factors, int capacity_offsets) {
  if (!x || !z || !n_factors || !n_offsets) return fail(HS_EINVAL, "null argument");
  if (!valid_dtype(dtype)) return fail(HS_EDTYPE, "dtype must be HS_C64 or HS_C128");
  hs::Plan p;
  std::string err;
  int rc = hs::make_plan(x, z, nullptr, n_terms, n_qubits, diag_budget, dtype, p, &err);
  if (rc != HS_OK) return fail(rc, err);
  const int G = int(p.groups.size());
  *n_factors = G;
  *n_offsets = int(p.offs.size());
  if (value_bytes) *value_bytes = (p.total_elems + p.total_vt) * int64_t(hs::elem_bytes(dtype));
  if (group_first && group_last && n_diags && capacity_factors >= G)
    for (int g = 0; g < G; ++g) {
      group_first[g] = p.groups[g].first;
      group_last[g] = p.groups[g].last;
      n_diags[g] = p.groups[g].D;
    }
  if (offsets && capacity_offsets >= int(p.offs.size()))
    for (size_t k = 0; k < p.offs.size(); ++k) offsets[k] = p.offs[k];
  return HS_OK;
}

int hs_plan_schedule(const uint64_t* x, const uint64_t* z, size_t n_terms, int n_qubits, int diag_budget, int order,
                     hs_dtype dtype, int n_steps, int tile_bits, int low_bits, int max_fuse, int commuting,
                     int* n_apps, int* n_sweeps, int* app_factor, int* app_step, int* sweep_of, int capacity) {
  if (!x || !z || !n_apps || !n_sweeps) return fail(HS_EINVAL, "null argument");
  if (!valid_dtype(dtype)) return fail(HS_EDTYPE, "dtype must be HS_C64 or HS_C128");
  if (n_steps < 0 || n_steps > 65535) return fail(HS_EINVAL, "n_steps must be 0..65535");
  if (tile_bits < 1 || low_bits < 0 || low_bits > tile_bits) return fail(HS_EINVAL, "tile_bits / low_bits out of range");
  hs::Plan p;
  std::string err;
  int rc = hs::make_plan(x, z, nullptr, n_terms, n_qubits, diag_budget, dtype, p, &err, order);
  if (rc != HS_OK) return fail(rc, err);
  if (max_fuse <= 0 || max_fuse > hs::kMaxSweepFactors) max_fuse = hs::kMaxSweepFactors;
  const std::vector<hs::Sweep> sw =
      commuting ? hs::plan_sweeps_commuting(p, n_steps, tile_bits, low_bits, hs::kMaxFusedDiags, max_fuse)
                : hs::plan_sweeps(p, n_steps, tile_bits, low_bits, true, hs::kMaxFusedDiags, max_fuse);
  int k = 0;
  const bool fill = app_factor && app_step && sweep_of &&
                    int64_t(capacity) >= int64_t(n_steps) * int64_t(p.step_seq.size());
  for (size_t w = 0; w < sw.size(); ++w)
    for (size_t i = 0; i < sw[w].factors.size(); ++i, ++k)
      if (fill) {
        app_factor[k] = sw[w].factors[i];
        app_step[k] = sw[w].steps[i];
        sweep_of[k] = int(w);
      }
  *n_apps = k;
  *n_sweeps = int(sw.size());
  return HS_OK;
}

// Resolve evolve options: method, tile bits, rhs block, low bits.
int resolve_opts(const hs_factors* f, int n_rhs, const hs_evolve_opts* opts, hs_evolve_opts& o, int& tb, int& rb) {
  o = hs_evolve_opts{HS_METHOD_AUTO, 0, 0, 0, 0, 0, 0, 0};
  if (opts) o = *opts;
  if (o.method == HS_METHOD_AUTO && o.tile_bits == 0 && o.rhs_block == 0 && o.low_bits == 0 && o.max_fuse == 0 &&
      o.smem_kb == 0 && o.no_tables == 0) {
    hs_evolve_opts t;
    if (hs::tuned_opts(f, n_rhs, &t)) {
      t.use_graph = o.use_graph;
      o = t;
    }
  }
  if (o.low_bits <= 0) o.low_bits = min_low_bits(f->dtype);
  if (o.max_fuse <= 0 || o.max_fuse > hs::kMaxSweepFactors) o.max_fuse = hs::kMaxSweepFactors;
  if (o.smem_kb < 0 || size_t(o.smem_kb) * 1024 > hs::kSweepSmemMax) return fail(HS_EINVAL, "smem_kb must be 0..227");
  if (o.low_bits < (f->dtype == HS_C64 ? 1 : 0) || o.low_bits > 12) return fail(HS_EINVAL, "low_bits out of range");
  if (o.method != HS_METHOD_AUTO && o.method != HS_METHOD_PLAIN && o.method != HS_METHOD_FUSED &&
      o.method != HS_METHOD_REG)
    return fail(HS_EINVAL, "unknown method");
  if (o.reg_bits != 0 && o.reg_bits != 4 && o.reg_bits != 5) return fail(HS_EINVAL, "reg_bits must be 0, 4 or 5");
  if (o.method == HS_METHOD_REG) {
    const bool c64 = f->dtype == HS_C64;
    const int B = o.reg_bits > 0 ? o.reg_bits : (c64 ? 5 : 4);
    if (!c64 && B != 4) return fail(HS_EINVAL, "complex128 register sweeps use reg_bits 4");
    const int n = f->plan.n_qubits;
    if (n >= B + 5) {
      o.reg_bits = B;
      rb = 1;
      tb = o.tile_bits > 0 ? o.tile_bits : std::min(c64 ? 13 : 12, n);
      if (tb > n) tb = n;
      const int tb_max = (c64 && B == 5) ? 14 : 13;  // 2^(tile_bits - reg_bits) threads, at most 512
      if (tb < B + 5 || tb > tb_max)
        return fail(HS_EINVAL, "register sweeps take tile_bits reg_bits + 5 .. 13 (14 for complex64 with reg_bits 5)");
      return HS_OK;
    }
    // States too small for a register tile: fused sweeps with their defaults.
    o.method = HS_METHOD_FUSED;
    o.reg_bits = 0;
    o.tile_bits = 0;
    o.rhs_block = 0;
  }
  o.reg_bits = 0;
  rb = o.rhs_block > 0 ? o.rhs_block : pick_rhs_block(f->dtype, n_rhs);
  if (rb != 1 && rb != 2 && rb != 4 && rb != 8 && !(rb == 16 && f->dtype == HS_C64))
    return fail(HS_EINVAL, "rhs_block must be 1, 2, 4, 8 (or 16 for complex64)");
  tb = o.tile_bits > 0 ? o.tile_bits : pick_tile_bits(f, rb);
  if (tb > f->plan.n_qubits) tb = f->plan.n_qubits;
  if (o.method != HS_METHOD_PLAIN && tb > hs::max_tile_bits(f->dtype, rb, fused_dmax(f), hs::kSweepSmemMax))
    return fail(HS_EINVAL, "tile_bits exceeds the shared-memory tile for this rhs_block");
  if (tb < 1) return fail(HS_EINVAL, "tile_bits must be >= 1");
  return HS_OK;
}

int hs_evolve_plan(const hs_factors* f, int n_rhs, int n_steps, const hs_evolve_opts* opts, int* n_sweeps,
                   int* n_plain, int* tile_bits, int* rhs_block) {
  if (!f) return fail(HS_EINVAL, "factors is NULL");
  if (n_rhs < 1 || n_steps < 0) return fail(HS_EINVAL, "n_rhs must be >= 1 and n_steps >= 0");
  hs_evolve_opts o;
  int tb = 0, rb = 0;
  int rc = resolve_opts(f, n_rhs, opts, o, tb, rb);
  if (rc != HS_OK) return rc;
  std::vector<hs::Sweep> sw = schedule(f, n_steps, o, tb);
  QPlans qp;
  if (o.method == HS_METHOD_REG) plan_reg(f, sw, tb, o.reg_bits, qp);
  int ns = 0, np = 0;
  for (const hs::Sweep& w : sw) (w.fused ? ns : np) += 1;
  if (n_sweeps) *n_sweeps = ns;
  if (n_plain) *n_plain = np;
  if (tile_bits) *tile_bits = tb;
  if (rhs_block) *rhs_block = rb;
  return HS_OK;
}

int hs_evolve_ex(const hs_factors* f, void* psi, int n_rhs, int n_steps, const hs_evolve_opts* opts,
                 void* cuda_stream) {
  if (!f) return fail(HS_EINVAL, "factors is NULL");
  if (!psi) return fail(HS_EINVAL, "psi is NULL");
  if (n_rhs < 1) return fail(HS_EINVAL, "n_rhs must be >= 1");
  if (n_steps < 0) return fail(HS_EINVAL, "n_steps must be >= 0");
  if (reinterpret_cast<uintptr_t>(psi) % 16) return fail(HS_EINVAL, "psi must be 16-byte aligned");
  hs_evolve_opts o;
  int tb = 0, rb = 0;
  int rc0 = resolve_opts(f, n_rhs, opts, o, tb, rb);
  if (rc0 != HS_OK) return rc0;
  if (n_steps == 0) return HS_OK;
  {
    cudaError_t e = hs::prepare_kernels();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const size_t state_bytes = size_t(n_rhs) * size_t(f->plan.N) * hs::elem_bytes(f->dtype);
  std::vector<hs::Sweep> sw = schedule(f, n_steps, o, tb);
  QPlans qp;
  if (o.method == HS_METHOD_REG) {
    cudaError_t e = hs::q::prepare_qsweep();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    plan_reg(f, sw, tb, o.reg_bits, qp);
  }
  const QPlans* qpp = qp.empty() ? nullptr : &qp;
  const bool scratch_needed = has_plain(sw);
  const size_t smem_budget = o.smem_kb > 0 ? size_t(o.smem_kb) * 1024 : hs::kSweepSmemDefault;
  if (o.method != HS_METHOD_REG || scratch_needed) {  // the schedule reads stored diagonals
    cudaError_t e = hs::ensure_diagonals(f, s);
    if (e != cudaSuccess) return cuda_fail(e, "factor build launch");
  }

  if (o.use_graph) {
    hs_factors::GraphKey key{psi, n_rhs, n_steps, int(o.method) * 128 + o.max_fuse + 16384 * o.reg_bits,
                             tb + 64 * o.smem_kb, (rb * 64 + o.low_bits) * 2 + (o.no_tables != 0), nullptr, 0};
    cudaGraphExec_t exec = nullptr;
    {
      std::lock_guard<std::mutex> lk(f->graph_mu);
      auto it = f->graphs.find(key);
      if (it != f->graphs.end()) exec = it->second;
    }
    if (!exec) {
      if (scratch_needed) return fail(HS_EINVAL, "use_graph needs a schedule without plain fallbacks");
      cudaStream_t cs;
      cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) { cudaStreamDestroy(cs); return cuda_fail(e, "cudaStreamBeginCapture"); }
      hs::begin_capture_count();
      int rc = enqueue_evolve(f, sw, psi, n_rhs, tb, rb, smem_budget, o.no_tables == 0, nullptr, cs, qpp,
                              o.reg_bits);
      const uint64_t n_kernels = hs::end_capture_count();
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(cs, &graph);
      cudaStreamDestroy(cs);
      if (rc != HS_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      std::lock_guard<std::mutex> lk(f->graph_mu);
      f->graphs[key] = exec;
      std::lock_guard<std::mutex> lk2(g_graph_mu);
      g_graph_kernels[exec] = n_kernels;
    }
    cudaError_t e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    {
      std::lock_guard<std::mutex> lk2(g_graph_mu);
      hs::note_launches(g_graph_kernels[exec]);
    }
    return HS_OK;
  }

  void* scratch = nullptr;
  if (scratch_needed) {
    cudaError_t e = hs::pool_malloc(&scratch, state_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(scratch state)");
  }
  int rc = enqueue_evolve(f, sw, psi, n_rhs, tb, rb, smem_budget, o.no_tables == 0, scratch, s, qpp, o.reg_bits);
  if (scratch) cudaFreeAsync(scratch, s);
  return rc;
}

int hs_evolve(const hs_factors* f, void* psi, int n_rhs, int n_steps, void* cuda_stream) {
  return hs_evolve_ex(f, psi, n_rhs, n_steps, nullptr, cuda_stream);
}

// The launches of a time-dependent evolution. Register sweeps generate their
// factor values from per-term records, so with the records of every step
// computed up front (one set per drive sample) a sweep may span steps as in
// hs_evolve_ex; that holds when every sweep of the n_steps-step schedule is a
// register sweep (returns true). Otherwise (stored factors, value tables,
// plain launches) the values change from step to step and sw is one step's
// launches, repeated.
static bool plan_td(const hs_factors* f, int n_steps, const hs_evolve_opts& o, int tb, std::vector<hs::Sweep>& sw,
                    QPlans& qp) {
  if (o.method == HS_METHOD_REG && n_steps > 1 && n_steps <= 65535) {
    sw = schedule(f, n_steps, o, tb);
    plan_reg(f, sw, tb, o.reg_bits, qp, int(f->plan.x.size()) * f->plan.n_kinds);
    if (!has_plain(sw)) return true;
  }
  sw = schedule(f, 1, o, tb);
  qp.clear();
  if (o.method == HS_METHOD_REG) plan_reg(f, sw, tb, o.reg_bits, qp);
  return false;
}

int hs_evolve_td_plan(const hs_factors* f, int n_rhs, int n_steps, const hs_evolve_opts* opts, int* n_sweeps,
                      int* n_plain, int* tile_bits, int* rhs_block) {
  if (!f) return fail(HS_EINVAL, "factors is NULL");
  if (!f->bin.coeff1) return fail(HS_EINVAL, "factors are not time-dependent (built without H1 coefficients)");
  if (n_rhs < 1 || n_steps < 0) return fail(HS_EINVAL, "n_rhs must be >= 1 and n_steps >= 0");
  hs_evolve_opts o;
  int tb = 0, rb = 0;
  int rc = resolve_opts(f, n_rhs, opts, o, tb, rb);
  if (rc != HS_OK) return rc;
  int ns = 0, np = 0;
  if (n_steps > 0) {
    std::vector<hs::Sweep> sw;
    QPlans qp;
    const int reps = plan_td(f, n_steps, o, tb, sw, qp) ? 1 : n_steps;
    for (const hs::Sweep& w : sw) (w.fused ? ns : np) += reps;
  }
  if (n_sweeps) *n_sweeps = ns;
  if (n_plain) *n_plain = np;
  if (tile_bits) *tile_bits = tb;
  if (rhs_block) *rhs_block = rb;
  return HS_OK;
}

// Rebuild the values of the groups that depend on the drive for the drive
// value at d_fval: angles, the value tables of those groups, then the stored
// diagonals of the listed groups.
static cudaError_t enqueue_drive_rebuild(const hs_factors* f, const double* d_fval, const int* diag_groups,
                                         int n_diag, cudaStream_t s) {
  const hs_build_inputs& b = f->bin;
  cudaError_t e = hs::launch_sincos(f, d_fval, s);
  if (e == cudaSuccess && b.n_dep_tab > 0) e = hs::launch_value_tables(f, b.dep_tab, b.n_dep_tab, s);
  if (e == cudaSuccess && n_diag > 0) {
    if (diag_groups == b.dep_all)  // every driven factor: copy the tabled ones, build the others
      e = hs::launch_build_split(f, b.dep_tab, b.n_dep_tab, b.dep_notab, b.n_dep_notab, s);
    else if (diag_groups == b.dep_notab)
      e = hs::launch_build_split(f, nullptr, 0, b.dep_notab, b.n_dep_notab, s);
    else
      e = hs::launch_build(f, diag_groups, n_diag, s);
  }
  return e;
}

int hs_factors_set_drive(hs_factors* f, double drive, void* cuda_stream) {
  if (!f) return fail(HS_EINVAL, "factors is NULL");
  if (!f->bin.coeff1) return fail(HS_EINVAL, "factors are not time-dependent (built without H1 coefficients)");
  if (!std::isfinite(drive)) return fail(HS_EINVAL, "drive value must be finite");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaError_t(stage_upload(f->bin.fval, &drive, sizeof(double), s));
  if (e == cudaSuccess) e = enqueue_drive_rebuild(f, f->bin.fval, f->bin.dep_all, f->bin.n_dep_all, s);
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "drive rebuild");
}

int hs_evolve_td(hs_factors* f, void* psi, int n_rhs, const double* drive, int n_steps, const hs_evolve_opts* opts,
                 void* cuda_stream) {
  if (!f) return fail(HS_EINVAL, "factors is NULL");
  if (!f->bin.coeff1) return fail(HS_EINVAL, "factors are not time-dependent (built without H1 coefficients)");
  if (!psi) return fail(HS_EINVAL, "psi is NULL");
  if (n_rhs < 1) return fail(HS_EINVAL, "n_rhs must be >= 1");
  if (n_steps < 0) return fail(HS_EINVAL, "n_steps must be >= 0");
  if (n_steps > 0 && !drive) return fail(HS_EINVAL, "drive is NULL");
  if (reinterpret_cast<uintptr_t>(psi) % 16) return fail(HS_EINVAL, "psi must be 16-byte aligned");
  for (int k = 0; k < n_steps; ++k)
    if (!std::isfinite(drive[k])) return fail(HS_EINVAL, "non-finite drive value at step " + std::to_string(k));
  hs_evolve_opts o;
  int tb = 0, rb = 0;
  int rc0 = resolve_opts(f, n_rhs, opts, o, tb, rb);
  if (rc0 != HS_OK) return rc0;
  if (n_steps == 0) return HS_OK;
  {
    cudaError_t e = hs::prepare_kernels();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const hs_build_inputs& b = f->bin;
  if (o.method == HS_METHOD_REG) {
    cudaError_t e = hs::q::prepare_qsweep();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
  }
  std::vector<hs::Sweep> sw;
  QPlans qp;
  const bool cross = plan_td(f, n_steps, o, tb, sw, qp);
  const int stride = int(f->plan.x.size()) * f->plan.n_kinds;  // records per step
  const QPlans* qpp = qp.empty() ? nullptr : &qp;
  const bool scratch_needed = has_plain(sw);
  const size_t smem_budget = o.smem_kb > 0 ? size_t(o.smem_kb) * 1024 : hs::kSweepSmemDefault;
  const bool tables = o.no_tables == 0;
  // Sweeps that read value tables need only the tables of table groups
  // rebuilt each step; plain launches and table-free sweeps read diagonals.
  // Register sweeps read value tables, the angles and their cos/sin (all
  // rebuilt each step) and no diagonals, so a schedule of register sweeps
  // alone rebuilds no diagonals: they are left to be rebuilt when read.
  const bool reg_only = qpp && !scratch_needed;
  const bool diag_all = !tables || scratch_needed;
  const int* diag_groups = reg_only ? nullptr : (diag_all ? b.dep_all : b.dep_notab);
  const int n_diag = reg_only ? 0 : (diag_all ? b.n_dep_all : b.n_dep_notab);

  // Drive samples and per-step records in library-owned device buffers
  // (captured graphs read them, so growing one drops those graphs).
  auto drop_td_graphs = [&]() {
    std::lock_guard<std::mutex> lk(f->graph_mu);
    bool any = false;
    for (const auto& kv : f->graphs) any = any || kv.first.variant == 1;
    if (!any) return;
    cudaStreamSynchronize(s);
    for (auto it = f->graphs.begin(); it != f->graphs.end();) {
      if (it->first.variant == 1) {
        cudaGraphExecDestroy(it->second);
        it = f->graphs.erase(it);
      } else {
        ++it;
      }
    }
  };
  if (f->drive_cap < n_steps) {
    drop_td_graphs();
    if (f->d_drive) cudaFreeAsync(f->d_drive, s);
    f->d_drive = nullptr;
    f->drive_cap = 0;
    const int cap = std::max(n_steps, 64);
    cudaError_t e = hs::pool_malloc((void**)&f->d_drive, size_t(cap) * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(drive)");
    f->drive_cap = cap;
  }
  const size_t rec_doubles = size_t(6) * stride * n_steps;  // 4 (rq) + 2 (cos, sin) per record
  if (cross && f->steprec_cap < rec_doubles) {
    drop_td_graphs();
    if (f->d_steprec) cudaFreeAsync(f->d_steprec, s);
    f->d_steprec = nullptr;
    f->steprec_cap = 0;
    const size_t cap = std::max(rec_doubles, size_t(6) * stride * 64);
    cudaError_t e = hs::pool_malloc((void**)&f->d_steprec, cap * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(step records)");
    f->steprec_cap = cap;
  }
  {
    cudaError_t e = cudaError_t(stage_upload(f->d_drive, drive, size_t(n_steps) * sizeof(double), s));
    if (e != cudaSuccess) return cuda_fail(e, "drive upload");
  }
  auto enqueue_all = [&](cudaStream_t cs, void* scratch) -> int {
    if (cross) {
      StepRecords rec;
      rec.rq = f->d_steprec;
      rec.cs = f->d_steprec + size_t(4) * stride * n_steps;
      rec.stride = stride;
      rec.n_steps = n_steps;
      cudaError_t e = hs::launch_sincos_steps(f, f->d_drive, n_steps, const_cast<double*>(rec.cs),
                                              const_cast<double*>(rec.rq), cs);
      if (e != cudaSuccess) return cuda_fail(e, "step records launch");
      int rc = enqueue_evolve(f, sw, psi, n_rhs, tb, rb, smem_budget, tables, nullptr, cs, qpp, o.reg_bits, &rec);
      if (rc != HS_OK) return rc;
      // The angles and value tables at the last step's drive; the stored
      // diagonals follow when something reads them (diag_pending below).
      e = enqueue_drive_rebuild(f, f->d_drive + (n_steps - 1), nullptr, 0, cs);
      return e == cudaSuccess ? HS_OK : cuda_fail(e, "drive rebuild");
    }
    for (int k = 0; k < n_steps; ++k) {
      cudaError_t e = enqueue_drive_rebuild(f, f->d_drive + k, diag_groups, n_diag, cs);
      if (e != cudaSuccess) return cuda_fail(e, "drive rebuild");
      int rc = enqueue_evolve(f, sw, psi, n_rhs, tb, rb, smem_budget, tables, scratch, cs, qpp, o.reg_bits);
      if (rc != HS_OK) return rc;
    }
    // Leave every stored value at the last step's drive (register sweeps
    // alone: the angles and tables are; the diagonals follow when read).
    if (!reg_only && !diag_all && b.n_dep_tab > 0) {
      cudaError_t e = hs::launch_build_split(f, b.dep_tab, b.n_dep_tab, nullptr, 0, cs);
      if (e != cudaSuccess) return cuda_fail(e, "factor build launch");
    }
    return HS_OK;
  };
  // Schedules that read stored diagonals need those of every factor current
  // (a register-sweep evolution before leaves them to be rebuilt on first
  // read); after one of register sweeps alone they are left that way.
  if (!reg_only) {
    cudaError_t e = hs::ensure_diagonals(f, s);
    if (e != cudaSuccess) return cuda_fail(e, "factor build launch");
  }
  auto mark_pending = [&]() {
    if (!reg_only) return;
    std::lock_guard<std::mutex> lk(f->diag_mu);
    f->diag_pending = true;
  };

  if (o.use_graph) {
    if (scratch_needed) return fail(HS_EINVAL, "use_graph needs a schedule without plain fallbacks");
    hs_factors::GraphKey key{psi, n_rhs, n_steps, int(o.method) * 128 + o.max_fuse + 16384 * o.reg_bits,
                             tb + 64 * o.smem_kb, (rb * 64 + o.low_bits) * 2 + (o.no_tables != 0), nullptr, 1};
    cudaGraphExec_t exec = nullptr;
    {
      std::lock_guard<std::mutex> lk(f->graph_mu);
      auto it = f->graphs.find(key);
      if (it != f->graphs.end()) exec = it->second;
    }
    if (!exec) {
      cudaStream_t cs;
      cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) { cudaStreamDestroy(cs); return cuda_fail(e, "cudaStreamBeginCapture"); }
      hs::begin_capture_count();
      int rc = enqueue_all(cs, nullptr);
      const uint64_t n_kernels = hs::end_capture_count();
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(cs, &graph);
      cudaStreamDestroy(cs);
      if (rc != HS_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      std::lock_guard<std::mutex> lk(f->graph_mu);
      f->graphs[key] = exec;
      std::lock_guard<std::mutex> lk2(g_graph_mu);
      g_graph_kernels[exec] = n_kernels;
    }
    cudaError_t e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    mark_pending();
    std::lock_guard<std::mutex> lk2(g_graph_mu);
    hs::note_launches(g_graph_kernels[exec]);
    return HS_OK;
  }

  void* scratch = nullptr;
  if (scratch_needed) {
    cudaError_t e = hs::pool_malloc(&scratch, size_t(n_rhs) * size_t(f->plan.N) * hs::elem_bytes(f->dtype), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(scratch state)");
  }
  int rc = enqueue_all(s, scratch);
  if (scratch) cudaFreeAsync(scratch, s);
  if (rc == HS_OK) mark_pending();
  return rc;
}

int hs_apply_factor(const hs_factors* f, int g, const void* x, void* y, int n_rhs, void* cuda_stream) {
  if (!f) return fail(HS_EINVAL, "factors is NULL");
  if (g < 0 || g >= int(f->plan.groups.size())) return fail(HS_EINVAL, "factor index out of range");
  if (!x || !y || x == y) return fail(HS_EINVAL, "x and y must be distinct non-NULL buffers");
  if (n_rhs < 1) return fail(HS_EINVAL, "n_rhs must be >= 1");
  cudaError_t e = hs::ensure_diagonals(f, reinterpret_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "factor build launch");
  e = hs::launch_apply_plain(f, g, x, y, n_rhs, reinterpret_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "apply launch");
}

int hs_inner_device(const void* a, const void* b, int n_qubits, hs_dtype dtype, double* out_device, void* cuda_stream) {
  if (!a || !b || !out_device) return fail(HS_EINVAL, "null buffer");
  if (!valid_dtype(dtype)) return fail(HS_EDTYPE, "dtype must be HS_C64 or HS_C128");
  if (n_qubits < 1 || n_qubits > HS_MAX_QUBITS) return fail(HS_EINVAL, "n_qubits out of range");
  cudaError_t e = hs::launch_inner(a, b, int64_t(1) << n_qubits, dtype, out_device,
                                   reinterpret_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? HS_OK : cuda_fail(e, "inner product launch");
}

int hs_fidelity(const void* a, const void* b, int n_qubits, hs_dtype dtype, void* cuda_stream, double* fid,
                double* norm_a2, double* norm_b2) {
  if (!fid) return fail(HS_EINVAL, "fid is NULL");
  if (!a || !b) return fail(HS_EINVAL, "null buffer");
  if (!valid_dtype(dtype)) return fail(HS_EDTYPE, "dtype must be HS_C64 or HS_C128");
  if (n_qubits < 1 || n_qubits > HS_MAX_QUBITS) return fail(HS_EINVAL, "n_qubits out of range");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  double* d_out = nullptr;
  cudaError_t e = hs::pool_malloc((void**)&d_out, 4 * sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
  e = hs::launch_inner(a, b, int64_t(1) << n_qubits, dtype, d_out, s);
  double h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d_out, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "fidelity");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamSynchronize");
  const double den = h[2] * h[3];
  *fid = den > 0 ? (h[0] * h[0] + h[1] * h[1]) / den : 0.0;
  if (norm_a2) *norm_a2 = h[2];
  if (norm_b2) *norm_b2 = h[3];
  return HS_OK;
}

int hs_factors_info(const hs_factors* f, int* n_factors, int* n_qubits, int* n_steps, hs_dtype* dtype,
                    int64_t* value_bytes) {
  if (!f) return fail(HS_EINVAL, "factors is NULL");
  if (n_factors) *n_factors = int(f->plan.groups.size());
  if (n_qubits) *n_qubits = f->plan.n_qubits;
  if (n_steps) *n_steps = f->n_steps;
  if (dtype) *dtype = f->dtype;
  if (value_bytes) *value_bytes = (f->plan.total_elems + f->plan.total_vt) * int64_t(hs::elem_bytes(f->dtype));
  return HS_OK;
}

int hs_factor_get(const hs_factors* f, int g, int* term_first, int* term_last, int* n_diags, int64_t* offsets,
                  double* values) {
  if (!f) return fail(HS_EINVAL, "factors is NULL");
  if (g < 0 || g >= int(f->plan.groups.size())) return fail(HS_EINVAL, "factor index out of range");
  const hs::Group& G = f->plan.groups[g];
  if (term_first) *term_first = G.first;
  if (term_last) *term_last = G.last;
  if (n_diags) *n_diags = G.D;
  if (offsets)
    for (int k = 0; k < G.D; ++k) offsets[k] = f->plan.offs[G.diag0 + k];
  if (values) {
    cudaError_t e = hs::ensure_diagonals(f, nullptr);  // (legacy stream; the synchronise below covers it)
    if (e != cudaSuccess) return cuda_fail(e, "factor build launch");
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    const int64_t N = f->plan.N;
    const size_t es = hs::elem_bytes(f->dtype);
    int64_t out = 0;
    for (int k = 0; k < G.D; ++k) {
      const int64_t d = f->plan.offs[G.diag0 + k];
      const int64_t len = N - (d < 0 ? -d : d);
      std::vector<unsigned char> buf(size_t(len) * es);
      e = cudaMemcpy(buf.data(), static_cast<const unsigned char*>(f->d_vals) + size_t(f->plan.dstart[G.diag0 + k]) * es,
                     buf.size(), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
      for (int64_t i = 0; i < len; ++i, ++out) {
        if (f->dtype == HS_C64) {
          float v[2];
          std::memcpy(v, buf.data() + size_t(i) * 8, 8);
          values[2 * out] = v[0];
          values[2 * out + 1] = v[1];
        } else {
          std::memcpy(values + 2 * out, buf.data() + size_t(i) * 16, 16);
        }
      }
    }
  }
  return HS_OK;
}

void hs_free_factors(hs_factors* f) {
  if (!f) return;
  cudaDeviceSynchronize();
  release(f, nullptr);
  cudaDeviceSynchronize();
}

int hs_free_factors_async(hs_factors* f, void* cuda_stream) {
  if (!f) return HS_OK;
  release(f, reinterpret_cast<cudaStream_t>(cuda_stream));
  return HS_OK;
}

}  // extern "C"
