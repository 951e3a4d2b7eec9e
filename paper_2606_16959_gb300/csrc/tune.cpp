// Autotuner for the evolution launch parameters (tile bits, contiguous low
// bits, states per tile, plain vs fused), with a process-wide cache keyed by
// the shape of the problem, so that factor sets built later for the same shape
// (new instances of a family, serving requests) reuse the measured choice.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "hs_internal.h"

namespace hs {
int report_error(int code, const std::string& msg);

namespace {
std::mutex g_tune_mu;
std::map<std::string, hs_evolve_opts> g_tune_cache;
}  // namespace

// Shape class: qubits, precision, number of states, and per factor its flip
// span and slot count (which decide the sweep schedule and stage sizes).
std::string shape_key(const hs_factors* f, int n_rhs) {
  std::ostringstream k;
  k << f->plan.n_qubits << ':' << int(f->dtype) << ':' << n_rhs;
  for (const Group& g : f->plan.groups) k << ':' << std::hex << g.span << '/' << std::dec << g.nslot << '/' << g.D;
  return k.str();
}

bool tuned_opts(const hs_factors* f, int n_rhs, hs_evolve_opts* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune_cache.find(shape_key(f, n_rhs));
  if (it == g_tune_cache.end()) return false;
  *out = it->second;
  return true;
}

void store_tuned(const hs_factors* f, int n_rhs, const hs_evolve_opts& o) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[shape_key(f, n_rhs)] = o;
}

}  // namespace hs

extern "C" int hs_autotune(const hs_factors* f, const void* psi, int n_rhs, int n_steps, void* cuda_stream,
                           hs_evolve_opts* best) {
  if (!f || !psi || !best) return hs::report_error(HS_EINVAL, "null argument");
  if (n_rhs < 1 || n_steps < 1) return hs::report_error(HS_EINVAL, "n_rhs and n_steps must be >= 1");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const hs_dtype dt = f->dtype;
  const size_t bytes = size_t(n_rhs) * size_t(f->plan.N) * hs::elem_bytes(dt);
  void* work = nullptr;
  cudaError_t e = hs::pool_malloc(&work, bytes, s);
  if (e != cudaSuccess) return hs::report_error(e == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA,
                                                std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  std::vector<hs_evolve_opts> cand;
  cand.push_back(hs_evolve_opts{HS_METHOD_PLAIN, 0, 0, 0, 0, 0, 0, 0});
  int planes = 1;
  for (const hs::Group& g : f->plan.groups) planes = std::max(planes, g.nslot);
  const int cap = dt == HS_C64 ? 16 : 8;
  int rb_max = 1;
  while (rb_max * 2 <= n_rhs && rb_max * 2 <= cap) rb_max *= 2;
  for (int rb : {rb_max, rb_max / 2}) {
    if (rb < 1 || (rb != rb_max && rb_max < 4)) continue;
    const int tmax = std::min(f->plan.n_qubits, hs::max_tile_bits(dt, rb, planes, hs::kSweepSmemDefault));
    for (int tb = tmax; tb >= std::max(3, tmax - 4); --tb)
      for (int lb : {1, 2, 3}) {
        if (dt == HS_C128 && lb == 3) continue;
        if (lb > tb) continue;
        for (int kb : {0, 48}) cand.push_back(hs_evolve_opts{HS_METHOD_FUSED, tb, rb, 0, lb, 0, kb, 0});
      }
  }
  // Register-blocked sweeps: register bits, tile bits, contiguous low bits.
  const int n = f->plan.n_qubits;
  for (int B : {5, 4}) {
    if (dt == HS_C128 && B != 4) continue;
    const int tmax = std::min((dt == HS_C64 && B == 5) ? 14 : 13, n);
    for (int tb = tmax; tb >= std::max(B + 5, tmax - 2); --tb)
      for (int lb : {2, 3, 4}) {
        if (lb > tb) continue;
        hs_evolve_opts o{HS_METHOD_REG, tb, 1, 0, lb, 0, 0, 0};
        o.reg_bits = B;
        cand.push_back(o);
      }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  hs_evolve_opts best_o = cand[0];
  int rc = HS_OK;
  auto measure = [&](const hs_evolve_opts& o) {
    float t_min = 1e30f;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      cudaMemcpyAsync(work, psi, bytes, cudaMemcpyDeviceToDevice, s);
      cudaEventRecord(e0, s);
      if (hs_evolve_ex(f, work, n_rhs, n_steps, &o, cuda_stream) != HS_OK) ok = false;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { ok = false; rc = HS_ECUDA; break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      t_min = std::min(t_min, ms);
    }
    if (rc == HS_OK && ok && t_min < best_ms) {
      best_ms = t_min;
      best_o = o;
    }
  };
  for (const hs_evolve_opts& o : cand) {
    measure(o);
    if (rc != HS_OK) break;
  }
  // Step-fusion depth: the most factor applications one sweep launch applies,
  // tried on the winner (the default is the limit, 64).
  if (rc == HS_OK && best_o.method != HS_METHOD_PLAIN) {
    const hs_evolve_opts win = best_o;
    for (int mf : {8, 16, 32}) {
      hs_evolve_opts o = win;
      o.max_fuse = mf;
      measure(o);
      if (rc != HS_OK) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(work, s);
  cudaStreamSynchronize(s);
  if (rc != HS_OK) return hs::report_error(rc, "autotune: a CUDA call failed");
  hs::store_tuned(f, n_rhs, best_o);
  *best = best_o;
  return HS_OK;
}

extern "C" int hs_batch_autotune(const hs_batch_job* jobs, size_t n_jobs, void* cuda_stream, hs_batch_opts* best) {
  if (!jobs || n_jobs == 0 || !best) return hs::report_error(HS_EINVAL, "null argument or no jobs");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const hs_dtype dt = jobs[0].factors ? jobs[0].factors->dtype : HS_C64;
  // Scratch copies of every job's states (16-byte aligned each).
  std::vector<size_t> off(n_jobs + 1, 0);
  for (size_t j = 0; j < n_jobs; ++j) {
    if (!jobs[j].factors || !jobs[j].psi || jobs[j].n_rhs < 1)
      return hs::report_error(HS_EINVAL, "job " + std::to_string(j) + ": null factors or psi");
    const size_t bytes = size_t(jobs[j].n_rhs) * size_t(jobs[j].factors->plan.N) * hs::elem_bytes(jobs[j].factors->dtype);
    off[j + 1] = off[j] + (bytes + 255) / 256 * 256;
  }
  unsigned char* work = nullptr;
  cudaError_t e = hs::pool_malloc(reinterpret_cast<void**>(&work), off[n_jobs], s);
  if (e != cudaSuccess) return hs::report_error(e == cudaErrorMemoryAllocation ? HS_ENOMEM : HS_ECUDA,
                                                std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  std::vector<hs_batch_job> wj(jobs, jobs + n_jobs);
  for (size_t j = 0; j < n_jobs; ++j) wj[j].psi = work + off[j];
  std::vector<hs_batch_opts> cand;
  for (int tb : {9, 10, 11})
    for (int kb : {24, 48})
      for (int tpc : {4, 8}) cand.push_back(hs_batch_opts{tb, 0, 0, kb, 0, tpc, 0, 0});
  for (int B : {5, 4}) {
    if (dt == HS_C128 && B != 4) continue;
    for (int tb : {13, 12})
      for (int lb : {2, 3}) cand.push_back(hs_batch_opts{tb, lb, 0, 0, 0, 0, HS_METHOD_REG, B});
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  hs_batch_opts best_o = cand[0];
  int rc = HS_OK;
  for (const hs_batch_opts& o : cand) {
    hs_batch* b = nullptr;
    if (hs_batch_create(wj.data(), n_jobs, &o, &b) != HS_OK) continue;  // options that do not apply
    float t_min = 1e30f;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      for (size_t j = 0; j < n_jobs; ++j)
        cudaMemcpyAsync(wj[j].psi, jobs[j].psi,
                        size_t(jobs[j].n_rhs) * size_t(jobs[j].factors->plan.N) * hs::elem_bytes(dt),
                        cudaMemcpyDeviceToDevice, s);
      cudaEventRecord(e0, s);
      if (hs_batch_launch(b, cuda_stream) != HS_OK) ok = false;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { ok = false; rc = HS_ECUDA; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      t_min = std::min(t_min, ms);
    }
    hs_batch_free_async(b, cuda_stream);
    if (rc != HS_OK) break;
    if (ok && t_min < best_ms) {
      best_ms = t_min;
      best_o = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(work, s);
  cudaStreamSynchronize(s);
  if (rc != HS_OK) return hs::report_error(rc, "batch autotune: a CUDA call failed");
  best_o.use_graph = best->use_graph == 1 ? 1 : 0;
  *best = best_o;
  return HS_OK;
}
