// Host-side structural planning: label parsing, budgeted grouping, the
// structural offset sets of each factor (the "structural dry run" of the
// diagonal-set estimation paragraph, Sec. 3.2), canonical diagonal order
// (Tab. 1), the padded storage layout (Eq. 6 with alignment padding only),
// and the tile-sweep schedule used by the fused evolution.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "hs_internal.h"

namespace hs {

namespace {

// All signed sums sum_{k in u} +-2^k, appended to out (2^popcount(u) values).
void append_offsets(uint64_t u, std::vector<int64_t>& out) {
  size_t base = out.size();
  out.push_back(0);
  for (int k = 0; k < 63; ++k) {
    if (!((u >> k) & 1ull)) continue;
    size_t cur = out.size();
    for (size_t i = base; i < cur; ++i) {
      int64_t o = out[i];
      out[i] = o + (int64_t(1) << k);
      out.push_back(o - (int64_t(1) << k));
    }
  }
}

bool canonical_less(int64_t a, int64_t b) {
  int64_t aa = a < 0 ? -a : a, bb = b < 0 ? -b : b;
  return aa != bb ? aa < bb : a < b;
}

// Open group state: GF(2) basis of the x-mask space (reduced echelon form),
// the list of its elements, and the sorted set of structural offsets.
struct OpenGroup {
  std::vector<uint64_t> basis;
  std::vector<int> pivot;
  std::vector<uint64_t> elems{0};
  std::vector<int64_t> offs{0};  // sorted ascending, unique

  uint64_t reduce(uint64_t v) const {
    for (size_t i = 0; i < basis.size(); ++i)
      if ((v >> pivot[i]) & 1ull) v ^= basis[i];
    return v;
  }
  // Offsets of the enlarged set when v (already reduced, nonzero) joins.
  std::vector<int64_t> offsets_with(uint64_t v) const {
    std::vector<int64_t> add;
    for (uint64_t u : elems) append_offsets(u ^ v, add);
    std::vector<int64_t> merged;
    merged.reserve(offs.size() + add.size());
    std::sort(add.begin(), add.end());
    std::set_union(offs.begin(), offs.end(), add.begin(), add.end(), std::back_inserter(merged));
    merged.erase(std::unique(merged.begin(), merged.end()), merged.end());
    return merged;
  }
  void admit(uint64_t v, std::vector<int64_t>&& new_offs) {
    int p = 63 - __builtin_clzll(v);
    for (size_t i = 0; i < basis.size(); ++i)
      if ((basis[i] >> p) & 1ull) basis[i] ^= v;
    basis.push_back(v);
    pivot.push_back(p);
    size_t n = elems.size();
    for (size_t i = 0; i < n; ++i) elems.push_back(elems[i] ^ v);
    offs = std::move(new_offs);
  }
};

}  // namespace

int parse_labels(const char* const* labels, size_t n, std::vector<uint64_t>& x, std::vector<uint64_t>& z,
                 int& n_qubits, std::string* err) {
  if (n == 0 || labels == nullptr) {
    *err = "no terms";
    return HS_EINVAL;
  }
  x.assign(n, 0);
  z.assign(n, 0);
  n_qubits = -1;
  for (size_t j = 0; j < n; ++j) {
    const char* s = labels[j];
    if (!s) {
      *err = "null label at term " + std::to_string(j);
      return HS_EINVAL;
    }
    int len = 0;
    while (s[len]) ++len;
    if (n_qubits < 0) n_qubits = len;
    if (len != n_qubits) {
      *err = "label " + std::to_string(j) + " has length " + std::to_string(len) + ", expected " +
             std::to_string(n_qubits);
      return HS_EINVAL;
    }
    if (len < 1 || len > HS_MAX_QUBITS) {
      *err = "label length must be 1.." + std::to_string(HS_MAX_QUBITS);
      return HS_EINVAL;
    }
    for (int p = 0; p < len; ++p) {
      uint64_t bit = 1ull << (len - 1 - p);
      switch (s[p]) {
        case 'I': break;
        case 'X': x[j] |= bit; break;
        case 'Z': z[j] |= bit; break;
        case 'Y': x[j] |= bit; z[j] |= bit; break;
        default:
          *err = std::string("invalid Pauli character '") + s[p] + "' in label " + std::to_string(j);
          return HS_EINVAL;
      }
    }
  }
  return HS_OK;
}

std::vector<double> kind_steps(int order, double dt) {
  if (order == 2) return {dt * 0.5};
  if (order == 4) {
    // Suzuki's fourth-order recursion S2(p dt)^2 S2((1 - 4p) dt) S2(p dt)^2,
    // p = 1 / (4 - 4^(1/3)); each Strang stage turns its step into two halves.
    const double p = 1.0 / (4.0 - std::pow(4.0, 1.0 / 3.0));
    return {(p * dt) * 0.5, ((1.0 - 4.0 * p) * dt) * 0.5};
  }
  return {dt};
}

int make_plan(const uint64_t* x, const uint64_t* z, const double* coeff, size_t n, int n_qubits, int budget,
              hs_dtype dt, Plan& plan, std::string* err, int order) {
  if (n == 0) { *err = "no terms"; return HS_EINVAL; }
  if (order != 1 && order != 2 && order != 4) { *err = "order must be 1, 2 or 4"; return HS_EINVAL; }
  if (n_qubits < 1 || n_qubits > HS_MAX_QUBITS) {
    *err = "n_qubits must be 1.." + std::to_string(HS_MAX_QUBITS);
    return HS_EINVAL;
  }
  if (budget < 1) { *err = "diag_budget must be >= 1"; return HS_EINVAL; }
  const uint64_t N = 1ull << n_qubits;
  for (size_t j = 0; j < n; ++j) {
    if ((x[j] | z[j]) >= N) { *err = "mask of term " + std::to_string(j) + " exceeds n_qubits"; return HS_EINVAL; }
    if (coeff && !std::isfinite(coeff[j])) { *err = "non-finite coefficient at term " + std::to_string(j); return HS_EINVAL; }
    if (__builtin_popcountll(x[j]) > 12) {
      *err = "term " + std::to_string(j) + " flips more than 12 qubits (over 4096 diagonals)";
      return HS_EINVAL;
    }
  }
  plan = Plan();
  plan.n_qubits = n_qubits;
  plan.N = int64_t(N);
  plan.x.assign(x, x + n);
  plan.z.assign(z, z + n);
  if (coeff) plan.coeff.assign(coeff, coeff + n);
  else plan.coeff.assign(n, 0.0);
  plan.term_cx.assign(n, 0);

  // Next-fit grouping in input order.
  std::vector<std::pair<int, OpenGroup>> closed;
  OpenGroup g;
  int first = 0;
  for (size_t j = 0; j < n; ++j) {
    uint64_t v = g.reduce(x[j]);
    if (v == 0) continue;  // x_j already in the set: offsets unchanged, always admitted
    std::vector<int64_t> nxt = g.offsets_with(v);
    bool empty = (int(j) == first);
    if (empty || int64_t(nxt.size()) <= budget || nxt == g.offs) {
      g.admit(v, std::move(nxt));
    } else {
      closed.emplace_back(first, std::move(g));
      g = OpenGroup();
      first = int(j);
      uint64_t v2 = g.reduce(x[j]);
      if (v2) g.admit(v2, g.offsets_with(v2));
    }
    if (int(g.basis.size()) > kMaxXDim || int(g.offs.size()) > kMaxDiags) {
      *err = "factor starting at term " + std::to_string(first) + " exceeds the implementation limits (" +
             std::to_string(kMaxDiags) + " diagonals, x-mask set of 2^" + std::to_string(kMaxXDim) + ")";
      return HS_EINVAL;
    }
  }
  closed.emplace_back(first, std::move(g));

  // Stored factors: each group once per (angle kind, direction) of the
  // product formula, and the sequence one step applies.
  const int G0 = int(closed.size());
  struct Stage { int kind, dir; };
  std::vector<Stage> stages;
  if (order == 1) stages = {{0, 1}};
  else if (order == 2) stages = {{0, 1}, {0, -1}};
  else stages = {{0, 1}, {0, -1}, {1, 1}, {1, -1}};
  plan.order = order;
  plan.n_kinds = order == 4 ? 2 : 1;
  auto strang = [&](int kind) {  // forward groups, then the reversed groups in reverse order
    for (int i = 0; i < G0; ++i) plan.step_seq.push_back((2 * kind) * G0 + i);
    for (int i = G0 - 1; i >= 0; --i) plan.step_seq.push_back((2 * kind + 1) * G0 + i);
  };
  if (order == 1) {
    for (int i = 0; i < G0; ++i) plan.step_seq.push_back(i);
  } else if (order == 2) {
    strang(0);
  } else {
    for (int kind : {0, 0, 1, 0, 0}) strang(kind);
  }

  // Canonical order, padded layout, bases.
  const int64_t A = align_elems(dt);
  int64_t cursor = 0;
  for (size_t rep = 0; rep < stages.size() * closed.size(); ++rep) {
    const size_t gi = rep % closed.size();
    OpenGroup& og = closed[gi].second;
    Group G;
    G.kind = stages[rep / closed.size()].kind;
    G.dir = stages[rep / closed.size()].dir;
    G.first = closed[gi].first;
    G.last = (gi + 1 < closed.size()) ? closed[gi + 1].first : int(n);
    std::vector<int64_t> o = og.offs;
    std::sort(o.begin(), o.end(), canonical_less);
    G.D = int(o.size());
    G.diag0 = int(plan.offs.size());
    G.xdim = int(og.basis.size());
    for (int i = 0; i < G.xdim; ++i) {
      G.basis[i] = og.basis[i];
      G.pivot[i] = og.pivot[i];
      G.span |= og.basis[i];
    }
    for (int64_t d : o) {
      int64_t len = plan.N - (d < 0 ? -d : d);
      int64_t pad = d < 0 ? ((-d) % A) : 0;  // makes rowbase = start + pad + d a multiple of A
      int64_t start = cursor + pad;
      plan.offs.push_back(d);
      plan.dstart.push_back(start);
      plan.rowbase.push_back(start + (d < 0 ? d : 0));
      G.S += len;
      cursor = (start + len + A - 1) / A * A;
    }
    // Slot tables of a factor that sweeps can hold.
    if (G.D <= kMaxFusedDiags) {
      G.slot0 = int(plan.slot_u.size());
      G.nslot = 1 << G.xdim;
      for (int sl = 0; sl < G.nslot; ++sl) {
        uint64_t u = 0;
        for (int i = 0; i < G.xdim; ++i)
          if ((sl >> i) & 1) u ^= G.basis[i];
        int bits[64], w = 0;
        for (int b = 0; b < 63; ++b)
          if ((u >> b) & 1ull) bits[w++] = b;
        plan.slot_u.push_back(uint32_t(u));
        plan.slot_tab.push_back(int32_t(plan.tab_rb.size()));
        for (int pat = 0; pat < (1 << w); ++pat) {
          int64_t d = 0;
          for (int j = 0; j < w; ++j) d += ((pat >> j) & 1) ? -(int64_t(1) << bits[j]) : (int64_t(1) << bits[j]);
          int k = 0;
          while (k < G.D && plan.offs[G.diag0 + k] != d) ++k;
          if (k == G.D) { *err = "internal: slot offset missing from the factor's diagonals"; return HS_EINVAL; }
          plan.tab_rb.push_back(plan.rowbase[G.diag0 + k]);
        }
      }
    }
    for (int j = G.first; j < G.last; ++j) {
      uint32_t c = 0;
      for (int i = 0; i < G.xdim; ++i)
        if ((x[j] >> G.pivot[i]) & 1ull) c |= 1u << i;
      plan.term_cx[j] = c;
    }
    // Value table of a factor whose terms touch few qubits.  A support that
    // spans at most kMaxVtBits consecutive qubits with at most two gaps is
    // indexed by the whole window (the entries of the gap bits repeat), so a
    // row's index is a shift and a mask.
    if (G.nslot > 0) {
      uint64_t sm = 0;
      for (int j = G.first; j < G.last; ++j) sm |= x[j] | z[j];
      int bits = __builtin_popcountll(sm);
      if (sm) {
        const int lo = __builtin_ctzll(sm), span = 64 - __builtin_clzll(sm) - lo;
        if (span <= kMaxVtBits && span <= bits + 2) {
          sm = ((1ull << span) - 1ull) << lo;
          bits = span;
        }
      }
      if (bits <= kMaxVtBits && sm < (1ull << 32) && (G.nslot << bits) <= kMaxVtSweep) {
        G.smask = uint32_t(sm);
        G.vt0 = int(plan.total_vt);
        G.vt_n = G.nslot << bits;
        plan.total_vt += G.vt_n;
      }
    }
    plan.groups.push_back(G);
  }
  // One extra aligned block: a 16-byte staging copy that straddles the end of
  // the last diagonal stays inside the allocation.
  plan.total_elems = cursor + A;
  plan.slot_tab.push_back(int32_t(plan.tab_rb.size()));

  // Which groups commute: g and h do when every term of one commutes with
  // every term of the other (Pauli strings (x1, z1) and (x2, z2) commute iff
  // |x1 & z2| + |z1 & x2| is even), and then so do their exponentials; the
  // entry of g with itself says whether its own terms commute pairwise (then
  // its factors at any angle and in either term order commute).
  plan.g0 = G0;
  if (G0 <= kMaxCommuteGroups) {
    plan.commute.assign(size_t(G0) * G0, 1);
    auto terms_commute = [&](int i, int j) {
      return (__builtin_popcountll((x[i] & z[j]) ^ (z[i] & x[j])) & 1) == 0;
    };
    for (int g = 0; g < G0; ++g)
      for (int h = g; h < G0; ++h) {
        const Group& A = plan.groups[g];
        const Group& B = plan.groups[h];
        bool ok = true;
        for (int i = A.first; ok && i < A.last; ++i)
          for (int j = (g == h ? i + 1 : B.first); ok && j < B.last; ++j) ok = terms_commute(i, j);
        plan.commute[size_t(g) * G0 + h] = plan.commute[size_t(h) * G0 + g] = ok;
      }
  }
  return HS_OK;
}

Runs runs_of(uint64_t mask, int n_bits) {
  Runs r;
  int b = 0;
  while (b < n_bits) {
    if (!((mask >> b) & 1ull)) { ++b; continue; }
    int s = b;
    while (b < n_bits && ((mask >> b) & 1ull)) ++b;
    r.pos[r.n] = int8_t(s);
    r.len[r.n] = int8_t(b - s);
    ++r.n;
  }
  return r;
}

uint64_t two_run_mask(uint64_t used, int n, int T, int low_bits) {
  const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  if (T >= n) return all;
  for (int a = std::max(low_bits, 0); a <= T; ++a) {
    const uint64_t lowm = (1ull << a) - 1;
    const uint64_t hi = used & ~lowm;
    const int w = T - a;
    if (hi == 0) return (1ull << T) - 1;
    if (w == 0) continue;
    const int lo_b = __builtin_ctzll(hi), hi_b = 63 - __builtin_clzll(hi);
    if (hi_b - lo_b + 1 > w) continue;
    int h = lo_b;
    if (h + w > n) h = n - w;
    return lowm | (((1ull << w) - 1) << h);
  }
  return 0;
}


std::vector<Sweep> plan_sweeps_commuting(const Plan& p, int n_steps, int tile_bits, int min_low_bits,
                                         int max_fused_diags, int max_fuse) {
  if (max_fuse < 1 || max_fuse > kMaxSweepFactors) max_fuse = kMaxSweepFactors;
  const int n = p.n_qubits;
  tile_bits = std::min(tile_bits, n);
  const int G0 = p.g0;
  const int per_step = int(p.step_seq.size());
  if (p.commute.empty() || int64_t(n_steps) * per_step > (int64_t(1) << 26))  // no table, or too long to mark
    return plan_sweeps(p, n_steps, tile_bits, min_low_bits, true, max_fused_diags, max_fuse);
  const int L = n_steps * per_step;
  auto fits_alone = [&](int g) {
    return p.groups[g].D <= max_fused_diags && p.groups[g].nslot > 0 && min_low_bits <= tile_bits &&
           two_run_mask(p.groups[g].span, n, tile_bits, min_low_bits) != 0;
  };
  // Applications in the formula's order; a sweep takes the first one not yet
  // applied and then every later one that fits its tile and commutes with all
  // the applications it passes over (those stay, in order, for later sweeps),
  // looking at most two steps past the last one it took.
  std::vector<char> done(size_t(L), 0);
  std::vector<Sweep> out;
  int head = 0;
  while (head < L) {
    const int gh = p.step_seq[head % per_step];
    if (!fits_alone(gh)) {
      Sweep pl;
      pl.fused = false;
      pl.factors.push_back(gh);
      pl.steps.push_back(head / per_step);
      out.push_back(std::move(pl));
      done[head] = 1;
    } else {
      Sweep cur;
      uint64_t used = 0;
      std::vector<int> passed;  // factor ids passed over
      int last = head;
      for (int i = head; i < L && i - last <= 2 * per_step && int(cur.factors.size()) < max_fuse; ++i) {
        if (done[i]) continue;
        const int g = p.step_seq[i % per_step];
        bool take = fits_alone(g) && two_run_mask(used | p.groups[g].span, n, tile_bits, min_low_bits) != 0;
        for (size_t k = 0; take && k < passed.size(); ++k)
          take = p.commute[size_t(g % G0) * G0 + passed[k] % G0] != 0;
        if (take) {
          cur.factors.push_back(g);
          cur.steps.push_back(i / per_step);
          used |= p.groups[g].span;
          done[i] = 1;
          last = i;
        } else {
          passed.push_back(g);
        }
      }
      cur.local_mask = uint32_t(two_run_mask(used, n, tile_bits, min_low_bits));
      out.push_back(std::move(cur));
    }
    while (head < L && done[head]) ++head;
  }
  std::vector<Sweep> in_order = plan_sweeps(p, n_steps, tile_bits, min_low_bits, true, max_fused_diags, max_fuse);
  return in_order.size() <= out.size() ? in_order : out;
}

std::vector<Sweep> plan_sweeps(const Plan& p, int n_steps, int tile_bits, int min_low_bits, bool fused,
                               int max_fused_diags, int max_fuse) {
  if (max_fuse < 1 || max_fuse > kMaxSweepFactors) max_fuse = kMaxSweepFactors;
  std::vector<Sweep> out;
  const int n = p.n_qubits;
  tile_bits = std::min(tile_bits, n);
  auto close = [&](Sweep& s, uint64_t used) {
    s.local_mask = uint32_t(two_run_mask(used, n, tile_bits, min_low_bits));
    out.push_back(std::move(s));
    s = Sweep();
  };
  Sweep cur;
  uint64_t used = 0;
  for (int st = 0; st < n_steps; ++st) {
    for (int g : p.step_seq) {
      const uint64_t span = p.groups[g].span;
      const bool fits_alone = fused && p.groups[g].D <= max_fused_diags && p.groups[g].nslot > 0 &&
                              min_low_bits <= tile_bits &&
                              two_run_mask(span, n, tile_bits, min_low_bits) != 0;
      if (!fits_alone) {
        if (!cur.factors.empty()) close(cur, used);
        used = 0;
        Sweep pl;
        pl.fused = false;
        pl.factors.push_back(g);
        pl.steps.push_back(st);
        out.push_back(std::move(pl));
        continue;
      }
      if (!cur.factors.empty() && (two_run_mask(used | span, n, tile_bits, min_low_bits) == 0 ||
                                   int(cur.factors.size()) >= max_fuse)) {
        close(cur, used);
        used = 0;
      }
      cur.factors.push_back(g);
      cur.steps.push_back(st);
      used |= span;
    }
  }
  if (!cur.factors.empty()) close(cur, used);
  return out;
}

}  // namespace hs
