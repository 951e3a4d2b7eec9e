// Host planner of the register-blocked tile sweep (qsweep.h): the factors of
// a fused sweep become register ops (TAB, ROT, PHASE) and the register
// layouts between them.
#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "hs_internal.h"
#include "qsweep.h"

namespace hs {
namespace q {

namespace {

struct HOp {
  uint8_t type;
  int g;                  // factor
  int term;               // ROT: term index
  std::vector<int> terms; // PHASE: term indices
  uint32_t need;          // ROT / TAB: local bits the op flips
  int rs = 0;             // step of the factor application relative to the sweep's first
};

// Lowest bit of u when u's bits are consecutive (patterns are then a shift and
// a mask), -1 otherwise (patterns gather the bits one by one).
int8_t pattern_shift_of(uint32_t u) {
  if (!u) return 0;
  const int lo = __builtin_ctz(u);
  const uint32_t w = u >> lo;
  return (w & (w + 1u)) == 0 ? int8_t(lo) : int8_t(-1);
}

// pext over a 32-bit mask: the bits of v at the set bits of m, packed.
uint32_t pext32(uint32_t v, uint32_t m) {
  uint32_t out = 0;
  int j = 0;
  for (uint32_t t = m; t; t &= t - 1u, ++j)
    if (v & (t & (0u - t))) out |= 1u << j;
  return out;
}

}  // namespace

bool plan_qsweep(const hs_factors* f, const std::vector<int>& factors, uint32_t local_mask, int T, int B,
                 Args& a, std::string* why, const std::vector<int>* steps, int step_stride) {
  const Plan& p = f->plan;
  const int n = p.n_qubits;
  const int m = int(p.x.size());
  auto fail = [&](const std::string& s) {
    if (why) *why = s;
    return false;
  };
  if (B < 4 || B > kMaxB || T < B + 5 || T > n || __builtin_popcount(local_mask) != T)
    return fail("tile and register bits out of range");
  const bool c64 = f->dtype == HS_C64;
  if (!c64 && B != 4) return fail("complex128 uses 4 register bits");
  // Two-run local mask [0, lo) U [h, h + w).
  int lo = 0;
  while (lo < 32 && ((local_mask >> lo) & 1u)) ++lo;
  const uint32_t hi = lo < 32 ? (local_mask & ~((1u << lo) - 1u)) : 0u;
  const int w = __builtin_popcount(hi);
  const int h = hi ? __builtin_ctz(hi) : lo;
  if (lo + w != T || (hi && hi != (((1u << w) - 1u) << h))) return fail("local mask is not two runs");
  if (c64 && lo < 1) return fail("complex64 tiles keep bit 0");
  a = Args();
  a.tile_bits = T;
  a.m0 = lo >= 32 ? 0xffffffffu : ((1u << lo) - 1u);
  a.m1 = ((1u << w) - 1u) << lo;
  a.sh = h - lo;
  const uint64_t all = (1ull << n) - 1ull;
  a.rest = runs_of(~uint64_t(local_mask) & all, n);
  auto loc = [&](uint64_t g) -> uint32_t {  // local image of global bits inside the tile
    const uint32_t v = uint32_t(g & local_mask);
    return (v & a.m0) | ((v >> a.sh) & a.m1);
  };
  auto glob = [&](uint32_t l) -> uint32_t { return (l & a.m0) | ((l & a.m1) << a.sh); };

  // 1. Ops of every factor, in application order.
  if (steps && steps->size() != factors.size()) return fail("one step per factor application");
  std::vector<HOp> ops;
  for (size_t fi = 0; fi < factors.size(); ++fi) {
    const int g = factors[fi];
    const int rs = steps ? (*steps)[fi] - (*steps)[0] : 0;
    const size_t first_op = ops.size();
    const Group& G = p.groups[g];
    if ((G.span & ~uint64_t(local_mask)) != 0) return fail("factor flips outside the tile");
    // A factor of several terms with a value table of at most two slots (a
    // Heisenberg bond) is read from its table; a single term is cheaper as
    // its rotation.
    if (G.last - G.first > 1 && G.vt0 >= 0 && G.nslot >= 1 && G.nslot <= 2 && G.vt_n <= kMaxVt) {
      const uint32_t u = G.nslot == 2 ? p.slot_u[G.slot0 + 1] : 0u;
      if (__builtin_popcount(loc(u)) <= 2) {
        // (value tables hold one step's values: not in a sweep that spans steps)
        if (steps) return fail("a value-table factor in a sweep over steps");
        ops.push_back(HOp{OP_TAB, g, -1, {}, loc(u)});
        continue;
      }
    }
    std::vector<int> run;
    const int cnt = G.last - G.first;
    for (int q = 0; q < cnt; ++q) {
      const int j = G.dir > 0 ? G.first + q : G.last - 1 - q;
      if (p.x[j] == 0) {
        run.push_back(j);
        continue;
      }
      if (!run.empty()) {
        ops.push_back(HOp{OP_PHASE, g, -1, run, 0});
        run.clear();
      }
      const uint32_t need = loc(p.x[j]);
      if (__builtin_popcount(need) > 2) return fail("a term flips more than two qubits");
      ops.push_back(HOp{OP_ROT, g, j, {}, need});
    }
    if (!run.empty()) ops.push_back(HOp{OP_PHASE, g, -1, run, 0});
    for (size_t k = first_op; k < ops.size(); ++k) ops[k].rs = rs;
  }

  // 2. Register layouts: a register op needs its flips (and, for complex64,
  // local bit 0, which a 16-byte chunk keeps in one thread) in the register
  // bits; a new layout takes the needs of as many following ops as fit.
  const uint32_t pin = c64 ? 1u : 0u;
  const uint32_t tile_all = (T >= 32) ? 0xffffffffu : ((1u << T) - 1u);
  // Spare register slots take bits above the five lowest chunk bits (local
  // bits 1..5 for complex64, 0..4 for complex128) first, highest first, so
  // that those bits stay thread bits: the lanes then span 32 consecutive
  // 16-byte chunks and the direct stores of the last layout write whole
  // 32-byte sectors.
  const int lane_lo = c64 ? 1 : 0, lane_hi = lane_lo + 5;
  auto fill = [&](uint32_t R) {
    for (int b = T - 1; b >= 0 && __builtin_popcount(R) < B; --b)
      if (b >= lane_hi || b < lane_lo) R |= 1u << b;
    for (int b = lane_lo; b < lane_hi && b < T && __builtin_popcount(R) < B; ++b) R |= 1u << b;
    return R;
  };
  std::vector<uint32_t> lay_of(ops.size(), 0);
  uint32_t cur = 0;
  bool have = false;
  for (size_t i = 0; i < ops.size(); ++i) {
    const bool reg = ops[i].type != OP_PHASE;
    if (reg && (!have || ((ops[i].need | pin) & ~cur))) {
      uint32_t R = ops[i].need | pin;
      if (__builtin_popcount(R) > B) return fail("an op needs more register bits than a thread has");
      for (size_t j = i + 1; j < ops.size(); ++j) {
        if (ops[j].type == OP_PHASE) continue;
        if (__builtin_popcount(R | ops[j].need) > B) break;
        R |= ops[j].need;
      }
      cur = fill(R);
      if (!have)  // ops before the first register op run in the first layout
        for (size_t k = 0; k < i; ++k) lay_of[k] = cur;
      have = true;
    }
    lay_of[i] = have ? cur : 0u;
  }
  if (!have) {
    cur = fill(pin);
    for (size_t i = 0; i < ops.size(); ++i) lay_of[i] = cur;
  }

  // 3. Emit the descriptor.  Thread positions of a layout: five lane bits,
  // then the warp bits (thread index bits 5 and up).  A layout keeps the
  // previous layout's warp bits when they are still thread bits, so that the
  // change is a warp-local exchange (each warp writes and reads back the same
  // rows, with no CTA-wide barrier); otherwise it prefers warp bits that the
  // next layout can keep.
  std::vector<uint32_t> seq;  // distinct consecutive layouts
  for (size_t i = 0; i < ops.size(); ++i)
    if (seq.empty() || seq.back() != lay_of[i]) seq.push_back(lay_of[i]);
  const int n_warp_bits = std::max(0, (T - B) - 5);
  std::vector<std::vector<int>> warp_pos(seq.size());
  for (size_t li = 0; li < seq.size(); ++li) {
    const uint32_t thr_mask = tile_all & ~seq[li];
    std::vector<int> w;
    if (li > 0) {
      bool keep = true;
      for (int b : warp_pos[li - 1]) keep = keep && ((thr_mask >> b) & 1u);
      if (keep) w = warp_pos[li - 1];
    }
    if (w.empty() && n_warp_bits > 0) {
      const uint32_t next = li + 1 < seq.size() ? (tile_all & ~seq[li + 1]) : 0u;
      // highest thread bits first, those the next layout also has as thread bits before the others
      for (int pass = 0; pass < 2 && int(w.size()) < n_warp_bits; ++pass)
        for (int b = T - 1; b >= 0 && int(w.size()) < n_warp_bits; --b)
          if (((thr_mask >> b) & 1u) && (pass == 1 || ((next >> b) & 1u)) &&
              std::find(w.begin(), w.end(), b) == w.end())
            w.push_back(b);
      std::sort(w.begin(), w.end());
    }
    warp_pos[li] = w;
  }
  std::map<std::pair<uint32_t, std::vector<int>>, int> lay_id;
  std::map<int, int> rot_id, tab_id;
  std::map<std::tuple<int, int, uint32_t, int>, int> phase_id;  // (factor, first term of the run, layout, relative step)
  auto add_layout = [&](uint32_t R, const std::vector<int>& wpos) -> int {
    const auto key = std::make_pair(R, wpos);
    auto it = lay_id.find(key);
    if (it != lay_id.end()) return it->second;
    if (a.n_lay >= kMaxLayouts) return -1;
    Layout& L = a.lay[a.n_lay];
    L = Layout();
    L.reg = R;
    int i = 0;
    for (uint32_t t = R; t; t &= t - 1u, ++i) {
      const int rp = __builtin_ctz(t);
      const uint32_t bit = 1u << rp;
      L.qoff[i] = (c64 && rp == 0) ? 0u : swz(c64 ? (bit >> 1) : bit);
      L.goff[i] = glob(bit);
    }
    // Lanes: the thread bits that are not warp bits, three whose chunk bits
    // differ mod 3 first (the eight threads of a quarter-warp then hit
    // distinct 16-byte bank groups).
    std::vector<int> lanes;
    for (int b = 0; b < T; ++b)
      if (!((R >> b) & 1u) && std::find(wpos.begin(), wpos.end(), b) == wpos.end()) lanes.push_back(b);
    std::vector<int> order, restp;
    bool used_res[3] = {false, false, false};
    for (int b : lanes) {
      const int res = (c64 ? b - 1 : b) % 3;
      if (order.size() < 3 && res >= 0 && !used_res[res]) {
        used_res[res] = true;
        order.push_back(b);
      } else {
        restp.push_back(b);
      }
    }
    order.insert(order.end(), restp.begin(), restp.end());
    order.insert(order.end(), wpos.begin(), wpos.end());
    L.n_thr = int(order.size());
    for (size_t k = 0; k < order.size(); ++k) L.thr[k] = int8_t(order[k]);
    // The warp's chunk bits W (register and lane bits; chunk bit = local bit
    // - 1 for complex64, whose bit 0 stays inside a chunk), in address order.
    std::vector<int> W;
    for (int b = c64 ? 1 : 0; b < T; ++b)
      if (std::find(wpos.begin(), wpos.end(), b) == wpos.end()) W.push_back(c64 ? b - 1 : b);
    if (W.size() < 5) return -1;
    for (int k = 0; k < 5; ++k) L.wlo[k] = int8_t(W[k]);
    const int nj = 1 << (B - (c64 ? 1 : 0));
    if (int(W.size()) != 5 + (B - (c64 ? 1 : 0))) return -1;
    for (int mm = 0; mm < nj; ++mm) {
      uint32_t c = 0;
      for (int k = 0; k < B - (c64 ? 1 : 0); ++k)
        if ((mm >> k) & 1) c |= 1u << W[5 + k];
      L.mswz[mm] = swz(c);
      L.mglob[mm] = glob(c64 ? (c << 1) : c);
    }
    lay_id[key] = a.n_lay;
    return a.n_lay++;
  };
  auto reg_coords = [&](uint32_t lmask, uint32_t R) { return pext32(lmask & R, R); };

  uint32_t emitted = 0xffffffffu;  // no layout yet
  int seq_i = -1;
  std::vector<PClass> cls;
  std::vector<PTerm> pts;
  for (size_t i = 0; i < ops.size(); ++i) {
    const HOp& h = ops[i];
    const uint32_t R = lay_of[i];
    if (R != emitted) {
      ++seq_i;
      const int li = add_layout(R, warp_pos[seq_i]);
      if (li < 0) return fail("too many register layouts");
      if (a.n_ops >= kMaxOps) return fail("too many ops");
      Op& o = a.ops[a.n_ops++];
      o = Op();
      o.type = OP_LAYOUT;
      o.idx = int16_t(li);
      // bit 0: the warp bits are those of the previous layout (warp-local exchange)
      o.flags = uint8_t(seq_i > 0 && warp_pos[seq_i] == warp_pos[seq_i - 1] ? 1 : 0);
      emitted = R;
    }
    if (a.n_ops >= kMaxOps) return fail("too many ops");
    const Group& G = p.groups[h.g];
    Op o = Op();
    o.type = h.type;
    if (h.type == OP_TAB) {
      auto it = tab_id.find(h.g);
      int ti;
      if (it != tab_id.end()) {
        ti = it->second;
      } else {
        if (a.n_tab >= kMaxTab || a.n_vt + 1 + G.vt_n > kMaxVt) return fail("value tables exceed the sweep's limits");
        ti = a.n_tab++;
        Tab& t = a.tab[ti];
        t.vt0 = G.vt0;
        a.n_vt += a.n_vt & 1;  // every table starts on a 16-byte boundary (two complex64 entries)
        t.s0 = a.n_vt;
        t.n = G.vt_n;
        t.sm = G.smask;
        t.sh = pattern_shift_of(G.smask);
        t.ns = int8_t(G.nslot);
        a.n_vt += G.vt_n;
        tab_id[h.g] = ti;
      }
      o.idx = int16_t(ti);
      o.ku = uint8_t(reg_coords(h.need, R));
    } else if (h.type == OP_ROT || (h.type == OP_PHASE && h.terms.size() == 1)) {
      // (a run of one diagonal term is a diagonal rotation, DROT)
      const int term = h.type == OP_ROT ? h.term : h.terms[0];
      const int key = h.rs * step_stride + G.kind * m + term;
      auto it = rot_id.find(key);
      int ri;
      if (it != rot_id.end()) {
        ri = it->second;
      } else {
        if (a.n_rot >= kMaxRot) return fail("too many rotations");
        ri = a.n_rot++;
        a.rot[ri].cs = key;
        a.rot[ri].fast = (p.x[term] != 0 && p.z[term] == 0) ? 1 : 0;
        rot_id[key] = ri;
      }
      const uint64_t x = p.x[term], z = p.z[term];
      const int y = __builtin_popcountll(x & z);
      o.type = x ? OP_ROT : OP_DROT;
      o.idx = int16_t(ri);
      o.ku = uint8_t(reg_coords(h.need, R));
      const uint32_t zl = loc(z);
      o.zk = uint8_t(reg_coords(zl, R));
      o.zthr = zl & ~R & tile_all;
      o.zrest = uint32_t(z & ~uint64_t(local_mask));
      o.flags = uint8_t((x != 0 && z == 0 ? 1 : 0) | (((y + 3) & 3) << 1));
    } else {
      const auto key = std::make_tuple(h.g, h.terms.front(), R, h.rs);
      auto it = phase_id.find(key);
      int pi;
      if (it != phase_id.end()) {
        pi = it->second;
      } else {
        if (a.n_phase >= kMaxPhase) return fail("too many phase runs");
        pi = a.n_phase++;
        // Classes by local part of z_j; the constant class first.
        std::map<uint32_t, std::vector<int>> by_local;
        by_local[0];
        for (int j : h.terms) by_local[loc(p.z[j])].push_back(j);
        std::vector<std::pair<uint32_t, uint32_t>> keys;  // (mu, local part), constant class excluded
        for (auto& kv : by_local)
          if (kv.first) keys.push_back({reg_coords(kv.first, R), kv.first});
        std::sort(keys.begin(), keys.end());
        Phase& P = a.ph[pi];
        P = Phase();
        P.cls0 = int16_t(cls.size());
        P.ncls = int16_t(1 + keys.size());
        auto add_class = [&](uint32_t lpart, int c0p) {
          PClass c{};
          c.thr = lpart & ~R & tile_all;
          c.t0 = int16_t(pts.size());
          c.c0p = int16_t(c0p);
          c.mu = int16_t(reg_coords(lpart, R));
          for (int j : by_local[lpart])
            pts.push_back(PTerm{h.rs * step_stride + G.kind * m + j, uint32_t(p.z[j] & ~uint64_t(local_mask))});
          c.nt = int16_t(int(pts.size()) - c.t0);
          cls.push_back(c);
        };
        add_class(0u, pi);
        const int NR = 1 << B;
        int pos = 1;
        size_t kk = 0;
        for (int mu = 0; mu < NR; ++mu) {
          P.mu_beg[mu] = int16_t(pos);
          while (kk < keys.size() && int(keys[kk].first) == mu) {
            add_class(keys[kk].second, -1);
            ++kk;
            ++pos;
          }
          if (pos > P.mu_beg[mu]) P.mu_mask |= 1u << mu;
        }
        P.mu_beg[NR] = int16_t(pos);
        if (kk != keys.size()) return fail("internal: phase class outside the register patterns");
        if (int(cls.size()) > kMaxClasses || int(pts.size()) > kMaxPTerms) return fail("phase runs too long");
        phase_id[key] = pi;
      }
      o.idx = int16_t(pi);
    }
    a.ops[a.n_ops++] = o;
  }
  if (a.n_ops == 0) return fail("empty sweep");
  a.n_vt += a.n_vt & 1;
  // Runs of consecutive fast rotations (y = 0, z = 0: X-type terms, which all
  // commute) on distinct single register bits become one ROTN op.
  {
    int w = 0;
    for (int r = 0; r < a.n_ops;) {
      const Op& o = a.ops[r];
      const bool single = o.type == OP_ROT && (o.flags & 1) && __builtin_popcount(o.ku) == 1;
      if (!single) {
        a.ops[w++] = a.ops[r++];
        continue;
      }
      Op n = Op();
      n.type = OP_ROTN;
      int k = r;
      while (k < a.n_ops) {
        const Op& q = a.ops[k];
        if (!(q.type == OP_ROT && (q.flags & 1) && __builtin_popcount(q.ku) == 1) || (n.ku & q.ku)) break;
        const int bit = __builtin_ctz(q.ku);
        if (q.idx > 255) break;
        n.ku |= q.ku;
        if (bit < 4) n.zthr |= uint32_t(q.idx) << (8 * bit);
        else n.zrest |= uint32_t(q.idx) << (8 * (bit - 4));
        ++k;
      }
      a.ops[w++] = n;
      r = k;
    }
    a.n_ops = w;
  }
  a.n_cls = int(cls.size());
  a.n_pterm = int(pts.size());
  std::copy(cls.begin(), cls.end(), a.cls);
  std::copy(pts.begin(), pts.end(), a.pt);
  a.full = 0;
  for (int i = 0; i < a.n_ops; ++i)
    if (a.ops[i].type == OP_TAB || (a.ops[i].type == OP_ROT && !(a.ops[i].flags & 1))) a.full = 1;
  return true;
}

bool plan_qsweep_runs(const hs_factors* f, const std::vector<int>& factors, uint32_t local_mask, int T, int B,
                      std::vector<std::pair<std::vector<int>, std::shared_ptr<Args>>>& out, std::string* why,
                      const std::vector<int>* steps, int step_stride) {
  auto a = std::make_shared<Args>();
  if (plan_qsweep(f, factors, local_mask, T, B, *a, why, steps, step_stride)) {
    out.emplace_back(factors, std::move(a));
    return true;
  }
  if (factors.size() < 2) return false;
  const size_t h = factors.size() / 2;
  const std::vector<int> lo(factors.begin(), factors.begin() + h), hi(factors.begin() + h, factors.end());
  if (!steps) return plan_qsweep_runs(f, lo, local_mask, T, B, out, why) && plan_qsweep_runs(f, hi, local_mask, T, B, out, why);
  // each piece addresses its records relative to its own first step
  const std::vector<int> slo(steps->begin(), steps->begin() + h), shi(steps->begin() + h, steps->end());
  return plan_qsweep_runs(f, lo, local_mask, T, B, out, why, &slo, step_stride) &&
         plan_qsweep_runs(f, hi, local_mask, T, B, out, why, &shi, step_stride);
}

}  // namespace q
}  // namespace hs
