// Gate programs: gate -> item conversion, pass planning and operation fusion.
//
// A program is an ordered list of items on an nq-qubit vector (dense one-qubit
// matrices, diagonal one-qubit gates, CZ, and the variant-selected diagonal
// local terms of cut gates).  compile_program() splits it into passes whose
// tiles fit shared memory, and inside each pass fuses the items into as few
// shared-memory sweeps as possible:
//   * consecutive one-qubit gates on a qubit multiply into one 2x2 matrix;
//   * every diagonal factor (CZ, phase gates, cut terms) is deferred and
//     applied, as a per-amplitude function of index bits, at the start of the
//     next dense sweep -- diagonal operators commute with each other, and a
//     deferred factor never touches a qubit whose pending matrix is still open.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace cc {

namespace {

inline bool is_zero(cd z) { return z.real() == 0.0 && z.imag() == 0.0; }

void mat_h(cd* u) {
  const double r = 1.0 / std::sqrt(2.0);
  u[0] = r; u[1] = r; u[2] = r; u[3] = -r;
}

// u <- a * u  (2x2, row-major)
void mat_lmul(const cd* a, cd* u) {
  cd r[4];
  r[0] = a[0] * u[0] + a[1] * u[2];
  r[1] = a[0] * u[1] + a[1] * u[3];
  r[2] = a[2] * u[0] + a[3] * u[2];
  r[3] = a[2] * u[1] + a[3] * u[3];
  std::memcpy(u, r, sizeof(r));
}

}  // namespace

cc_status check_gates(const cc_gate* gates, int n_gates, int q) {
  if (n_gates < 0) return fail(CC_EINVAL, "n_gates < 0");
  if (n_gates > 0 && !gates) return fail(CC_EINVAL, "gates is NULL");
  for (int i = 0; i < n_gates; ++i) {
    const cc_gate& g = gates[i];
    if (g.kind < CC_GATE_U3 || g.kind > CC_GATE_CX)
      return fail(CC_EINVAL, "gate " + std::to_string(i) + ": unknown kind " + std::to_string(g.kind));
    if (g.q0 < 0 || g.q0 >= q)
      return fail(CC_EINVAL, "gate " + std::to_string(i) + ": qubit " + std::to_string(g.q0) +
                                 " out of range for q=" + std::to_string(q));
    const bool two = g.kind == CC_GATE_CZ || g.kind == CC_GATE_CX;
    if (two) {
      if (g.q1 < 0 || g.q1 >= q)
        return fail(CC_EINVAL, "gate " + std::to_string(i) + ": qubit " + std::to_string(g.q1) +
                                   " out of range for q=" + std::to_string(q));
      if (g.q1 == g.q0)
        return fail(CC_EINVAL, "gate " + std::to_string(i) + ": two-qubit gate on one qubit");
    }
    if (g.reserved != 0) return fail(CC_EINVAL, "gate " + std::to_string(i) + ": reserved != 0");
    if (g.kind == CC_GATE_U3 &&
        !(std::isfinite(g.theta) && std::isfinite(g.phi) && std::isfinite(g.lambda)))
      return fail(CC_EINVAL, "gate " + std::to_string(i) + ": non-finite U3 angle");
  }
  return CC_OK;
}

cc_status gate_items(const cc_gate& g, int qoff, std::vector<Item>& out) {
  Item it;
  const cd I(0.0, 1.0);
  const int a = g.q0 - qoff;
  switch (g.kind) {
    case CC_GATE_U3: {
      const double c = std::cos(0.5 * g.theta), s = std::sin(0.5 * g.theta);
      it.kind = IT_DENSE;
      it.a = a;
      it.u[0] = c;
      it.u[1] = -std::polar(1.0, g.lambda) * s;
      it.u[2] = std::polar(1.0, g.phi) * s;
      it.u[3] = std::polar(1.0, g.phi + g.lambda) * c;
      out.push_back(it);
      return CC_OK;
    }
    case CC_GATE_H:
      it.kind = IT_DENSE; it.a = a; mat_h(it.u); out.push_back(it); return CC_OK;
    case CC_GATE_X:
      it.kind = IT_DENSE; it.a = a;
      it.u[0] = 0.0; it.u[1] = 1.0; it.u[2] = 1.0; it.u[3] = 0.0;
      out.push_back(it); return CC_OK;
    case CC_GATE_Z: case CC_GATE_S: case CC_GATE_SDG: case CC_GATE_T: case CC_GATE_TDG: {
      cd d1;
      if (g.kind == CC_GATE_Z) d1 = -1.0;
      else if (g.kind == CC_GATE_S) d1 = I;
      else if (g.kind == CC_GATE_SDG) d1 = -I;
      else {
        const double r = 1.0 / std::sqrt(2.0);  // e^{+-i pi/4}
        d1 = cd(r, g.kind == CC_GATE_T ? r : -r);
      }
      it.kind = IT_DIAG1; it.a = a;
      it.u[0] = 1.0; it.u[1] = 0.0; it.u[2] = 0.0; it.u[3] = d1;
      out.push_back(it); return CC_OK;
    }
    case CC_GATE_CZ:
      it.kind = IT_CZ; it.a = a; it.b = g.q1 - qoff; out.push_back(it); return CC_OK;
    case CC_GATE_CX: {  // CX = (I (x) H) CZ (I (x) H)
      Item h;
      h.kind = IT_DENSE; h.a = g.q1 - qoff; mat_h(h.u);
      out.push_back(h);
      it.kind = IT_CZ; it.a = a; it.b = g.q1 - qoff; out.push_back(it);
      out.push_back(h);
      return CC_OK;
    }
    default:
      return fail(CC_EINVAL, "unknown gate kind");
  }
}

namespace {

inline uint64_t item_mask(const Item& it) {
  uint64_t m = 1ull << it.a;
  if (it.kind == IT_CZ) m |= 1ull << it.b;
  return m;
}

// Forward scan: an item is applied when none of its qubits is blocked and it
// is diagonal or its qubit is in the tile; otherwise its qubits become blocked
// (so no later item on them can overtake it).
int scan_pass(const std::vector<Item>& items, const std::vector<char>& applied, uint64_t tile,
              std::vector<int>* take) {
  uint64_t blocked = 0;
  int dense = 0;
  for (size_t i = 0; i < items.size(); ++i) {
    if (applied[i]) continue;
    const Item& it = items[i];
    const uint64_t m = item_mask(it);
    if ((m & blocked) || (it.kind == IT_DENSE && !(tile & (1ull << it.a)))) {
      blocked |= m;
      continue;
    }
    if (it.kind == IT_DENSE) ++dense;
    if (take) take->push_back((int)i);
  }
  return dense;
}

struct PassBuilder {
  HostProgram& hp;
  int nq, k;
  int vpos[64];
  std::vector<DTerm> pend_sign, pend_tab;
  cd pend_u[64][4];
  bool pend_has[64];

  PassBuilder(HostProgram& h, int nq_, const std::vector<int>& tile_bits) : hp(h), nq(nq_) {
    k = (int)tile_bits.size();
    uint64_t tmask = 0;
    for (int t = 0; t < k; ++t) {
      vpos[tile_bits[t]] = t;
      tmask |= 1ull << tile_bits[t];
    }
    int r = 0;
    for (int j = 0; j < nq; ++j)
      if (!(tmask & (1ull << j))) vpos[j] = k + r++;
    for (int j = 0; j < 64; ++j) pend_has[j] = false;
  }

  int add_table(const cd* t4) {
    const int id = (int)(hp.tabs.size() / 4);
    for (int i = 0; i < 4; ++i) hp.tabs.push_back(t4[i]);
    return id;
  }

  void add_diag1(int j, cd d0, cd d1) {
    if (d0 == cd(1.0) && d1 == cd(1.0)) return;
    DTerm t{};
    t.p0 = (uint8_t)vpos[j];
    t.p1 = (uint8_t)vpos[j];
    if (d0 == cd(1.0) && d1 == cd(-1.0)) {
      t.kind = TERM_SIGN;
      pend_sign.push_back(t);
      return;
    }
    cd tab[4] = {d0, 0.0, 0.0, d1};  // index bit + 2 * index bit is 0 or 3
    t.kind = TERM_TABLE;
    t.tab = add_table(tab);
    pend_tab.push_back(t);
  }

  void emit(int type, int t_bit, const cd* u) {
    DOp op{};
    op.type = type;
    op.t = t_bit;
    op.term_begin = (int32_t)hp.terms.size();
    for (auto& d : pend_sign) hp.terms.push_back(d);
    op.term_sign_end = (int32_t)hp.terms.size();
    for (auto& d : pend_tab) hp.terms.push_back(d);
    op.term_end = (int32_t)hp.terms.size();
    pend_sign.clear();
    pend_tab.clear();
    op.mat = -1;
    if (u) {
      op.mat = (int32_t)(hp.mats.size() / 4);
      for (int i = 0; i < 4; ++i) hp.mats.push_back(u[i]);
    }
    hp.ops.push_back(op);
  }

  void flush(int j) {
    if (!pend_has[j]) return;
    pend_has[j] = false;
    const cd* u = pend_u[j];
    if (is_zero(u[1]) && is_zero(u[2])) {
      add_diag1(j, u[0], u[3]);
    } else {
      emit(OP_DENSE, vpos[j], u);
    }
  }

  void add(const Item& it) {
    switch (it.kind) {
      case IT_DENSE:
      case IT_DIAG1:
        if (!pend_has[it.a]) {
          pend_has[it.a] = true;
          std::memcpy(pend_u[it.a], it.u, sizeof(it.u));
        } else {
          mat_lmul(it.u, pend_u[it.a]);
        }
        return;
      case IT_CZ: {
        flush(it.a);
        flush(it.b);
        DTerm t{};
        t.kind = TERM_SIGN;
        t.p0 = (uint8_t)vpos[it.a];
        t.p1 = (uint8_t)vpos[it.b];
        pend_sign.push_back(t);
        return;
      }
      case IT_VAR: {
        flush(it.a);
        DTerm t{};
        t.p0 = (uint8_t)vpos[it.a];
        t.p1 = (uint8_t)(nq + it.slot);
        if (it.var_sign) {
          t.kind = TERM_SIGN;
          pend_sign.push_back(t);
        } else {
          cd tab[4] = {it.d[0][0], it.d[0][1], it.d[1][0], it.d[1][1]};  // x + 2b
          t.kind = TERM_TABLE;
          t.tab = add_table(tab);
          pend_tab.push_back(t);
        }
        return;
      }
    }
  }

  void finish() {
    for (int j = 0; j < nq; ++j) flush(j);
    if (!pend_sign.empty() || !pend_tab.empty()) emit(OP_DIAG, 0, nullptr);
  }
};

void add_pass(HostProgram& hp, const std::vector<Item>& items, const std::vector<int>& take,
              const std::vector<int>& tile_bits, bool first) {
  DPass P{};
  P.nq = hp.nq;
  P.k = (int)tile_bits.size();
  P.n_rest = P.nq - P.k;
  P.init_zero = first ? 1 : 0;
  int low = 0;
  while (low < P.k && tile_bits[low] == low) ++low;
  P.low = low;
  for (int t = 0; t < P.k; ++t) P.tile_bit[t] = (int8_t)tile_bits[t];
  uint64_t tmask = 0;
  for (int b : tile_bits) tmask |= 1ull << b;
  int r = 0;
  for (int j = 0; j < P.nq; ++j)
    if (!(tmask & (1ull << j))) P.rest_bit[r++] = (int8_t)j;
  P.op_begin = (int32_t)hp.ops.size();
  PassBuilder pb(hp, hp.nq, tile_bits);
  for (int i : take) pb.add(items[i]);
  pb.finish();
  P.op_end = (int32_t)hp.ops.size();
  hp.passes.push_back(P);
}

}  // namespace

HostProgram compile_program(const std::vector<Item>& items, int nq, int var_bits, int kmax,
                            int low) {
  HostProgram hp;
  hp.nq = nq;
  hp.var_bits = var_bits;
  std::vector<char> applied(items.size(), 0);
  if (nq <= kmax) {
    std::vector<int> take(items.size());
    for (size_t i = 0; i < items.size(); ++i) take[i] = (int)i;
    std::vector<int> tile(nq);
    for (int j = 0; j < nq; ++j) tile[j] = j;
    add_pass(hp, items, take, tile, true);
    return hp;
  }
  low = std::min(low, kmax);
  const int n_high = kmax - low;
  size_t left = items.size();
  bool first = true;
  while (left > 0 || first) {
    // Urgency of each high qubit: program position of its first pending dense item.
    std::vector<long> urg(nq, (long)items.size() + 1);
    {
      uint64_t seen = 0;
      for (size_t i = 0; i < items.size(); ++i) {
        if (applied[i] || items[i].kind != IT_DENSE) continue;
        const int a = items[i].a;
        if (!(seen & (1ull << a))) {
          seen |= 1ull << a;
          urg[a] = (long)i;
        }
      }
    }
    std::vector<std::vector<int>> cands;
    {
      std::vector<int> hi;
      for (int j = low; j < nq; ++j) hi.push_back(j);
      std::stable_sort(hi.begin(), hi.end(), [&](int x, int y) { return urg[x] < urg[y]; });
      hi.resize(n_high);
      std::sort(hi.begin(), hi.end());
      cands.push_back(hi);
    }
    for (int s = low; s + n_high <= nq; ++s) {
      std::vector<int> hi;
      for (int j = s; j < s + n_high; ++j) hi.push_back(j);
      cands.push_back(hi);
    }
    int best = 0, best_dense = -1;
    for (size_t c = 0; c < cands.size(); ++c) {
      uint64_t tile = (low >= 64) ? ~0ull : ((1ull << low) - 1);
      for (int j : cands[c]) tile |= 1ull << j;
      const int d = scan_pass(items, applied, tile, nullptr);
      if (d > best_dense) {
        best_dense = d;
        best = (int)c;
      }
    }
    uint64_t tile = (1ull << low) - 1;
    std::vector<int> tile_bits;
    for (int j = 0; j < low; ++j) tile_bits.push_back(j);
    for (int j : cands[best]) {
      tile |= 1ull << j;
      tile_bits.push_back(j);
    }
    std::vector<int> take;
    scan_pass(items, applied, tile, &take);
    if (take.empty() && left > 0) {  // cannot happen: the first pending item is always applicable
      hp.nq = -1;
      return hp;
    }
    for (int i : take) applied[i] = 1;
    left -= take.size();
    add_pass(hp, items, take, tile_bits, first);
    first = false;
  }
  return hp;
}

}  // namespace cc
