// Gate programs: gate -> item conversion, pass planning and operation fusion.
//
// A program is an ordered list of items on an nq-qubit vector (dense one-qubit
// matrices, diagonal one-qubit gates, CZ, and the variant-selected diagonal
// local terms of cut gates).  compile_program() splits it into passes whose
// tiles fit shared memory, and inside each pass fuses the items into as few
// shared-memory sweeps as possible:
//   * consecutive one-qubit gates on a qubit multiply into one 2x2 matrix;
//   * every diagonal factor (CZ, phase gates, cut terms) is deferred and
//     applied, as a per-amplitude function of index bits, just before the
//     first dense matrix on a bit it depends on -- diagonal operators commute
//     with each other and with matrices on other bits, and a deferred factor
//     never touches a qubit whose pending matrix is still open;
//   * each fused unitary 2x2 matrix u splits as u = g D_L R D_R (Euler
//     angles: g a scalar, D_L, D_R diagonal phases, R a real rotation), R
//     runs in tangent form at 2 multiply-adds per amplitude instead of the 8
//     of a complex matrix, and every one-bit phase and scalar pending at a
//     flush is applied as one phase block (a few complex products per
//     amplitude however many phases it holds).  The open matrices of a stage
//     are flushed together, so their D_R factors share one phase block.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <stdexcept>

#include "internal.h"

namespace cc {

namespace {

inline bool is_zero(cd z) { return z.real() == 0.0 && z.imag() == 0.0; }

// U3(theta, phi, lambda) = [[cos t/2, -e^{i lambda} sin t/2],
//                            [e^{i phi} sin t/2, e^{i (phi + lambda)} cos t/2]]
void u3_matrix(const double* ang, cd* u) {
  const double c = std::cos(0.5 * ang[0]), s = std::sin(0.5 * ang[0]);
  u[0] = c;
  u[1] = -std::polar(1.0, ang[2]) * s;
  u[2] = std::polar(1.0, ang[1]) * s;
  u[3] = std::polar(1.0, ang[1] + ang[2]) * c;
}

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

// Euler split of a unitary 2x2 matrix u (row-major):
//   u = g diag(e^{iA}, e^{-iA}) T diag(e^{iB}, e^{-iB})
// with T = [[1, -t], [t, 1]] (rot = OP_ROT, t = s/c) or [[t, -1], [1, t]]
// (OP_ROTC, t = c/s) and |t| <= 1: u = w [[p, -conj q], [q, conj p]] with
// w^2 = det u, p = c e^{i theta_p}, q = s e^{i theta_q}, A = (theta_p -
// theta_q)/2, B = (theta_p + theta_q)/2, and the larger of c, s goes into g.
// The half-angle phases come from square roots of unit complex numbers (no
// trigonometric calls); their common sign is fixed by e^{iA} e^{iB} =
// e^{i theta_p}.  False where the product does not reproduce u to 1e-12 (a
// matrix that is not unitary).
struct EulerSplit {
  int rot;
  double t;
  cd g, dl0, dl1, dr0, dr1;
};

// Square root of a unit complex number z = x + iy, in the right half-plane:
// the larger component from its half-angle formula, the smaller as
// y / (2 * larger), which avoids the cancellation in 1 - x near z = 1.
inline cd unit_sqrt(cd z) {
  const double x = std::max(-1.0, std::min(1.0, z.real())), y = z.imag();
  if (x >= 0.0) {
    const double re = std::sqrt(0.5 * (1.0 + x));
    return cd(re, y / (2.0 * re));
  }
  double im = std::sqrt(0.5 * (1.0 - x));
  if (y < 0.0) im = -im;
  return cd(y / (2.0 * im), im);
}

bool euler_split(const cd* u, EulerSplit& e) {
  const cd det = u[0] * u[3] - u[1] * u[2];
  const double ad = std::sqrt(std::norm(det));
  if (!(ad > 0.5 && ad < 2.0)) return false;
  const cd w1 = unit_sqrt(det / ad);  // w = w1 sqrt(ad), |w1| = 1
  const double rw = 1.0 / std::sqrt(ad);
  const cd w = w1 * std::sqrt(ad);
  const cd p = u[0] * std::conj(w1) * rw, q = u[2] * std::conj(w1) * rw;
  const double c = std::sqrt(std::norm(p)), s = std::sqrt(std::norm(q));
  const cd ep = c > 0.0 ? p / c : cd(1.0), eq = s > 0.0 ? q / s : cd(1.0);
  cd eA = unit_sqrt(ep * std::conj(eq)), eB = unit_sqrt(ep * eq);
  if (((eA * eB) * std::conj(ep)).real() < 0.0) eA = -eA;
  double scale;
  if (c >= s) {
    e.rot = OP_ROT;
    e.t = s / c;
    scale = c;
  } else {
    e.rot = OP_ROTC;
    e.t = c / s;
    scale = s;
  }
  e.g = w * scale;
  e.dl0 = eA;
  e.dl1 = std::conj(eA);
  e.dr0 = eB;
  e.dr1 = std::conj(eB);
  const cd T[4] = {e.rot == OP_ROT ? cd(1.0) : cd(e.t), e.rot == OP_ROT ? cd(-e.t) : cd(-1.0),
                   e.rot == OP_ROT ? cd(e.t) : cd(1.0), e.rot == OP_ROT ? cd(1.0) : cd(e.t)};
  const cd dl[2] = {e.dl0, e.dl1}, dr[2] = {e.dr0, e.dr1};
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < 2; ++k)
      if (std::norm(e.g * dl[r] * T[2 * r + k] * dr[k] - u[2 * r + k]) > 1e-24) return false;
  return true;
}

// The rotation engine (Euler split + phase blocks); CUTSIM_ROT=0 applies every
// fused matrix as a complex 2x2 and every phase as a table term instead.
bool rot_engine() {
  const char* e = std::getenv("CUTSIM_ROT");
  return !(e && e[0] == '0');
}

}  // namespace

bool is_two_qubit(int kind) {
  return kind == CC_GATE_CZ || kind == CC_GATE_CX || is_rank4(kind);
}
bool is_rank4(int kind) {
  return kind == CC_GATE_SWAP || kind == CC_GATE_ISWAP || kind == CC_GATE_CAN;
}

// exp(-i (tx XX + ty YY + tz ZZ) / 2) = prod over P of (cos(t_P/2) II - i sin(t_P/2) PP);
// the three factors commute and XX YY = -ZZ, XX ZZ = -YY, YY ZZ = -XX.
void pauli_weights(const cc_gate& g, cd c[4]) {
  const cd I(0.0, 1.0);
  if (g.kind == CC_GATE_SWAP) {  // (II + XX + YY + ZZ) / 2
    c[0] = c[1] = c[2] = c[3] = 0.5;
    return;
  }
  if (g.kind == CC_GATE_ISWAP) {  // (II + ZZ) / 2 + i (XX + YY) / 2
    c[0] = c[3] = 0.5;
    c[1] = c[2] = 0.5 * I;
    return;
  }
  const cd cx = std::cos(0.5 * g.theta), sx = -I * std::sin(0.5 * g.theta);
  const cd cy = std::cos(0.5 * g.phi), sy = -I * std::sin(0.5 * g.phi);
  const cd cz = std::cos(0.5 * g.lambda), sz = -I * std::sin(0.5 * g.lambda);
  c[0] = cx * cy * cz - sx * sy * sz;
  c[1] = sx * cy * cz - cx * sy * sz;
  c[2] = cx * sy * cz - sx * cy * sz;
  c[3] = cx * cy * sz - sx * sy * cz;
}

cc_status check_gates(const cc_gate* gates, int n_gates, int q) {
  if (n_gates < 0) return fail(CC_EINVAL, "n_gates < 0");
  if (n_gates > 0 && !gates) return fail(CC_EINVAL, "gates is NULL");
  for (int i = 0; i < n_gates; ++i) {
    const cc_gate& g = gates[i];
    if (g.kind < CC_GATE_U3 || g.kind > CC_GATE_CAN)
      return fail(CC_EINVAL, "gate " + std::to_string(i) + ": unknown kind " + std::to_string(g.kind));
    if (g.q0 < 0 || g.q0 >= q)
      return fail(CC_EINVAL, "gate " + std::to_string(i) + ": qubit " + std::to_string(g.q0) +
                                 " out of range for q=" + std::to_string(q));
    const bool two = is_two_qubit(g.kind);
    if (two) {
      if (g.q1 < 0 || g.q1 >= q)
        return fail(CC_EINVAL, "gate " + std::to_string(i) + ": qubit " + std::to_string(g.q1) +
                                   " out of range for q=" + std::to_string(q));
      if (g.q1 == g.q0)
        return fail(CC_EINVAL, "gate " + std::to_string(i) + ": two-qubit gate on one qubit");
    }
    if (g.reserved != 0) return fail(CC_EINVAL, "gate " + std::to_string(i) + ": reserved != 0");
    if ((g.kind == CC_GATE_U3 || g.kind == CC_GATE_CAN) &&
        !(std::isfinite(g.theta) && std::isfinite(g.phi) && std::isfinite(g.lambda)))
      return fail(CC_EINVAL, "gate " + std::to_string(i) + ": non-finite angle");
  }
  return CC_OK;
}

cc_status gate_items(const cc_gate& g, int qoff, std::vector<Item>& out) {
  Item it;
  const cd I(0.0, 1.0);
  const int a = g.q0 - qoff;
  switch (g.kind) {
    case CC_GATE_U3: {
      it.kind = IT_DENSE;
      it.a = a;
      it.u3 = true;
      it.ang[0] = g.theta;
      it.ang[1] = g.phi;
      it.ang[2] = g.lambda;
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
    case CC_GATE_SWAP: case CC_GATE_ISWAP: case CC_GATE_CAN: {
      // U = exp(-i (tx XX + ty YY + tz ZZ)/2) times a global phase:
      // SWAP = e^{-i pi/4} CAN(-pi/2, -pi/2, -pi/2), ISWAP = CAN(-pi/2, -pi/2, 0).
      // Each factor is a ZZ phase conjugated into the X basis (H) or the Y
      // basis (V = S H maps Z to Y: V Z V^dag = Y).
      const int b = g.q1 - qoff;
      double t[3] = {g.theta, g.phi, g.lambda};
      cd phase = 1.0;
      if (g.kind != CC_GATE_CAN) {
        t[0] = t[1] = -0.5 * M_PI;
        t[2] = g.kind == CC_GATE_SWAP ? -0.5 * M_PI : 0.0;
        if (g.kind == CC_GATE_SWAP) phase = std::polar(1.0, -0.25 * M_PI);
      }
      auto dense = [&](int q, const cd* u) {
        Item d;
        d.kind = IT_DENSE;
        d.a = q;
        for (int e = 0; e < 4; ++e) d.u[e] = u[e];
        out.push_back(d);
      };
      auto zz = [&](double th) {  // exp(-i th/2 ZZ): e^{-i th/2} on equal bits, e^{+i th/2} else
        if (th == 0.0) return;
        Item d;
        d.kind = IT_DIAG2;
        d.a = a;
        d.b = b;
        const cd e0 = std::polar(1.0, -0.5 * th), e1 = std::polar(1.0, 0.5 * th);
        d.d[0][0] = e0; d.d[0][1] = e1; d.d[1][0] = e1; d.d[1][1] = e0;
        out.push_back(d);
      };
      cd h[4];
      mat_h(h);
      const double r = 1.0 / std::sqrt(2.0);
      const cd vdag[4] = {r, -I * r, r, I * r};  // (S H)^dag = H S^dag
      const cd v[4] = {r, r, I * r, -I * r};     // S H
      zz(t[2]);
      if (t[0] != 0.0) {
        dense(a, h); dense(b, h);
        zz(t[0]);
        dense(a, h); dense(b, h);
      }
      if (t[1] != 0.0) {
        dense(a, vdag); dense(b, vdag);
        zz(t[1]);
        dense(a, v); dense(b, v);
      }
      if (phase != cd(1.0)) {
        Item d;
        d.kind = IT_DIAG1;
        d.a = a;
        d.u[0] = phase; d.u[1] = 0.0; d.u[2] = 0.0; d.u[3] = phase;
        out.push_back(d);
      }
      return CC_OK;
    }
    default:
      return fail(CC_EINVAL, "unknown gate kind");
  }
}

namespace {

inline uint64_t item_mask(const Item& it) {
  uint64_t m = 1ull << it.a;
  if (it.kind == IT_CZ || it.kind == IT_VAR || it.kind == IT_DIAG2) m |= 1ull << it.b;
  return m;
}

// What the planners read of an item, packed: its qubit mask and, for a dense
// item, its qubit's bit (0 for diagonal items).
struct ItemBits {
  uint64_t mask, dense;
};

std::vector<ItemBits> item_bits(const std::vector<Item>& items) {
  std::vector<ItemBits> b(items.size());
  for (size_t i = 0; i < items.size(); ++i)
    b[i] = {item_mask(items[i]), items[i].kind == IT_DENSE ? 1ull << items[i].a : 0ull};
  return b;
}

// The entries of `order` not yet applied, in order.
void drop_applied(std::vector<int>& order, const std::vector<char>& applied) {
  size_t w = 0;
  for (int i : order)
    if (!applied[i]) order[w++] = i;
  order.resize(w);
}

// Forward scan over the items listed in `order` that are not yet applied: an
// item is taken when none of its qubits is blocked and it is diagonal or its
// qubit is in `dense_ok`; otherwise its qubits become blocked, so no later item
// on them can overtake it.  The taken items are appended to `take`.
void scan(const std::vector<ItemBits>& bits, const std::vector<int>& order,
          const std::vector<char>& applied, uint64_t dense_ok, std::vector<int>& take) {
  uint64_t blocked = 0;
  for (int i : order) {
    if (applied[i]) continue;
    const ItemBits b = bits[i];
    if ((b.mask & blocked) || (b.dense & ~dense_ok)) {
      blocked |= b.mask;
      continue;
    }
    take.push_back(i);
  }
}

// counts[c] = the number of dense items scan() would take with dense_ok =
// oks[c], for every candidate c in one pass over the items and without
// branches on them: the candidates' blocked masks are independent chains, so
// the pass runs at instruction throughput rather than at the latency of one
// chain.  Once every allowed qubit of a candidate is blocked no dense item
// can be taken for it any more (such an item's qubit is blocked), so the pass
// stops when that holds for all of them.
constexpr int kMaxCands = 66;  // the earliest-items set and up to 64 windows

void count_dense(const std::vector<ItemBits>& bits, const std::vector<int>& order,
                 const std::vector<char>& applied, const uint64_t* oks, int nc, int* counts) {
  uint64_t blocked[kMaxCands];
  for (int c = 0; c < nc; ++c) {
    blocked[c] = 0;
    counts[c] = 0;
  }
  for (int i : order) {
    const ItemBits b = bits[i];
    const uint64_t live = applied[i] ? 0ull : ~0ull;
    uint64_t open = 0;
    for (int c = 0; c < nc; ++c) {
      const uint64_t hit = ((b.mask & blocked[c]) | (b.dense & ~oks[c])) ? ~0ull : 0ull;
      blocked[c] |= b.mask & hit & live;
      counts[c] += (int)((b.dense & ~hit & live) != 0);
      open |= oks[c] & ~blocked[c];
    }
    if (!open) break;
  }
}

// Choose `width` qubits out of `pool` (ascending) for the dense items to act
// on, plus the always-included `fixed` mask: the candidates are the qubits of
// the earliest pending dense items and every window of `width` consecutive
// pool entries; the one that admits the most dense items wins.
uint64_t choose_set(const std::vector<ItemBits>& bits, const std::vector<int>& order,
                    const std::vector<char>& applied, const std::vector<int>& pool, int width,
                    uint64_t fixed) {
  if (width >= (int)pool.size()) {
    uint64_t m = fixed;
    for (int j : pool) m |= 1ull << j;
    return m;
  }
  std::vector<uint64_t> cands;
  {
    std::vector<int> picked;
    uint64_t seen = 0, in_pool = 0;
    for (int j : pool) in_pool |= 1ull << j;
    for (int i : order) {
      const uint64_t b = bits[i].dense;
      if (applied[i] || !b) continue;
      if ((b & in_pool) && !(b & seen)) {
        seen |= b;
        picked.push_back(__builtin_ctzll(b));
        if ((int)picked.size() == width) break;
      }
    }
    for (int j : pool) {
      if ((int)picked.size() == width) break;
      if (!(seen & (1ull << j))) {
        seen |= 1ull << j;
        picked.push_back(j);
      }
    }
    uint64_t m = fixed;
    for (int j : picked) m |= 1ull << j;
    cands.push_back(m);
  }
  for (size_t s = 0; s + width <= pool.size(); ++s) {
    uint64_t m = fixed;
    for (int w = 0; w < width; ++w) m |= 1ull << pool[s + w];
    cands.push_back(m);
  }
  const int nc = (int)cands.size();  // <= 65: a pool holds at most 64 qubits
  if (nc > kMaxCands) throw std::length_error("candidate qubit sets");
  int counts[kMaxCands];
  count_dense(bits, order, applied, cands.data(), nc, counts);
  uint64_t best = cands[0];
  int best_d = -1;
  for (int c = 0; c < nc; ++c)
    if (counts[c] > best_d) {
      best_d = counts[c];
      best = cands[c];
    }
  return best;
}

struct PassBuilder {
  HostProgram& hp;
  int nq;
  int vpos[64];
  int reg_of[64];
  std::vector<DTerm> pend_sign, pend_tab;
  uint64_t pend_adj = 0;
  cd pend_u[64][4];
  bool pend_has[64];
  // one-bit phases diag(ph0, ph1) on virtual bit p, and a pending scalar
  const bool rot = rot_engine();
  cd ph0[64], ph1[64];
  uint64_t ph_mask = 0;  // virtual bits with a pending one-bit phase
  cd pend_const = 1.0;
  int reg_index[64];  // register index of virtual bit p in the current stage, or -1
  uint64_t reg_mask = 0;  // virtual bits held in registers in the current stage
  bool overflow = false;  // an op with more than 65535 terms of one kind
  int js[64];             // flush_all's open matrices and their splits
  EulerSplit es[64];
  std::vector<std::pair<int, int>> folded_buf;  // emit's working lists, kept between ops
  std::vector<DTerm> signs_buf;

  PassBuilder(HostProgram& h, int nq_, const std::vector<int>& tile_bits) : hp(h), nq(nq_) {
    const int k = (int)tile_bits.size();
    uint64_t tmask = 0;
    for (int t = 0; t < k; ++t) {
      vpos[tile_bits[t]] = t;
      tmask |= 1ull << tile_bits[t];
    }
    int r = 0;
    for (int j = 0; j < nq; ++j)
      if (!(tmask & (1ull << j))) vpos[j] = k + r++;
    for (int j = 0; j < 64; ++j) {
      pend_has[j] = false;
      reg_of[j] = -1;
      reg_index[j] = -1;
    }
  }

  int add_table(const cd* t4) {
    const int id = (int)(hp.tabs.size() / 4);
    for (int i = 0; i < 4; ++i) hp.tabs.push_back(t4[i]);
    return id;
  }

  void add_sign(int p0, int p1) {
    if (p0 > p1) std::swap(p0, p1);
    if (p1 == p0 + 1) {
      pend_adj ^= 1ull << p0;  // a repeated CZ cancels
      return;
    }
    DTerm t{};
    t.kind = TERM_SIGN;
    t.p0 = (uint8_t)p0;
    t.p1 = (uint8_t)p1;
    pend_sign.push_back(t);
  }

  void add_diag1(int j, cd d0, cd d1) {
    if (d0 == cd(1.0) && d1 == cd(1.0)) return;
    if (d0 == cd(1.0) && d1 == cd(-1.0)) {
      add_sign(vpos[j], vpos[j]);
      return;
    }
    if (rot && std::norm(d0) > 1e-300) {  // ph1 / ph0 exists (the entries are finite)
      const int p = vpos[j];
      if ((ph_mask >> p) & 1ull) {
        ph0[p] *= d0;
        ph1[p] *= d1;
      } else {
        ph_mask |= 1ull << p;
        ph0[p] = d0;
        ph1[p] = d1;
      }
      return;
    }
    DTerm t{};
    t.p0 = (uint8_t)vpos[j];
    t.p1 = (uint8_t)vpos[j];
    cd tab[4] = {d0, 0.0, 0.0, d1};  // index bit + 2 * index bit is 0 or 3
    t.kind = TERM_TABLE;
    t.tab = add_table(tab);
    pend_tab.push_back(t);
  }

  // Does a pending diagonal factor depend on index bit vp?
  bool pending_touches(int vp) const {
    if ((ph_mask >> vp) & 1ull) return true;
    if ((pend_adj >> vp) & 1ull) return true;
    if (vp > 0 && ((pend_adj >> (vp - 1)) & 1ull)) return true;
    for (const auto& d : pend_sign)
      if (d.p0 == vp || d.p1 == vp) return true;
    for (const auto& d : pend_tab)
      if (d.p0 == vp || d.p1 == vp) return true;
    return false;
  }

  // Emit an op on index bit vp.  Pending diagonal factors commute with a
  // matrix on a bit they do not depend on, so they stay pending until an op
  // whose bit one of them depends on (or the pass's final OP_DIAG); then all
  // of them ride on that op at once, and a layer of CZs costs one sign sweep.
  void emit(int type, int t_reg, const cd* u, int vp, uint8_t cot = 0,
            uint64_t more_vps = 0) {
    DOp op{};
    op.type = (int8_t)type;
    op.t = (int8_t)t_reg;
    op.cot = cot;
    bool touches = type == OP_DIAG || pending_touches(vp);
    for (uint64_t r = more_vps; r && !touches; r &= r - 1)
      touches = pending_touches(__builtin_ctzll(r));
    const bool attach = touches;
    // A sign whose bits are all register bits of the stage is the same for
    // every thread: when the op gets a phase block it joins the block's
    // entries instead of flipping amplitudes.
    uint64_t adj = attach ? pend_adj : 0;
    // register indices of folded signs, and the signs left as terms
    std::vector<std::pair<int, int>>& folded = folded_buf;
    std::vector<DTerm>& signs = signs_buf;
    folded.clear();
    signs.clear();
    if (attach) {
      const bool block = will_attach_block(type == OP_DIAG);
      for (uint64_t r = adj; block && r; r &= r - 1) {
        const int p = __builtin_ctzll(r);
        if (p + 1 < 64 && reg_index[p] >= 0 && reg_index[p + 1] >= 0) {
          folded.push_back({reg_index[p], reg_index[p + 1]});
          adj &= ~(1ull << p);
        }
      }
      for (const auto& d : pend_sign) {
        if (block && reg_index[d.p0] >= 0 && reg_index[d.p1] >= 0)
          folded.push_back({reg_index[d.p0], reg_index[d.p1]});
        else
          signs.push_back(d);
      }
    }
    op.sign_adj = adj;
    const size_t t0 = hp.terms.size();
    op.term_begin = (int32_t)t0;
    for (auto& d : signs) hp.terms.push_back(d);
    const size_t t1 = hp.terms.size();
    if (attach) attach_phase_block(type == OP_DIAG, folded);
    const size_t t2 = hp.terms.size();
    if (t2 > t1) {
      op.blk_p0 = hp.terms[t1].p0;
      op.blk_tab = hp.terms[t1].tab;
    }
    if (attach)
      for (auto& d : pend_tab) hp.terms.push_back(d);
    const size_t t3 = hp.terms.size();
    if (t1 - t0 > 0xFFFF || t2 - t1 > 0xFFFF || t3 - t2 > 0xFFFF || t3 > 0x7FFFFFFF) overflow = true;
    op.n_sign = (uint16_t)(t1 - t0);
    op.n_phase = (uint16_t)(t2 - t1);
    op.n_table = (uint16_t)(t3 - t2);
    if (attach) {
      pend_sign.clear();
      pend_tab.clear();
      pend_adj = 0;
    }
    op.mat = -1;
    if (u) {
      op.mat = (int32_t)(hp.mats.size() / 4);
      for (int i = 0; i < 4; ++i) hp.mats.push_back(u[i]);
    }
    hp.ops.push_back(op);
  }

  // The pending one-bit phases as one phase block.  An op on a register bit
  // takes the phases on the stage's register bits (they multiply into h_i; a
  // phase on another bit cannot be needed before a stage that holds its bit
  // in a register, or the pass's final OP_DIAG); the final OP_DIAG
  // (all = true) takes every phase, those on other bits as TERM_PFIX terms.
  // ph0 of every phase is a constant factor: it joins the pending scalar,
  // which only the final OP_DIAG applies (in its K), so each factor is
  // ph1 / ph0 on a set bit (a block folds the scalar in early once it falls
  // below 2^-24 in magnitude).  The block's 32 entries are the factors of the
  // 32 register slots, T[j] = K prod_{i: bit i of j set} h_i, so each
  // amplitude takes one complex product; its p0 has bit 0 set unless
  // T[0] = 1 (a product the complex128 kernel skips).
  // Whether attach_phase_block(all) emits a block.
  bool will_attach_block(bool all) const {
    const bool fold = all || std::norm(pend_const) < 0x1p-48;
    const uint64_t take = all ? ph_mask : (ph_mask & reg_mask);
    return take || (fold && pend_const != cd(1.0));
  }

  // `signs`: pairs (i0, i1) of register indices whose sign (-1)^(j_i0 j_i1)
  // (with i0 = i1: (-1)^(j_i0)) multiplies entry j; only passed when a block
  // is emitted.
  void attach_phase_block(bool all, const std::vector<std::pair<int, int>>& signs) {
    // the deferred scalar is folded in early once it is small, so the
    // amplitudes (which carry its inverse) stay far from FP32 overflow
    const bool fold = all || std::norm(pend_const) < 0x1p-48;
    const uint64_t take = all ? ph_mask : (ph_mask & reg_mask);
    if (!will_attach_block(all)) return;
    ph_mask &= ~take;
    cd h[MAX_REG_BITS];
    for (auto& x : h) x = 1.0;
    std::vector<DTerm> fix;
    for (uint64_t rest = take; rest; rest &= rest - 1) {
      const int p = __builtin_ctzll(rest);
      pend_const *= ph0[p];
      const cd r = ph1[p] / ph0[p];
      if (reg_index[p] >= 0) {
        h[reg_index[p]] *= r;
      } else if (r != cd(1.0)) {
        const cd tab[4] = {r, 0.0, 0.0, 0.0};
        DTerm t{};
        t.kind = TERM_PFIX;
        t.p0 = (uint8_t)p;
        t.p1 = (uint8_t)p;
        t.tab = add_table(tab);
        fix.push_back(t);
      }
    }
    cd K = 1.0;
    if (fold) {
      K = pend_const;
      pend_const = 1.0;
    }
    // T[j] = K prod_{i in j} h_i, multiplied in ascending i: entry j is
    // entry (j without its highest bit) times h of that bit
    cd T[32];
    cd P[32];
    P[0] = K;
    for (int j = 1; j < 32; ++j) {
      const int top = 31 - __builtin_clz((unsigned)j);
      P[j] = P[j ^ (1 << top)] * h[top];
    }
    // entry j is negated once for each sign pair whose two bits are both set
    // in j: bit j of slot_bit[i] is bit i of j
    static constexpr uint32_t slot_bit[MAX_REG_BITS] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u,
                                                        0xFF00FF00u, 0xFFFF0000u};
    uint32_t neg = 0;
    for (const auto& pr : signs) neg ^= slot_bit[pr.first] & slot_bit[pr.second];
    for (int j = 0; j < 32; ++j) T[j] = ((neg >> j) & 1u) ? -P[j] : P[j];
    DTerm b{};
    b.kind = TERM_PBLOCK;
    b.p0 = (uint8_t)(K != cd(1.0) ? 1 : 0);
    b.tab = (int)(hp.tabs.size() / 4);  // the 32 entries as 8 consecutive tables
    hp.tabs.insert(hp.tabs.end(), T, T + 32);
    hp.terms.push_back(b);
    for (auto& d : fix) hp.terms.push_back(d);
  }

  bool pending_terms() const {
    return pend_adj || !pend_sign.empty() || !pend_tab.empty() || pend_const != cd(1.0) ||
           ph_mask != 0;
  }

  void flush(int j) {
    if (!pend_has[j]) return;
    if (rot) {
      flush_all();
      return;
    }
    pend_has[j] = false;
    const cd* u = pend_u[j];
    if (is_zero(u[1]) && is_zero(u[2])) {
      add_diag1(j, u[0], u[3]);
    } else {
      emit(OP_DENSE, reg_of[j], u, vpos[j]);
    }
  }

  // Rotation engine: every open matrix at once.  The D_R phases of all of
  // them are pending before the first rotation, which carries them (and
  // whatever else is pending) as one phase block; the D_L phases and the
  // scalars stay pending after the rotations.  Flushing a matrix early is
  // always valid: it holds every gate so far on its qubit.
  void flush_all() {
    int n = 0;
    for (int j = 0; j < nq; ++j) {
      if (!pend_has[j]) continue;
      pend_has[j] = false;
      const cd* u = pend_u[j];
      if (is_zero(u[1]) && is_zero(u[2])) {
        add_diag1(j, u[0], u[3]);
        continue;
      }
      EulerSplit e;
      if (!euler_split(u, e)) {
        emit(OP_DENSE, reg_of[j], u, vpos[j]);
        continue;
      }
      js[n] = j;
      es[n++] = e;
    }
    for (int i = 0; i < n; ++i) add_diag1(js[i], es[i].dr0, es[i].dr1);
    if (n == 1) {
      const cd m[4] = {es[0].t, 0.0, 0.0, 0.0};
      emit(es[0].rot, reg_of[js[0]], m, vpos[js[0]]);
    } else if (n > 1) {
      // every rotation of the flush in one op: tangent of register bit i in
      // real slot i of the op's matrix
      double tr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      uint8_t bits = 0, cot = 0;
      uint64_t vps = 0;
      for (int i = 0; i < n; ++i) {
        const int r = reg_of[js[i]];
        bits |= (uint8_t)(1u << r);
        if (es[i].rot == OP_ROTC) cot |= (uint8_t)(1u << r);
        tr[r] = es[i].t;
        vps |= 1ull << vpos[js[i]];
      }
      const cd m[4] = {cd(tr[0], tr[1]), cd(tr[2], tr[3]), cd(tr[4], tr[5]), cd(tr[6], tr[7])};
      emit(OP_ROTS, bits, m, vpos[js[0]], cot, vps);
    }
    for (int i = 0; i < n; ++i) {
      add_diag1(js[i], es[i].dl0, es[i].dl1);
      pend_const *= es[i].g;
    }
  }

  void add(const Item& it) {
    switch (it.kind) {
      case IT_DENSE:
      case IT_DIAG1: {
        cd m[4];
        const cd* u = it.u;
        if (it.u3) {
          u3_matrix(it.ang, m);
          u = m;
        }
        if (!pend_has[it.a]) {
          pend_has[it.a] = true;
          std::memcpy(pend_u[it.a], u, sizeof(it.u));
        } else {
          mat_lmul(u, pend_u[it.a]);
        }
        return;
      }
      case IT_CZ:
        flush(it.a);
        flush(it.b);
        add_sign(vpos[it.a], vpos[it.b]);
        return;
      case IT_DIAG2: {
        flush(it.a);
        flush(it.b);
        DTerm t{};
        t.kind = TERM_TABLE;
        t.p0 = (uint8_t)vpos[it.a];
        t.p1 = (uint8_t)vpos[it.b];
        cd tab[4] = {it.d[0][0], it.d[0][1], it.d[1][0], it.d[1][1]};  // x_a + 2 x_b
        t.tab = add_table(tab);
        pend_tab.push_back(t);
        return;
      }
      case IT_VAR: {
        flush(it.a);
        if (it.var_sign) {
          add_sign(vpos[it.a], vpos[it.b]);
        } else {
          DTerm t{};
          t.p0 = (uint8_t)vpos[it.a];
          t.p1 = (uint8_t)vpos[it.b];
          cd tab[4] = {it.d[0][0], it.d[0][1], it.d[1][0], it.d[1][1]};  // x + 2b
          t.kind = TERM_TABLE;
          t.tab = add_table(tab);
          pend_tab.push_back(t);
        }
        return;
      }
    }
  }

  // Start a stage whose register bits are the tile bits of `qubits`.
  void begin_stage(const std::vector<int>& qubits, DStage& st) {
    for (int j = 0; j < 64; ++j) {
      reg_of[j] = -1;
      reg_index[j] = -1;
    }
    std::vector<int> pos;
    for (int j : qubits) pos.push_back(vpos[j]);
    std::sort(pos.begin(), pos.end());
    reg_mask = 0;
    for (size_t i = 0; i < pos.size(); ++i) {
      reg_index[pos[i]] = (int)i;
      reg_mask |= 1ull << pos[i];
    }
    for (int i = 0; i < 8; ++i) st.rb[i] = (int8_t)(i < (int)pos.size() ? pos[i] : 0);
    for (int j : qubits)
      for (size_t i = 0; i < pos.size(); ++i)
        if (pos[i] == vpos[j]) reg_of[j] = (int)i;
    st.op_begin = (int32_t)hp.ops.size();
  }

  // End a stage: every open matrix is emitted; diagonal factors may stay
  // pending into the next stage of the same pass.
  void end_stage(DStage& st, bool last) {
    if (rot) flush_all();
    for (int j = 0; j < nq; ++j) flush(j);
    if (last && pending_terms()) emit(OP_DIAG, 0, nullptr, -1);
    st.op_end = (int32_t)hp.ops.size();
  }
};

void add_pass(HostProgram& hp, const std::vector<Item>& items, const std::vector<ItemBits>& bits,
              const std::vector<int>& take, const std::vector<int>& tile_bits, bool first,
              int rb_max) {
  DPass P{};
  P.nq = hp.nq;
  P.k = (int)tile_bits.size();
  P.n_rest = P.nq - P.k;
  P.init_zero = first ? 1 : 0;
  int low = 0;
  while (low < P.k && tile_bits[low] == low) ++low;
  P.low = low;
  P.rbits = std::max(1, std::min(rb_max, P.k - 5));
  P.rbits = std::max(P.rbits, P.k - 9);  // at most 512 threads per CTA
  P.rbits = std::min(P.rbits, P.k);
  uint64_t tmask = 0;
  for (int t = 0; t < P.k; ++t) {
    P.tile_bit[t] = (int8_t)tile_bits[t];
    tmask |= 1ull << tile_bits[t];
    if (tile_bits[t] < hp.n_state) P.zero_tile |= 1u << t;
  }
  int r = 0;
  for (int j = 0; j < P.nq; ++j)
    if (!(tmask & (1ull << j))) {
      if (j < hp.n_state) P.zero_rest |= 1ull << r;
      P.rest_bit[r++] = (int8_t)j;
    }

  // Stages: register-bit sets chosen like tiles, one level down.
  P.stage_begin = (int32_t)hp.stages.size();
  PassBuilder pb(hp, hp.nq, tile_bits);
  std::vector<char> done(items.size(), 1);
  for (int i : take) done[i] = 0;
  std::vector<int> rest(take);  // the pass's items not yet in a stage
  size_t left = take.size();
  do {
    const uint64_t regs = choose_set(bits, rest, done, tile_bits, P.rbits, 0);
    std::vector<int> qubits;
    for (int j : tile_bits)
      if (regs & (1ull << j)) qubits.push_back(j);
    std::vector<int> st_items;
    st_items.reserve(rest.size());
    scan(bits, rest, done, regs, st_items);
    DStage st{};
    pb.begin_stage(qubits, st);
    for (int i : st_items) {
      pb.add(items[i]);
      done[i] = 1;
    }
    left -= st_items.size();
    if (st_items.empty() && left > 0) {  // cannot happen: the first pending item always fits
      hp.nq = -1;
      return;
    }
    drop_applied(rest, done);
    pb.end_stage(st, left == 0);
    if (pb.overflow) {
      hp.nq = -1;
      return;
    }
    hp.stages.push_back(st);
  } while (left > 0);
  P.stage_end = (int32_t)hp.stages.size();
  hp.passes.push_back(P);
}

}  // namespace

HostProgram compile_program(const std::vector<Item>& items, int nq, int n_state, int kmax,
                            int low, int rb_max) {
  HostProgram hp;
  hp.nq = nq;
  hp.n_state = n_state;
  // rough upper bounds (an op per item, a phase block per op), so the
  // vectors do not grow step by step
  hp.ops.reserve(items.size() + 16);
  hp.mats.reserve(4 * items.size() + 64);
  hp.terms.reserve(2 * items.size() + 64);
  hp.tabs.reserve(8 * items.size() + 256);
  const std::vector<ItemBits> bits = item_bits(items);
  std::vector<char> applied(items.size(), 0);
  std::vector<int> order(items.size());  // the items not yet in a pass, in order
  for (size_t i = 0; i < items.size(); ++i) order[i] = (int)i;
  std::vector<int> all_bits(nq);
  for (int j = 0; j < nq; ++j) all_bits[j] = j;
  if (nq <= kmax) {
    add_pass(hp, items, bits, order, all_bits, true, rb_max);
    if (hp.nq > 0) hp.passes.back().flags |= PASS_LAST;
    return hp;
  }
  low = std::min(low, kmax);
  std::vector<int> pool;
  for (int j = low; j < nq; ++j) pool.push_back(j);
  const uint64_t fixed = (low >= 64) ? ~0ull : ((1ull << low) - 1);
  size_t left = items.size();
  bool first = true;
  while (left > 0 || first) {
    const uint64_t tile = choose_set(bits, order, applied, pool, kmax - low, fixed);
    std::vector<int> tile_bits;
    for (int j = 0; j < nq; ++j)
      if (tile & (1ull << j)) tile_bits.push_back(j);
    std::vector<int> take;
    take.reserve(order.size());
    scan(bits, order, applied, tile, take);
    if (take.empty() && left > 0) {  // cannot happen: the first pending item always fits
      hp.nq = -1;
      return hp;
    }
    for (int i : take) applied[i] = 1;
    drop_applied(order, applied);
    left -= take.size();
    add_pass(hp, items, bits, take, tile_bits, first, rb_max);
    if (hp.nq < 0) return hp;
    first = false;
  }
  hp.passes.back().flags |= PASS_LAST;
  return hp;
}

}  // namespace cc
