// Preprocessing (Algorithm 1) and the host side of the C ABI.
//
// Algorithm 1 builds one subcircuit per segment and per bit string b of the
// segment's adjacent cuts.  With either rank-2 CZ split the local terms are
// diagonal (projectors / Z^b, or S / S^dag), and a cut CX only adds shared
// Hadamards on its target (CX = (I (x) H) CZ (I (x) H)).  All 2^{c_i} variants
// of segment i therefore share every non-diagonal gate, and the plan keeps a
// single gate program per segment in which each cut term is a diagonal factor
// selected by one bit of the variant number.  The cut's coefficient (1 for
// the projector split, 1/(1+i) and i/(1+i) for Eq. 2) is folded into the term
// on the segment of the gate's first qubit, so the merge sums plain products
// (alpha_m = prod_j coef_j[m_j] is carried by the first factor).
//
// The merge index table M of Algorithm 1 is bit slicing: segment i's variant
// number is r_i(m) = sum_t bit(m, j_t) 2^t over its adjacent cuts j_0 < j_1 <
// ... .  For n >= 3 segments on a line, the merge absorbs one segment at a
// time (see merge stages below), which needs every cut between neighbouring
// segments.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <new>
#include <thread>

#include "internal.h"
#include "plan.h"

using namespace cc;

namespace {

int amp_bytes(int precision) { return precision == CC_C128 ? 16 : 8; }

int seg_of_qubit(const cc_plan* p, int qb) {
  for (int i = 0; i < p->n_seg; ++i)
    if (qb >= p->seg_start[i] && qb < p->seg_start[i] + p->seg_q[i]) return i;
  return -1;
}

// Local term of cut j on one side, as a variant-selected diagonal factor.
Item cut_item(int decomp, bool first_side, int local_qubit, int slot, int seg_qubits) {
  Item it;
  it.kind = IT_VAR;
  it.a = local_qubit;
  it.slot = slot;
  it.b = seg_qubits + slot;  // the variant bit sits above the segment's qubits
  const cd I(0.0, 1.0);
  if (decomp == CC_DECOMP_PROJECTOR) {
    if (first_side) {  // |b><b|, coefficient 1
      it.d[0][0] = 1.0; it.d[0][1] = 0.0;
      it.d[1][0] = 0.0; it.d[1][1] = 1.0;
    } else {           // Z^b
      it.var_sign = true;
    }
  } else {             // Eq. 2: S for b = 0, S^dag for b = 1
    cd coef[2] = {1.0, 1.0};
    if (first_side) {
      coef[0] = 1.0 / (1.0 + I);
      coef[1] = I / (1.0 + I);
    }
    it.d[0][0] = coef[0]; it.d[0][1] = coef[0] * I;
    it.d[1][0] = coef[1]; it.d[1][1] = -coef[1] * I;
  }
  return it;
}

// Z^v on local qubit a, v the variant bit `slot`: a sign when both are set.
Item var_sign_item(int a, int slot, int seg_qubits) {
  Item it;
  it.kind = IT_VAR;
  it.a = a;
  it.slot = slot;
  it.b = seg_qubits + slot;
  it.var_sign = true;
  return it;
}

Item hadamard(int a) {
  Item h;
  h.kind = IT_DENSE;
  h.a = a;
  const double r = 1.0 / std::sqrt(2.0);
  h.u[0] = r; h.u[1] = r; h.u[2] = r; h.u[3] = -r;
  return h;
}

}  // namespace

cc_plan::~cc_plan() {
  if (arena) device_free(arena);
}

extern "C" cc_status cc_plan_create(const cc_gate* gates, int32_t n_gates, int32_t q,
                                    const int32_t* seg_sizes, int32_t n_seg, int32_t decomp,
                                    int32_t precision, cc_plan** out) {
  return cc::create_plan(gates, n_gates, q, seg_sizes, n_seg, decomp, precision,
                         seg_tile_bits(precision), out);
}

namespace {

// The segment compile threads of one plan: on leaving scope (a failed plan,
// an exception) the threads still waiting are told to leave, and all joined.
struct CompileThreads {
  std::atomic<int>& go;
  std::vector<std::thread> th;
  explicit CompileThreads(std::atomic<int>& g) : go(g) {}
  CompileThreads(const CompileThreads&) = delete;
  CompileThreads& operator=(const CompileThreads&) = delete;
  void join() {
    for (auto& t : th)
      if (t.joinable()) t.join();
  }
  ~CompileThreads() {
    int wait = 0;
    go.compare_exchange_strong(wait, 2);
    join();
  }
};

}  // namespace

cc_status cc::create_plan(const cc_gate* gates, int n_gates, int q, const int* seg_sizes,
                          int n_seg, int decomp, int precision, int seg_kmax, cc_plan** out,
                          bool host_only) {
  try {
    if (!out) return fail(CC_EINVAL, "out is NULL");
    *out = nullptr;
    if (q < 1 || q > CC_MAX_QUBITS) return fail(CC_ERANGE, "q must be in 1..34");
    if (n_seg < 1 || n_seg > CC_MAX_SEGMENTS) return fail(CC_ERANGE, "n_seg must be in 1..8");
    if (!seg_sizes) return fail(CC_EINVAL, "seg_sizes is NULL");
    if (decomp != CC_DECOMP_PROJECTOR && decomp != CC_DECOMP_S_SDG)
      return fail(CC_EINVAL, "unknown decomposition");
    if (precision != CC_C64 && precision != CC_C128) return fail(CC_EINVAL, "unknown precision");
    int sum = 0;
    for (int i = 0; i < n_seg; ++i) {
      if (seg_sizes[i] < 1) return fail(CC_EINVAL, "segment sizes must be positive");
      sum += seg_sizes[i];
    }
    if (sum != q) return fail(CC_EINVAL, "segment sizes do not sum to q");
    cc_status st = check_gates(gates, n_gates, q);
    if (st != CC_OK) return st;

    std::unique_ptr<cc_plan> p(new cc_plan());
    p->q = q;
    p->n_seg = n_seg;
    p->precision = precision;
    p->arith = gate_arith(precision);
    p->decomp = decomp;
    int acc = 0;
    for (int i = 0; i < n_seg; ++i) {
      p->seg_q.push_back(seg_sizes[i]);
      p->seg_start.push_back(acc);
      acc += seg_sizes[i];
    }

    // Scan the circuit for boundary gates (cut j in circuit order).  Each cut
    // adds one or two global bits; seg_cut_ids[i] lists segment i's bits in
    // order, and bit t of its variant number is its t-th entry.
    std::vector<std::vector<Item>> items(n_seg);
    {
      // most gates give one item: size each segment's list once
      std::vector<size_t> n_in(n_seg, 8);
      for (int g = 0; g < n_gates; ++g) ++n_in[seg_of_qubit(p.get(), gates[g].q0)];
      for (int i = 0; i < n_seg; ++i) items[i].reserve(n_in[i]);
    }
    p->seg_cut_ids.assign(n_seg, {});

    // One shared program per segment.  The programs are independent host
    // work, so segments after the first compile on their own threads.  The
    // threads start here, before the items are built, so that their start-up
    // (tens of microseconds) overlaps that work: each waits for `go`, then
    // compiles its segment, or leaves when the plan fails first.  Where a
    // thread cannot be started, its segment compiles on this one.
    std::vector<std::exception_ptr> errs(n_seg);
    std::atomic<int> go{0};  // 0: wait, 1: compile, 2: leave
    auto work = [&](int i) {
      try {
        p->hprog[i] = compile_program(items[i], p->seg_q[i] + p->seg_c[i], p->seg_q[i], seg_kmax,
                                      low_tile_bits(precision), reg_bits_max(precision));
      } catch (...) {
        errs[i] = std::current_exception();
      }
    };
    auto worker = [&](int i) {
      int g;
      while ((g = go.load(std::memory_order_acquire)) == 0) std::this_thread::yield();
      if (g == 1) work(i);
    };
    CompileThreads pool(go);
    std::vector<int> inline_segs;
    for (int i = 1; i < n_seg; ++i) {
      try {
        pool.th.emplace_back(worker, i);
      } catch (...) {
        inline_segs.push_back(i);
      }
    }

    for (int g = 0; g < n_gates; ++g) {
      const cc_gate& gt = gates[g];
      const bool two = is_two_qubit(gt.kind);
      const int s0 = seg_of_qubit(p.get(), gt.q0);
      const int s1 = two ? seg_of_qubit(p.get(), gt.q1) : s0;
      cd w[4];  // rank-4 Pauli weights (II, XX, YY, ZZ)
      bool use_a = false, use_b = false;
      if (s0 != s1 && is_rank4(gt.kind)) {
        pauli_weights(gt, w);
        use_a = w[1] != cd(0.0) || w[2] != cd(0.0);
        use_b = w[3] != cd(0.0) || w[2] != cd(0.0);
      }
      if (s0 == s1 || (is_rank4(gt.kind) && !use_a && !use_b)) {  // (the identity needs no cut)
        st = gate_items(gt, p->seg_start[s0], items[s0]);
        if (st != CC_OK) return st;
        continue;
      }
      const int width = is_rank4(gt.kind) ? (int)use_a + (int)use_b : 1;
      if ((int)p->bits.size() + width > CC_MAX_CUTS)
        return fail(CC_ERANGE, "more than 24 cut bits");
      if (n_seg >= 3 && std::abs(s0 - s1) != 1)
        return fail(CC_EUNSUPPORTED, "gate " + std::to_string(g) +
                                         " crosses non-adjacent segments; the chained merge needs "
                                         "every cut between neighbouring segments");
      const int j = (int)p->cuts.size();
      p->cuts.push_back({gt.q0, gt.q1, gt.kind, s0, s1});
      auto new_bit = [&](int& slot0, int& slot1) {
        slot0 = (int)p->seg_cut_ids[s0].size();
        slot1 = (int)p->seg_cut_ids[s1].size();
        const int bit = (int)p->bits.size();
        p->bits.push_back({j, s0, s1});
        p->seg_cut_ids[s0].push_back(bit);
        p->seg_cut_ids[s1].push_back(bit);
      };
      const int l0 = gt.q0 - p->seg_start[s0], l1 = gt.q1 - p->seg_start[s1];
      if (!is_rank4(gt.kind)) {
        int slot0, slot1;
        new_bit(slot0, slot1);
        items[s0].push_back(cut_item(decomp, true, l0, slot0, p->seg_q[s0]));
        if (gt.kind == CC_GATE_CX) items[s1].push_back(hadamard(l1));
        items[s1].push_back(cut_item(decomp, false, l1, slot1, p->seg_q[s1]));
        if (gt.kind == CC_GATE_CX) items[s1].push_back(hadamard(l1));
        continue;
      }
      // Rank 4: U = sum_{a,b} w_ab (X^a Z^b) (x) (X^a Z^b) with w_00 = c_II,
      // w_10 = c_XX, w_01 = c_ZZ, w_11 = -c_YY (X Z = -i Y, so (XZ)(x)(XZ) = -YY).
      // Both sides apply Z^b, then X^a = H Z^a H; the weight rides on the
      // first side as a table over its two variant bits.
      int a0 = -1, a1 = -1, b0 = -1, b1 = -1;
      if (use_a) new_bit(a0, a1);
      if (use_b) new_bit(b0, b1);
      const int side_seg[2] = {s0, s1}, side_q[2] = {l0, l1};
      const int side_a[2] = {a0, a1}, side_b[2] = {b0, b1};
      for (int side = 0; side < 2; ++side) {
        const int sg = side_seg[side], lq = side_q[side], nq_s = p->seg_q[sg];
        if (use_b) items[sg].push_back(var_sign_item(lq, side_b[side], nq_s));
        if (use_a) {
          items[sg].push_back(hadamard(lq));
          items[sg].push_back(var_sign_item(lq, side_a[side], nq_s));
          items[sg].push_back(hadamard(lq));
        }
      }
      const cd w00 = w[0], w10 = w[1], w01 = w[3], w11 = -w[2];
      Item co;
      co.kind = IT_VAR;
      if (use_a && use_b) {  // d[bit b][bit a]
        co.a = p->seg_q[s0] + a0;
        co.b = p->seg_q[s0] + b0;
        co.d[0][0] = w00; co.d[0][1] = w10; co.d[1][0] = w01; co.d[1][1] = w11;
      } else {  // one bit: the table is read at (bit, bit)
        const int slot = use_a ? a0 : b0;
        co.a = co.b = p->seg_q[s0] + slot;
        co.d[0][0] = w00; co.d[0][1] = 0.0; co.d[1][0] = 0.0; co.d[1][1] = use_a ? w10 : w01;
      }
      co.slot = -1;
      items[s0].push_back(co);
    }
    p->c_total = (int)p->cuts.size();

    const int ab = amp_bytes(precision);
    int64_t off = 0;
    p->n_sub = 0;
    for (int i = 0; i < n_seg; ++i) {
      const int ci = (int)p->seg_cut_ids[i].size();
      p->seg_c.push_back(ci);
      if (p->seg_q[i] + ci > CC_MAX_QUBITS)
        return fail(CC_ERANGE, "segment " + std::to_string(i) + " needs 2^" +
                                   std::to_string(p->seg_q[i] + ci) + " amplitudes");
      p->seg_off.push_back(off);
      off += int64_t(1) << (p->seg_q[i] + ci);
      p->n_sub += int64_t(1) << ci;
    }
    p->seg_buf_bytes = (uint64_t)off * ab;
    p->psi_bytes = (uint64_t(1) << q) * ab;

    // The segment programs (the threads started above take segments 1..n-1).
    p->hprog.resize(n_seg);
    go.store(1, std::memory_order_release);
    work(0);
    for (int i : inline_segs) work(i);
    pool.join();
    for (auto& e : errs)
      if (e) std::rethrow_exception(e);
    for (int i = 0; i < n_seg; ++i)
      if (p->hprog[i].nq < 0) return fail(CC_ERANGE, "pass planner made no progress");

    // Merge stages: stage s absorbs segment s into the product of segments < s.
    //   U_s[z][x_s * N_{<s} + x_{<s}] = sum_k U_{s-1}[k][x_{<s}] * seg_s[r_s(k, z)][x_s]
    // k runs over the cut bits of boundary (s-1, s), z over those of (s, s+1).
    std::vector<int32_t> tab;
    if (n_seg >= 2) {
      std::vector<std::vector<int>> bcuts(n_seg - 1);
      for (int bit = 0; bit < (int)p->bits.size(); ++bit)
        bcuts[std::min(p->bits[bit].s0, p->bits[bit].s1)].push_back(bit);
      int qa = p->seg_q[0];
      uint64_t u_max = 0;
      for (int s = 1; s < n_seg; ++s) {
        cc_plan::Stage sg;
        sg.seg = s;
        sg.qa = qa;
        sg.qb = p->seg_q[s];
        const std::vector<int>& kc = bcuts[s - 1];
        const std::vector<int> none;
        const std::vector<int>& zc = (s + 1 < n_seg) ? bcuts[s] : none;
        sg.K = int64_t(1) << kc.size();
        sg.Z = int64_t(1) << zc.size();
        sg.aidx_off = (int64_t)tab.size();
        for (int64_t z = 0; z < sg.Z; ++z)
          for (int64_t k = 0; k < sg.K; ++k) {
            int32_t ra = (int32_t)k;
            if (s == 1) {  // r_0 from the global combination
              uint64_t m = 0;
              for (size_t t = 0; t < kc.size(); ++t) m |= uint64_t((k >> t) & 1) << kc[t];
              ra = 0;
              for (size_t t = 0; t < p->seg_cut_ids[0].size(); ++t)
                ra |= int32_t((m >> p->seg_cut_ids[0][t]) & 1) << t;
            }
            tab.push_back(ra);
          }
        sg.bidx_off = (int64_t)tab.size();
        for (int64_t z = 0; z < sg.Z; ++z)
          for (int64_t k = 0; k < sg.K; ++k) {
            uint64_t m = 0;
            for (size_t t = 0; t < kc.size(); ++t) m |= uint64_t((k >> t) & 1) << kc[t];
            for (size_t t = 0; t < zc.size(); ++t) m |= uint64_t((z >> t) & 1) << zc[t];
            int32_t rb = 0;
            for (size_t t = 0; t < p->seg_cut_ids[s].size(); ++t)
              rb |= int32_t((m >> p->seg_cut_ids[s][t]) & 1) << t;
            tab.push_back(rb);
          }
        if (s + 1 < n_seg) u_max = std::max(u_max, (uint64_t)sg.Z << (qa + sg.qb));
        qa += sg.qb;
        p->stages.push_back(sg);
      }
      // Workspace: the two chained-merge intermediates (n >= 3), then the split
      // operands of a tensor-core form for the last (2^q-sized) stage.
      p->chain_ws_amps = u_max;
      const auto& last = p->stages.back();
      const uint64_t tc = std::max({merge_tc_workspace_bytes(last.qa, last.qb, last.K, CC_MERGE_TF32X3),
                                    merge_tc_workspace_bytes(last.qa, last.qb, last.K, CC_MERGE_BF16X3),
                                    merge_tc_workspace_bytes(last.qa, last.qb, last.K, CC_MERGE_F16X3)});
      const uint64_t oz = merge_ozaki_workspace_bytes(last.qa, last.qb, last.K);
      p->workspace_bytes = 2 * u_max * ab + (precision == CC_C64 ? tc : oz);
    }
    // All device tables of the plan (gate programs, merge index tables) go up
    // in one allocation and one copy.  Everything above is host work; the
    // device is needed from here on.
    if (host_only) {
      p->host_tables = std::move(tab);
      *out = p.release();
      return CC_OK;
    }
    st = check_device();
    if (st != CC_OK) return st;
    std::vector<unsigned char> img;
    std::vector<ImageLayout> lay;
    for (int i = 0; i < n_seg; ++i) lay.push_back(append_program_image(p->hprog[i], p->arith, img));
    const size_t tab_off = (img.size() + 255) & ~size_t(255);
    img.resize(tab_off + tab.size() * sizeof(int32_t));
    if (!tab.empty()) std::memcpy(img.data() + tab_off, tab.data(), tab.size() * sizeof(int32_t));
    // The segment passes as jobs of one persistent launch (see
    // cc_simulate_segments), then that launch's per-run counters.
    int n_jobs = 0, max_pass = 0;
    for (int i = 0; i < n_seg; ++i) {
      n_jobs += (int)p->hprog[i].passes.size();
      max_pass = std::max(max_pass, (int)p->hprog[i].passes.size());
    }
    const size_t jobs_off = (img.size() + 255) & ~size_t(255);
    const size_t state_off = (jobs_off + n_jobs * sizeof(BJob) + 255) & ~size_t(255);
    const size_t head_off = (state_off + n_jobs * sizeof(int) + 15) & ~size_t(15);
    img.resize(head_off + sizeof(unsigned long long), 0);
    void* arena = nullptr;
    if (cudaMalloc(&arena, img.size()) != cudaSuccess) {
      cudaGetLastError();
      return fail(CC_ENOMEM, "device allocation of the plan tables failed");
    }
    p->arena = arena;
    unsigned char* dev = static_cast<unsigned char*>(p->arena);
    for (int i = 0; i < n_seg; ++i) {
      DeviceProgram dp;
      bind_program(dp, p->hprog[i], dev, lay[i]);
      p->dprog.push_back(dp);
    }
    std::vector<BJob> jobs;
    std::vector<std::vector<int>> job_of(n_seg);
    int64_t n_items = 0;
    int block = 32, kmax = 0;
    for (int pi = 0; pi < max_pass; ++pi)
      for (int i = 0; i < n_seg; ++i) {
        const DeviceProgram& dp = p->dprog[i];
        if (pi >= (int)dp.passes.size()) continue;
        const DPass& P = dp.passes[pi];
        BJob J{};
        J.vec_off = p->seg_off[i];
        J.pass = reinterpret_cast<const DPass*>(static_cast<const char*>(dp.passes_dev) +
                                                sizeof(DPass) * pi);
        J.stages = dp.stages;
        J.ops = dp.ops;
        J.terms = dp.terms;
        J.mats = dp.mats;
        J.tabs = dp.tabs;
        J.tile_begin = n_items;
        J.n_tiles = int64_t(1) << (P.nq - P.k);
        J.dep = pi > 0 ? job_of[i][pi - 1] : -1;
        job_of[i].push_back((int)jobs.size());
        jobs.push_back(J);
        n_items += J.n_tiles;
        block = std::max(block, 1 << (P.k - P.rbits));
        kmax = std::max(kmax, P.k);
      }
    if (!jobs.empty()) std::memcpy(img.data() + jobs_off, jobs.data(), jobs.size() * sizeof(BJob));
    if (cudaMemcpy(arena, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return fail(CC_ECUDA, "upload of the plan tables failed");
    }
    p->seg_jobs = reinterpret_cast<const BJob*>(dev + jobs_off);
    p->seg_state = dev + state_off;
    p->seg_state_bytes = img.size() - state_off;
    p->seg_done = reinterpret_cast<int*>(dev + state_off);
    p->seg_head = reinterpret_cast<unsigned long long*>(dev + head_off);
    p->seg_n_jobs = (int)jobs.size();
    p->seg_n_items = n_items;
    p->seg_block = block;
    p->seg_smem = (size_t)ab << kmax;
    const int occ = batch_segments_occupancy(p->arith, block, p->seg_smem);
    p->seg_grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_items, (int64_t)num_sms() * std::max(occ, 1)));
    if (!device_error_flag()) return fail(CC_ENOMEM, "device error flag allocation failed");
    p->tables_dev = tab.empty() ? nullptr : dev + tab_off;
    p->table_bytes = img.size();
    *out = p.release();
    return CC_OK;
  } catch (const std::bad_alloc&) {
    return fail(CC_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(CC_EINVAL, "internal error in cc_plan_create");
  }
}

extern "C" cc_status cc_plan_info(const cc_plan* p, cc_plan_info_t* info) {
  if (!p || !info) return fail(CC_EINVAL, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->q = p->q;
  info->n_seg = p->n_seg;
  info->c_total = p->c_total;
  info->cut_bits = (int32_t)p->bits.size();
  info->precision = p->precision;
  info->decomp = p->decomp;
  for (int i = 0; i < p->n_seg; ++i) {
    info->seg_qubits[i] = p->seg_q[i];
    info->seg_start[i] = p->seg_start[i];
    info->seg_cuts[i] = p->seg_c[i];
    info->seg_offset[i] = p->seg_off[i];
    info->seg_passes[i] = (int32_t)p->hprog[i].passes.size();
    info->seg_ops[i] = (int32_t)p->hprog[i].ops.size();
  }
  info->n_sub = p->n_sub;
  info->seg_buf_bytes = p->seg_buf_bytes;
  info->psi_bytes = p->psi_bytes;
  info->workspace_bytes = p->workspace_bytes;
  info->table_bytes = p->table_bytes;
  return CC_OK;
}

extern "C" cc_status cc_plan_cut(const cc_plan* p, int32_t j, int32_t* q0, int32_t* q1,
                                 int32_t* kind, int32_t* seg0, int32_t* seg1) {
  if (!p) return fail(CC_EINVAL, "plan is NULL");
  if (j < 0 || j >= p->c_total) return fail(CC_ERANGE, "cut index out of range");
  const auto& c = p->cuts[j];
  if (q0) *q0 = c.q0;
  if (q1) *q1 = c.q1;
  if (kind) *kind = c.kind;
  if (seg0) *seg0 = c.s0;
  if (seg1) *seg1 = c.s1;
  return CC_OK;
}

extern "C" void cc_plan_destroy(cc_plan* p) { delete p; }

// ------------------------------------------------------------------ uncut
cc_uncut::~cc_uncut() { free_program(dprog); }

extern "C" cc_status cc_uncut_create(const cc_gate* gates, int32_t n_gates, int32_t q,
                                     int32_t precision, cc_uncut** out) {
  try {
    if (!out) return fail(CC_EINVAL, "out is NULL");
    *out = nullptr;
    if (q < 1 || q > CC_MAX_QUBITS) return fail(CC_ERANGE, "q must be in 1..34");
    if (precision != CC_C64 && precision != CC_C128) return fail(CC_EINVAL, "unknown precision");
    cc_status st = check_gates(gates, n_gates, q);
    if (st != CC_OK) return st;
    std::unique_ptr<cc_uncut> u(new cc_uncut());
    u->q = q;
    u->precision = precision;
    u->arith = gate_arith(precision);
    std::vector<Item> items;
    items.reserve((size_t)n_gates);
    for (int g = 0; g < n_gates; ++g) {
      st = gate_items(gates[g], 0, items);
      if (st != CC_OK) return st;
    }
    u->hprog = compile_program(items, q, q, uncut_tile_bits(precision), low_tile_bits(precision),
                               reg_bits_max(precision));
    if (u->hprog.nq < 0) return fail(CC_ERANGE, "pass planner made no progress");
    st = check_device();
    if (st != CC_OK) return st;
    st = upload_program(u->hprog, u->arith, u->dprog);
    if (st != CC_OK) return st;
    *out = u.release();
    return CC_OK;
  } catch (const std::bad_alloc&) {
    return fail(CC_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(CC_EINVAL, "internal error in cc_uncut_create");
  }
}

namespace {

// A host program as int64 words and doubles (the layout cc_program_image
// documents).
void serialize_program(const cc::HostProgram& hp, std::vector<int64_t>& w, std::vector<double>& r) {
  using namespace cc;
  w = {1, hp.nq, hp.n_state, (int64_t)hp.passes.size(), (int64_t)hp.stages.size(),
       (int64_t)hp.ops.size(), (int64_t)hp.terms.size(), (int64_t)hp.mats.size(),
       (int64_t)hp.tabs.size()};
  for (const DPass& P : hp.passes) {
    const int64_t f[10] = {P.nq, P.k, P.low, P.init_zero, P.stage_begin, P.stage_end,
                           P.rbits, P.n_rest, (int64_t)P.zero_tile, (int64_t)P.zero_rest};
    w.insert(w.end(), f, f + 10);
    for (int t = 0; t < MAX_TILE_BITS; ++t) w.push_back(P.tile_bit[t]);
    for (int q = 0; q < MAX_REST_BITS; ++q) w.push_back(P.rest_bit[q]);
  }
  for (const DStage& S : hp.stages) {
    w.push_back(S.op_begin);
    w.push_back(S.op_end);
    for (int i = 0; i < 8; ++i) w.push_back(S.rb[i]);
  }
  for (const DOp& o : hp.ops) {
    // OP_ROTS: the t word carries the OP_ROTC mask in bits 8..15
    const int64_t t = o.t | (o.type == OP_ROTS ? (int64_t)o.cot << 8 : 0);
    const int64_t f[8] = {o.type, t, o.term_begin, o.n_sign, o.n_phase, o.n_table, o.mat,
                          (int64_t)o.sign_adj};
    w.insert(w.end(), f, f + 8);
  }
  for (const DTerm& t : hp.terms) {
    w.push_back(t.kind);
    w.push_back(t.p0);
    w.push_back(t.p1);
    w.push_back(t.tab);
  }
  r.clear();
  for (const cd& z : hp.mats) {
    r.push_back(z.real());
    r.push_back(z.imag());
  }
  for (const cd& z : hp.tabs) {
    r.push_back(z.real());
    r.push_back(z.imag());
  }
}

// Copy an image out (or only report its sizes when words or reals is NULL).
cc_status export_image(const std::vector<int64_t>& w, const std::vector<double>& r, int64_t* words,
                       int64_t* n_words, double* reals, int64_t* n_reals) {
  const bool query = !words || !reals;
  const bool fits = !query && *n_words >= (int64_t)w.size() && *n_reals >= (int64_t)r.size();
  *n_words = (int64_t)w.size();
  *n_reals = (int64_t)r.size();
  if (query) return CC_OK;
  if (!fits) return cc::fail(CC_EBUFSIZE, "words or reals too small for the program image");
  std::memcpy(words, w.data(), w.size() * sizeof(int64_t));
  std::memcpy(reals, r.data(), r.size() * sizeof(double));
  return CC_OK;
}

}  // namespace

extern "C" cc_status cc_program_image(const cc_gate* gates, int32_t n_gates, int32_t q,
                                      int32_t precision, int32_t tile_bits, int64_t* words,
                                      int64_t* n_words, double* reals, int64_t* n_reals) {
  try {
    if (!n_words || !n_reals) return fail(CC_EINVAL, "n_words / n_reals is NULL");
    if (q < 1 || q > CC_MAX_QUBITS) return fail(CC_ERANGE, "q must be in 1..34");
    if (precision != CC_C64 && precision != CC_C128) return fail(CC_EINVAL, "unknown precision");
    const int low = low_tile_bits(precision);
    if (tile_bits == 0) tile_bits = uncut_tile_bits(precision);
    if (tile_bits <= low || tile_bits > max_tile_bits(precision))
      return fail(CC_ERANGE, "tile_bits must exceed the contiguous low tile bits and fit shared memory");
    cc_status st = check_gates(gates, n_gates, q);
    if (st != CC_OK) return st;
    std::vector<Item> items;
    items.reserve((size_t)n_gates);
    for (int g = 0; g < n_gates; ++g) {
      st = gate_items(gates[g], 0, items);
      if (st != CC_OK) return st;
    }
    const HostProgram hp = compile_program(items, q, q, tile_bits, low, reg_bits_max(precision));
    if (hp.nq < 0) return fail(CC_ERANGE, "pass planner made no progress");
    std::vector<int64_t> w;
    std::vector<double> r;
    serialize_program(hp, w, r);
    return export_image(w, r, words, n_words, reals, n_reals);
  } catch (const std::bad_alloc&) {
    return fail(CC_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(CC_EINVAL, "internal error in cc_program_image");
  }
}

extern "C" cc_status cc_plan_program_image(const cc_gate* gates, int32_t n_gates, int32_t q,
                                           const int32_t* seg_sizes, int32_t n_seg,
                                           int32_t decomp, int32_t precision, int32_t tile_bits,
                                           int32_t seg, int64_t* words, int64_t* n_words,
                                           double* reals, int64_t* n_reals) {
  try {
    if (!n_words || !n_reals) return fail(CC_EINVAL, "n_words / n_reals is NULL");
    if (precision != CC_C64 && precision != CC_C128) return fail(CC_EINVAL, "unknown precision");
    if (tile_bits == 0) tile_bits = seg_tile_bits(precision);
    if (tile_bits <= low_tile_bits(precision) || tile_bits > max_tile_bits(precision))
      return fail(CC_ERANGE, "tile_bits must exceed the contiguous low tile bits and fit shared memory");
    cc_plan* raw = nullptr;
    const cc_status st = create_plan(gates, n_gates, q, seg_sizes, n_seg, decomp, precision,
                                     tile_bits, &raw, true);
    if (st != CC_OK) return st;
    std::unique_ptr<cc_plan> p(raw);
    if (seg < 0 || seg >= p->n_seg) return fail(CC_ERANGE, "segment index out of range");
    std::vector<int64_t> w;
    std::vector<double> r;
    serialize_program(p->hprog[seg], w, r);
    w.push_back((int64_t)p->bits.size());
    w.push_back((int64_t)p->seg_cut_ids[seg].size());
    for (int b : p->seg_cut_ids[seg]) w.push_back(b);
    // the merge stages and their index tables
    w.push_back((int64_t)p->stages.size());
    for (const auto& sg : p->stages) {
      const int64_t f[7] = {sg.seg, sg.qa, sg.qb, sg.K, sg.Z, sg.aidx_off, sg.bidx_off};
      w.insert(w.end(), f, f + 7);
    }
    w.push_back((int64_t)p->host_tables.size());
    for (int32_t v : p->host_tables) w.push_back(v);
    return export_image(w, r, words, n_words, reals, n_reals);
  } catch (const std::bad_alloc&) {
    return fail(CC_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(CC_EINVAL, "internal error in cc_plan_program_image");
  }
}

extern "C" cc_status cc_uncut_info(const cc_uncut* u, int32_t* n_passes, int32_t* n_ops,
                                   int32_t* tile_bits) {
  if (!u) return fail(CC_EINVAL, "NULL argument");
  if (n_passes) *n_passes = (int32_t)u->hprog.passes.size();
  if (n_ops) *n_ops = (int32_t)u->hprog.ops.size();
  if (tile_bits) *tile_bits = u->hprog.passes.empty() ? 0 : u->hprog.passes[0].k;
  return CC_OK;
}

extern "C" void cc_uncut_destroy(cc_uncut* u) { delete u; }
