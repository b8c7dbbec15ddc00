// Batched cut simulation of many independent circuits.
//
// The paper runs the subcircuits of a circuit one after another and names
// their parallel execution as a way to lower the effective threshold
// (Sec. VI).  Here every circuit is planned as usual (Algorithm 1), and the
// passes of all segment programs of all circuits go into one persistent
// launch whose queue holds one item per (pass, tile), ordered by pass number;
// each pass waits (bounded) for the pass before it on the same segment.  The
// merges (Algorithm 3) of all circuits then run as one launch per chain
// level.  The sequence can be captured into one CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "plan.h"

using namespace cc;

namespace {

int amp_bytes(int precision) { return precision == CC_C128 ? 16 : 8; }
uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct PlanDeleter {
  void operator()(cc_plan* p) const { cc_plan_destroy(p); }
};
using PlanPtr = std::unique_ptr<cc_plan, PlanDeleter>;

// Everything that depends on the tile width and the merge tile shape.
struct Core {
  int tile_bits = 0, merge_rows = 32;
  int arith = 0;  // gate-pass arithmetic of the plans' device images
  std::vector<PlanPtr> plans;
  void* arena = nullptr;
  const BJob* jobs = nullptr;
  const BMergeJob* mjobs = nullptr;
  void* state = nullptr;  // zeroed before every run: done[n_jobs], circ_done[n_circ], head
  size_t state_bytes = 0;
  int* done = nullptr;
  int* circ_done = nullptr;
  unsigned long long* head = nullptr;
  int n_jobs = 0;
  int64_t n_items = 0;
  std::vector<int> level_begin;      // merge jobs of level L: [level_begin[L], level_begin[L+1])
  std::vector<int64_t> level_units;  // units of level L
  // Final stages run on the tensor cores (3xTF32) instead, one launch each
  // after their level's batched launch, sharing one split-operand workspace.
  struct TcJob {
    int level, circ;
    BMergeJob j;
  };
  std::vector<TcJob> tc_jobs;
  int block = 32, grid = 1;
  size_t smem = 0;
  ~Core() {
    if (arena) device_free(arena);
  }
};

}  // namespace

struct cc_batch {
  int n_circ = 0, precision = 0, decomp = 0;
  std::vector<cc_gate> gates;
  std::vector<int64_t> gate_off;
  std::vector<int> q, seg_sizes, seg_off;
  // Buffer layout (amplitudes), the same for every tile width.
  std::vector<uint64_t> seg_base, psi_base, work_base;
  uint64_t seg_amps = 0, psi_amps = 0, work_amps = 0;
  uint64_t tc_off = 0, tc_bytes = 0;  // tensor-core workspace inside the workspace (bytes)
  bool tc_ok = true;                  // CUTSIM_BATCH_TC=0: every merge on CUDA cores
  int64_t n_sub = 0;
  std::vector<int> c_total;
  std::unique_ptr<Core> core;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
  ~cc_batch() { drop_graph(); }
};

namespace {

// Plan every circuit with the given segment tile and build the launch tables.
cc_status build_core(cc_batch* b, int tile_bits, int merge_rows, std::unique_ptr<Core>& out) {
  std::unique_ptr<Core> c(new Core());
  c->tile_bits = tile_bits;
  c->merge_rows = merge_rows;
  const int ab = amp_bytes(b->precision);
  for (int i = 0; i < b->n_circ; ++i) {
    cc_plan* p = nullptr;
    const int ns = b->seg_off[i + 1] - b->seg_off[i];
    const cc_status st = create_plan(b->gates.data() + b->gate_off[i],
                                     (int)(b->gate_off[i + 1] - b->gate_off[i]), b->q[i],
                                     b->seg_sizes.data() + b->seg_off[i], ns, b->decomp,
                                     b->precision, tile_bits, &p);
    if (st != CC_OK) {
      set_error("circuit " + std::to_string(i) + ": " + cc_last_error());
      return st;
    }
    c->plans.emplace_back(p);
  }
  c->arith = c->plans.empty() ? gate_arith(b->precision) : c->plans[0]->arith;

  if (b->seg_base.empty()) {  // buffer layout: the same for every tile width
    uint64_t so = 0, po = 0, wo = 0;
    for (int i = 0; i < b->n_circ; ++i) {
      const cc_plan* p = c->plans[i].get();
      b->seg_base.push_back(so);
      b->psi_base.push_back(po);
      b->work_base.push_back(wo);
      so = round_up(so + p->seg_buf_bytes / ab, 32);
      po = round_up(po + p->psi_bytes / ab, 32);
      wo = round_up(wo + 2 * p->chain_ws_amps, 32);
      b->n_sub += p->n_sub;
      b->c_total.push_back(p->c_total);
    }
    b->seg_amps = so;
    b->psi_amps = po;
    // the shared tensor-core workspace follows the chain intermediates
    uint64_t tcb = 0;
    if (b->tc_ok && b->precision == CC_C64)
      for (int i = 0; i < b->n_circ; ++i) {
        const cc_plan* p = c->plans[i].get();
        if (p->stages.empty()) continue;
        const auto& sg = p->stages.back();
        if (sg.K >= kAutoTcMinTerms && sg.qa >= 7 && sg.qb >= 7 && sg.Z == 1)
          tcb = std::max(tcb, merge_tc_workspace_bytes(sg.qa, sg.qb, sg.K, kAutoTcForm));
      }
    b->tc_off = wo * ab;
    b->tc_bytes = tcb;
    b->work_amps = wo + (tcb + ab - 1) / ab;
  }

  // Segment jobs, ordered by pass number (then circuit, then segment).
  struct Ref {
    int circ, seg, pass;
  };
  std::vector<Ref> refs;
  int max_pass = 0;
  for (int i = 0; i < b->n_circ; ++i)
    for (int s = 0; s < c->plans[i]->n_seg; ++s)
      max_pass = std::max(max_pass, (int)c->plans[i]->dprog[s].passes.size());
  std::vector<std::vector<std::vector<int>>> job_of(b->n_circ);
  for (int i = 0; i < b->n_circ; ++i) {
    job_of[i].resize(c->plans[i]->n_seg);
    for (int s = 0; s < c->plans[i]->n_seg; ++s)
      job_of[i][s].assign(c->plans[i]->dprog[s].passes.size(), -1);
  }
  for (int pi = 0; pi < max_pass; ++pi)
    for (int i = 0; i < b->n_circ; ++i)
      for (int s = 0; s < c->plans[i]->n_seg; ++s)
        if (pi < (int)c->plans[i]->dprog[s].passes.size()) {
          job_of[i][s][pi] = (int)refs.size();
          refs.push_back({i, s, pi});
        }
  std::vector<BJob> jobs(refs.size());
  int64_t items = 0;
  int block = 32, kmax = 0;
  for (size_t j = 0; j < refs.size(); ++j) {
    const Ref& r = refs[j];
    const cc_plan* p = c->plans[r.circ].get();
    const DeviceProgram& dp = p->dprog[r.seg];
    const DPass& P = dp.passes[r.pass];
    BJob& J = jobs[j];
    J.vec_off = (int64_t)(b->seg_base[r.circ] + p->seg_off[r.seg]);
    J.pass = reinterpret_cast<const DPass*>(static_cast<const char*>(dp.passes_dev) +
                                            sizeof(DPass) * r.pass);
    J.stages = dp.stages;
    J.ops = dp.ops;
    J.terms = dp.terms;
    J.mats = dp.mats;
    J.tabs = dp.tabs;
    J.tile_begin = items;
    J.n_tiles = int64_t(1) << (P.nq - P.k);
    J.dep = r.pass > 0 ? job_of[r.circ][r.seg][r.pass - 1] : -1;
    J.pad = 0;
    items += J.n_tiles;
    block = std::max(block, 1 << (P.k - P.rbits));
    kmax = std::max(kmax, P.k);
  }
  c->n_jobs = (int)jobs.size();
  c->n_items = items;
  c->block = block;
  c->smem = (size_t)ab << kmax;

  // Merge jobs, one launch per chain level.
  std::vector<BMergeJob> mj;
  int max_stage = 0;
  for (int i = 0; i < b->n_circ; ++i) max_stage = std::max(max_stage, (int)c->plans[i]->stages.size());
  for (int L = 0; L < max_stage; ++L) {
    c->level_begin.push_back((int)mj.size());
    int64_t units = 0;
    for (int i = 0; i < b->n_circ; ++i) {
      const cc_plan* p = c->plans[i].get();
      if (L >= (int)p->stages.size()) continue;
      const auto& sg = p->stages[L];
      const bool last = L + 1 == (int)p->stages.size();
      BMergeJob J;
      std::memset(&J, 0, sizeof(J));
      if (L == 0) {
        J.a_buf = BUF_SEG;
        J.a_off = (int64_t)(b->seg_base[i] + p->seg_off[0]);
      } else {
        J.a_buf = BUF_WORK;
        J.a_off = (int64_t)(b->work_base[i] + ((L - 1) & 1) * p->chain_ws_amps);
      }
      J.b_buf = BUF_SEG;
      J.b_off = (int64_t)(b->seg_base[i] + p->seg_off[sg.seg]);
      if (last) {
        J.out_buf = BUF_PSI;
        J.out_off = (int64_t)b->psi_base[i];
      } else {
        J.out_buf = BUF_WORK;
        J.out_off = (int64_t)(b->work_base[i] + (L & 1) * p->chain_ws_amps);
      }
      J.qa = sg.qa;
      J.qb = sg.qb;
      J.K = sg.K;
      J.Z = sg.Z;
      J.out_stride = int64_t(1) << (sg.qa + sg.qb);
      const int32_t* tabs = static_cast<const int32_t*>(p->tables_dev);
      J.aidx = tabs + sg.aidx_off;
      J.bidx = tabs + sg.bidx_off;
      if (last && b->tc_ok && b->precision == CC_C64 && sg.K >= kAutoTcMinTerms && sg.qa >= 7 && sg.qb >= 7 &&
          sg.Z == 1) {
        J.circ = i;
        c->tc_jobs.push_back({L, i, J});
        continue;
      }
      J.unit_begin = units;
      J.n_units = merge_batch_units(b->precision, sg.qa, sg.qb, sg.Z, merge_rows, &J.kind);
      J.circ = last ? i : -1;
      units += J.n_units;
      mj.push_back(J);
    }
    c->level_units.push_back(units);
  }
  c->level_begin.push_back((int)mj.size());

  // One allocation: job tables, then the per-run state.
  const size_t o_jobs = 0;
  const size_t o_mjobs = round_up(o_jobs + jobs.size() * sizeof(BJob), 256);
  const size_t o_state = round_up(o_mjobs + mj.size() * sizeof(BMergeJob), 256);
  const size_t n_done = jobs.size(), n_circ_done = (size_t)b->n_circ;
  const size_t o_head = round_up(o_state + (n_done + n_circ_done) * sizeof(int), 16);
  const size_t total = o_head + sizeof(unsigned long long);
  std::vector<unsigned char> img(total, 0);
  if (!jobs.empty()) std::memcpy(img.data() + o_jobs, jobs.data(), jobs.size() * sizeof(BJob));
  if (!mj.empty()) std::memcpy(img.data() + o_mjobs, mj.data(), mj.size() * sizeof(BMergeJob));
  c->arena = device_alloc_copy(img.data(), img.size());
  if (!c->arena) return fail(CC_ENOMEM, "device allocation of the batch tables failed");
  unsigned char* d = static_cast<unsigned char*>(c->arena);
  c->jobs = reinterpret_cast<const BJob*>(d + o_jobs);
  c->mjobs = reinterpret_cast<const BMergeJob*>(d + o_mjobs);
  c->state = d + o_state;
  c->state_bytes = total - o_state;
  c->done = reinterpret_cast<int*>(d + o_state);
  c->circ_done = c->done + n_done;
  c->head = reinterpret_cast<unsigned long long*>(d + o_head);

  const int occ = batch_segments_occupancy(c->arith, c->block, c->smem);
  if (occ < 1) return fail(CC_ECUDA, "the batched gate-pass kernel does not fit on an SM");
  c->grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)num_sms() * occ));
  if (!device_error_flag()) return fail(CC_ENOMEM, "device error flag allocation failed");
  out = std::move(c);
  return CC_OK;
}

cc_status check_buffers(const cc_batch* b, const void* seg, uint64_t seg_bytes, const void* psi,
                        uint64_t psi_bytes, const void* work, uint64_t work_bytes) {
  const int ab = amp_bytes(b->precision);
  if (!seg || !psi) return fail(CC_EINVAL, "NULL buffer");
  if (!aligned16(seg) || !aligned16(psi) || (work && !aligned16(work)))
    return fail(CC_EINVAL, "buffers must be 16-byte aligned");
  if (seg_bytes < b->seg_amps * ab) return fail(CC_EBUFSIZE, "seg_buf too small for the batch");
  if (psi_bytes < b->psi_amps * ab) return fail(CC_EBUFSIZE, "psi too small for the batch");
  if (b->work_amps && (!work || work_bytes < b->work_amps * ab))
    return fail(CC_EBUFSIZE, "workspace too small for the batch");
  return CC_OK;
}

cc_status run_core(const cc_batch* b, const Core& c, void* seg, void* psi, void* work,
                   uint64_t* stamps, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(c.state, 0, c.state_bytes, s);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("memset: ") + cudaGetErrorString(e));
  unsigned long long* st = reinterpret_cast<unsigned long long*>(stamps);
  cc_status r = launch_batch_segments(seg, c.jobs, c.n_jobs, c.n_items, c.done, c.head, st,
                                      c.arith, c.block, c.smem, c.grid, stream);
  if (r != CC_OK) return r;
  const int ab = amp_bytes(b->precision);
  char* const bufs[3] = {static_cast<char*>(seg), static_cast<char*>(work), static_cast<char*>(psi)};
  for (size_t L = 0; L + 1 < c.level_begin.size(); ++L) {
    const int j0 = c.level_begin[L], j1 = c.level_begin[L + 1];
    r = launch_merge_batch(c.mjobs + j0, j1 - j0, c.level_units[L], seg, work, psi, c.circ_done,
                           st, b->precision, c.merge_rows, stream);
    if (r != CC_OK) return r;
    for (const auto& t : c.tc_jobs) {
      if (t.level != (int)L) continue;
      const BMergeJob& J = t.j;
      MergeStage ms{bufs[J.a_buf] + J.a_off * ab, bufs[J.b_buf] + J.b_off * ab,
                    bufs[J.out_buf] + J.out_off * ab, J.qa, J.qb, J.K, 1, J.out_stride, J.aidx,
                    J.bidx};
      r = launch_merge_tc(ms, kAutoTcForm, static_cast<char*>(work) + b->tc_off, b->tc_bytes,
                          stream);
      if (r == CC_EUNSUPPORTED) r = launch_merge_fma(ms, b->precision, stream);
      if (r != CC_OK) return r;
      if (st) {
        r = launch_stamp(st + 1 + t.circ, stream);
        if (r != CC_OK) return r;
      }
    }
  }
  return CC_OK;
}

int default_tile_bits(int precision) { return seg_tile_bits(precision); }

}  // namespace

extern "C" cc_status cc_batch_create(const cc_gate* gates, const int64_t* gate_offset,
                                     int32_t n_circ, const int32_t* q, const int32_t* seg_sizes,
                                     const int32_t* seg_offset, int32_t decomp, int32_t precision,
                                     int32_t tile_bits, int32_t merge_rows, cc_batch** out) {
  try {
    if (!out) return fail(CC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_circ < 1 || n_circ > 65536) return fail(CC_ERANGE, "n_circ must be in 1..65536");
    if (!gate_offset || !q || !seg_sizes || !seg_offset) return fail(CC_EINVAL, "NULL array");
    if (precision != CC_C64 && precision != CC_C128) return fail(CC_EINVAL, "unknown precision");
    if (decomp != CC_DECOMP_PROJECTOR && decomp != CC_DECOMP_S_SDG)
      return fail(CC_EINVAL, "unknown decomposition");
    if (tile_bits != 0 &&
        (tile_bits < low_tile_bits(precision) + 1 || tile_bits > max_tile_bits(precision)))
      return fail(CC_ERANGE, "tile_bits outside the range of the precision");
    if (merge_rows == 0) merge_rows = 32;
    if (merge_rows != 16 && merge_rows != 32) return fail(CC_EINVAL, "merge_rows must be 16 or 32");
    if (precision == CC_C128) merge_rows = 32;
    if (gate_offset[0] != 0 || seg_offset[0] != 0)
      return fail(CC_EINVAL, "offsets must start at 0");
    for (int i = 0; i < n_circ; ++i) {
      if (gate_offset[i + 1] < gate_offset[i] || seg_offset[i + 1] < seg_offset[i])
        return fail(CC_EINVAL, "offsets must not decrease");
      if (seg_offset[i + 1] - seg_offset[i] < 2)
        return fail(CC_EINVAL, "circuit " + std::to_string(i) + " has fewer than 2 segments");
      if (gate_offset[i + 1] - gate_offset[i] > (int64_t(1) << 30))
        return fail(CC_ERANGE, "too many gates in circuit " + std::to_string(i));
    }
    if (gate_offset[n_circ] > 0 && !gates) return fail(CC_EINVAL, "gates is NULL");

    std::unique_ptr<cc_batch> b(new cc_batch());
    b->n_circ = n_circ;
    b->precision = precision;
    b->decomp = decomp;
    b->gates.assign(gates, gates + gate_offset[n_circ]);
    b->gate_off.assign(gate_offset, gate_offset + n_circ + 1);
    b->q.assign(q, q + n_circ);
    b->seg_off.assign(seg_offset, seg_offset + n_circ + 1);
    b->seg_sizes.assign(seg_sizes, seg_sizes + seg_offset[n_circ]);
    if (const char* e = std::getenv("CUTSIM_BATCH_TC")) b->tc_ok = e[0] != '0';

    // Host checks of every circuit before any device work.
    for (int i = 0; i < n_circ; ++i) {
      if (q[i] < 1 || q[i] > CC_MAX_QUBITS)
        return fail(CC_ERANGE, "circuit " + std::to_string(i) + ": q out of range");
      int sum = 0;
      for (int k = seg_offset[i]; k < seg_offset[i + 1]; ++k) sum += seg_sizes[k];
      if (sum != q[i])
        return fail(CC_EINVAL, "circuit " + std::to_string(i) + ": segment sizes do not sum to q");
      const cc_status cs = check_gates(gates + gate_offset[i],
                                       (int)(gate_offset[i + 1] - gate_offset[i]), q[i]);
      if (cs != CC_OK) {
        set_error("circuit " + std::to_string(i) + ": " + cc_last_error());
        return cs;
      }
    }
    const int kb = tile_bits ? tile_bits : default_tile_bits(precision);
    std::unique_ptr<Core> core;
    cc_status st = build_core(b.get(), kb, merge_rows, core);
    if (st != CC_OK) return st;
    b->core = std::move(core);
    *out = b.release();
    return CC_OK;
  } catch (const std::bad_alloc&) {
    return fail(CC_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(CC_EINVAL, "internal error in cc_batch_create");
  }
}

extern "C" cc_status cc_batch_info(const cc_batch* b, cc_batch_info_t* info) {
  if (!b || !info) return fail(CC_EINVAL, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  const int ab = amp_bytes(b->precision);
  const Core& c = *b->core;
  info->n_circ = b->n_circ;
  info->precision = b->precision;
  info->tile_bits = c.tile_bits;
  info->merge_rows = c.merge_rows;
  info->n_jobs = c.n_jobs;
  info->merge_levels = (int32_t)c.level_units.size();
  info->n_items = c.n_items;
  info->n_sub = b->n_sub;
  info->seg_buf_bytes = b->seg_amps * ab;
  info->psi_bytes = b->psi_amps * ab;
  info->workspace_bytes = b->work_amps * ab;
  info->block = c.block;
  info->grid = c.grid;
  return CC_OK;
}

extern "C" cc_status cc_batch_circuit(const cc_batch* b, int32_t i, int64_t* psi_offset,
                                      int32_t* q, int32_t* c_total, int64_t* n_sub) {
  if (!b) return fail(CC_EINVAL, "batch is NULL");
  if (i < 0 || i >= b->n_circ) return fail(CC_ERANGE, "circuit index out of range");
  if (psi_offset) *psi_offset = (int64_t)b->psi_base[i];
  if (q) *q = b->q[i];
  if (c_total) *c_total = b->c_total[i];
  if (n_sub) *n_sub = b->core->plans[i]->n_sub;
  return CC_OK;
}

extern "C" cc_status cc_batch_run(const cc_batch* b, void* seg_buf, uint64_t seg_bytes, void* psi,
                                  uint64_t psi_bytes, void* workspace, uint64_t ws_bytes,
                                  uint64_t* stamps, void* stream) {
  if (!b) return fail(CC_EINVAL, "batch is NULL");
  cc_status st = check_buffers(b, seg_buf, seg_bytes, psi, psi_bytes, workspace, ws_bytes);
  if (st != CC_OK) return st;
  st = check_device();
  if (st != CC_OK) return st;
  return run_core(b, *b->core, seg_buf, psi, workspace, stamps, stream);
}

extern "C" cc_status cc_batch_capture(cc_batch* b, void* seg_buf, uint64_t seg_bytes, void* psi,
                                      uint64_t psi_bytes, void* workspace, uint64_t ws_bytes,
                                      uint64_t* stamps, void* stream) {
  if (!b) return fail(CC_EINVAL, "batch is NULL");
  if (!stream) return fail(CC_EINVAL, "capture needs a stream other than the legacy NULL stream");
  cc_status st = check_buffers(b, seg_buf, seg_bytes, psi, psi_bytes, workspace, ws_bytes);
  if (st != CC_OK) return st;
  st = check_device();
  if (st != CC_OK) return st;
  b->drop_graph();
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  st = run_core(b, *b->core, seg_buf, psi, workspace, stamps, stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  if (st != CC_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(CC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  b->graph = g;
  b->exec = x;
  return CC_OK;
}

extern "C" cc_status cc_batch_launch(const cc_batch* b, void* stream) {
  if (!b) return fail(CC_EINVAL, "batch is NULL");
  if (!b->exec) return fail(CC_EINVAL, "no captured graph (call cc_batch_capture first)");
  const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

extern "C" cc_status cc_batch_autotune(cc_batch* b, void* seg_buf, uint64_t seg_bytes, void* psi,
                                       uint64_t psi_bytes, void* workspace, uint64_t ws_bytes,
                                       void* stream, int32_t max_out, int32_t* n_out,
                                       int32_t* tile_bits, int32_t* merge_rows, float* ms) {
  try {
    if (!b) return fail(CC_EINVAL, "batch is NULL");
    cc_status st = check_buffers(b, seg_buf, seg_bytes, psi, psi_bytes, workspace, ws_bytes);
    if (st != CC_OK) return st;
    st = check_device();
    if (st != CC_OK) return st;
    b->drop_graph();
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      if (e0) cudaEventDestroy(e0);
      return fail(CC_ECUDA, "event creation failed");
    }
    const int kmax = max_tile_bits(b->precision);
    std::vector<int> rows_c = b->precision == CC_C128 ? std::vector<int>{32} : std::vector<int>{16, 32};
    float best = 0.f;
    std::unique_ptr<Core> best_core;
    int n = 0;
    for (int kb = std::max(10, low_tile_bits(b->precision) + 1); kb <= kmax; ++kb)
      for (int rows : rows_c) {
        std::unique_ptr<Core> c;
        st = build_core(b, kb, rows, c);
        if (st != CC_OK) break;
        st = run_core(b, *c, seg_buf, psi, workspace, nullptr, stream);  // warm-up
        if (st != CC_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && st == CC_OK; ++r)
          st = run_core(b, *c, seg_buf, psi, workspace, nullptr, stream);
        cudaEventRecord(e1, s);
        if (st != CC_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          st = fail(CC_ECUDA, "autotune timing failed");
          break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        t /= 3.f;
        if (n < max_out) {
          if (tile_bits) tile_bits[n] = kb;
          if (merge_rows) merge_rows[n] = rows;
          if (ms) ms[n] = t;
        }
        ++n;
        if (!best_core || t < best) {
          best = t;
          best_core = std::move(c);
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CC_OK) return st;
    if (n_out) *n_out = std::min(n, max_out);
    if (best_core) b->core = std::move(best_core);
    return CC_OK;
  } catch (const std::bad_alloc&) {
    return fail(CC_ENOMEM, "host allocation failed");
  }
}

extern "C" void cc_batch_destroy(cc_batch* b) { delete b; }
