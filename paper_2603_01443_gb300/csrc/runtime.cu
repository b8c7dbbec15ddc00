// Device runtime and the device-side C ABI entry points: errors, device
// checks, library scratch, program upload, and the launches behind
// cc_simulate_segments, cc_merge, cc_simulate_uncut, cc_compare, cc_gather.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "plan.h"

namespace cc {

namespace {
thread_local std::string g_error = "no error";

struct DeviceState {
  bool checked = false;
  cc_status status = CC_OK;
  int sms = 0;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  int* err_flag = nullptr;
};
std::mutex g_mu;
DeviceState g_dev[64];

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return -1;
  return d;
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
}  // namespace

void set_error(const std::string& msg) { g_error = msg; }

cc_status fail(cc_status s, const std::string& msg) {
  g_error = msg;
  return s;
}

cc_status check_device() {
  const int d = current_device();
  if (d < 0 || d >= 64) return fail(CC_ECUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& s = g_dev[d];
  if (!s.checked) {
    cudaDeviceProp prop;
    const cudaError_t e = cudaGetDeviceProperties(&prop, d);
    s.checked = true;
    if (e != cudaSuccess) {
      s.status = CC_ECUDA;
    } else if (!(prop.major == 10 && prop.minor == 3)) {
      s.status = CC_EDEVICE;
    } else {
      s.status = CC_OK;
      s.sms = prop.multiProcessorCount;
    }
  }
  if (s.status == CC_EDEVICE)
    return fail(CC_EDEVICE, "the library is built for sm_103a (GB300) devices only");
  if (s.status != CC_OK) return fail(s.status, "cudaGetDeviceProperties failed");
  return CC_OK;
}

int num_sms() {
  const int d = current_device();
  if (d < 0 || d >= 64) return 1;
  std::lock_guard<std::mutex> lk(g_mu);
  return std::max(1, g_dev[d].sms);
}

void* scratch(size_t bytes) {
  const int d = current_device();
  if (d < 0 || d >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& s = g_dev[d];
  if (s.scratch_bytes < bytes) {
    if (s.scratch) cudaFree(s.scratch);
    s.scratch = nullptr;
    s.scratch_bytes = 0;
    const size_t want = std::max(bytes, size_t(1) << 20);
    if (cudaMalloc(&s.scratch, want) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    s.scratch_bytes = want;
  }
  return s.scratch;
}

int* device_error_flag() {
  const int d = current_device();
  if (d < 0 || d >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& s = g_dev[d];
  if (!s.err_flag) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess || cudaMemset(p, 0, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      if (p) cudaFree(p);
      return nullptr;
    }
    s.err_flag = static_cast<int*>(p);
  }
  return s.err_flag;
}

void* device_alloc_copy(const void* host, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max(bytes, size_t(16))) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (bytes && cudaMemcpy(p, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p);
    return nullptr;
  }
  return p;
}

void device_free(void* p) {
  if (p) cudaFree(p);
}

int max_tile_bits(int precision) { return precision == CC_C128 ? 13 : 14; }
int low_tile_bits(int precision) { return precision == CC_C128 ? 3 : 4; }

int seg_tile_bits(int precision) {
  // 2^13-amplitude tiles leave room for two CTAs per SM (measured ~11% faster
  // than 2^14 on the 15-qubit, 64-variant segments)
  int k = std::min(13, max_tile_bits(precision));
  if (const char* e = std::getenv("CUTSIM_SEG_TILE_BITS")) {
    const int v = std::atoi(e);
    if (v >= low_tile_bits(precision) + 1 && v <= max_tile_bits(precision)) k = v;
  }
  return k;
}

bool seg_launch_per_pass() {
  const char* e = std::getenv("CUTSIM_SEG_LAUNCH");
  return e && std::strcmp(e, "passes") == 0;
}

int uncut_tile_bits(int precision) {
  // 2^13 as for segments: two CTAs per SM hide the tile load/store latency
  // (measured ~5% faster than 2^14 on the 30-qubit brickwork)
  int k = std::min(13, max_tile_bits(precision));
  if (const char* e = std::getenv("CUTSIM_UNCUT_TILE_BITS")) {
    const int v = std::atoi(e);
    if (v >= low_tile_bits(precision) + 1 && v <= max_tile_bits(precision)) k = v;
  }
  return k;
}

ImageLayout append_program_image(const HostProgram& hp, int arith,
                                 std::vector<unsigned char>& img) {
  const size_t rb = arith == GA_F32 ? 4 : 8;
  ImageLayout L;
  L.base = (img.size() + 255) & ~size_t(255);
  L.o_pass = 0;
  L.o_stages = align16(L.o_pass + hp.passes.size() * sizeof(DPass));
  L.o_ops = align16(L.o_stages + hp.stages.size() * sizeof(DStage));
  L.o_terms = align16(L.o_ops + hp.ops.size() * sizeof(DOp));
  L.o_mats = align16(L.o_terms + hp.terms.size() * sizeof(DTerm));
  L.o_tabs = align16(L.o_mats + hp.ops.size() * 4 * 2 * rb);  // one matrix slot per op
  L.end = align16(L.o_tabs + hp.tabs.size() * 2 * rb);
  img.resize(L.base + L.end, 0);
  unsigned char* p0 = img.data() + L.base;
  std::memcpy(p0 + L.o_pass, hp.passes.data(), hp.passes.size() * sizeof(DPass));
  std::memcpy(p0 + L.o_stages, hp.stages.data(), hp.stages.size() * sizeof(DStage));
  std::memcpy(p0 + L.o_ops, hp.ops.data(), hp.ops.size() * sizeof(DOp));
  std::memcpy(p0 + L.o_terms, hp.terms.data(), hp.terms.size() * sizeof(DTerm));
  auto put = [&](size_t off, const std::vector<cd>& v) {
    for (size_t i = 0; i < v.size(); ++i) {
      if (arith == GA_DFL) {  // h = fl32(x), l = fl32(x - h)
        float* p = reinterpret_cast<float*>(p0 + off) + 4 * i;
        const double re = v[i].real(), im = v[i].imag();
        p[0] = (float)re;
        p[1] = (float)(re - (double)p[0]);
        p[2] = (float)im;
        p[3] = (float)(im - (double)p[2]);
      } else if (rb == 8) {
        double* p = reinterpret_cast<double*>(p0 + off) + 2 * i;
        p[0] = v[i].real();
        p[1] = v[i].imag();
      } else {
        float* p = reinterpret_cast<float*>(p0 + off) + 2 * i;
        p[0] = (float)v[i].real();
        p[1] = (float)v[i].imag();
      }
    }
  };
  // The kernels read op o's matrix at slot o, so that it does not wait on the
  // op's descriptor; diagonal-only ops get a zero slot.
  std::vector<cd> per_op(hp.ops.size() * 4, cd(0.0, 0.0));
  for (size_t o = 0; o < hp.ops.size(); ++o)
    if (hp.ops[o].type != OP_DIAG)
      for (int e = 0; e < 4; ++e) per_op[4 * o + e] = hp.mats[4 * (size_t)hp.ops[o].mat + e];
  put(L.o_mats, per_op);
  put(L.o_tabs, hp.tabs);
  return L;
}

void bind_program(DeviceProgram& dp, const HostProgram& hp, unsigned char* dev_base,
                  const ImageLayout& L) {
  unsigned char* b = dev_base + L.base;
  dp.base = nullptr;  // not owned
  dp.bytes = L.end;
  dp.passes_dev = b + L.o_pass;
  dp.stages = reinterpret_cast<const DStage*>(b + L.o_stages);
  dp.ops = reinterpret_cast<const DOp*>(b + L.o_ops);
  dp.terms = reinterpret_cast<const DTerm*>(b + L.o_terms);
  dp.mats = b + L.o_mats;
  dp.tabs = b + L.o_tabs;
  dp.passes = hp.passes;
  dp.n_ops = (int)hp.ops.size();
}

namespace {
// Pass pi's blob (PassBlob layout) from the host program and its image
// (whose per-op matrices and tables already hold the arithmetic's reals,
// rb bytes each); false when it does not fit.
bool build_pass_blob(const HostProgram& hp, int pi, const unsigned char* p0,
                     const ImageLayout& L, size_t rb, PassBlob& out) {
  const DPass& P = hp.passes[pi];
  const int sb = P.stage_begin, se = P.stage_end;
  const int ob = se > sb ? hp.stages[sb].op_begin : 0;
  const int oe = se > sb ? hp.stages[se - 1].op_end : 0;
  int tb = 0, te = 0, ab = 0, ae = 0;
  bool any_t = false, any_a = false;
  auto tab_range = [&](int lo, int hi) {
    if (!any_a) { ab = lo; ae = hi; any_a = true; }
    ab = std::min(ab, lo);
    ae = std::max(ae, hi);
  };
  for (int o = ob; o < oe; ++o) {
    const DOp& op = hp.ops[o];
    if (op.term_end() > op.term_begin) {
      if (!any_t) { tb = op.term_begin; te = op.term_end(); any_t = true; }
      tb = std::min(tb, op.term_begin);
      te = std::max(te, op.term_end());
    }
    if (op.n_phase) tab_range(op.blk_tab, op.blk_tab + 8);
  }
  for (int t = tb; t < te; ++t) {
    const DTerm& d = hp.terms[t];
    if (d.kind == TERM_PBLOCK) tab_range(d.tab, d.tab + 8);
    else if (d.kind != TERM_SIGN) tab_range(d.tab, d.tab + 1);
  }
  const size_t n_st = se - sb, n_op = oe - ob, n_t = te - tb, n_tab = ae - ab;
  PassBlobHeader h{};
  size_t off = align16(sizeof(PassBlobHeader));
  h.o_pass = (int32_t)off;   off = align16(off + sizeof(DPass));
  h.o_stages = (int32_t)off; off = align16(off + n_st * sizeof(DStage));
  h.o_ops = (int32_t)off;    off = align16(off + n_op * sizeof(DOp));
  h.o_terms = (int32_t)off;  off = align16(off + n_t * sizeof(DTerm));
  h.o_mats = (int32_t)off;   off = align16(off + n_op * 8 * rb);
  h.o_tabs = (int32_t)off;   off = align16(off + n_tab * 8 * rb);
  if (off > sizeof(out.b)) return false;
  std::memset(out.b, 0, sizeof(out.b));
  std::memcpy(out.b, &h, sizeof(h));
  DPass q = P;
  q.stage_begin = 0;
  q.stage_end = (int32_t)n_st;
  std::memcpy(out.b + h.o_pass, &q, sizeof(q));
  for (size_t i = 0; i < n_st; ++i) {
    DStage st = hp.stages[sb + i];
    st.op_begin -= ob;
    st.op_end -= ob;
    std::memcpy(out.b + h.o_stages + i * sizeof(DStage), &st, sizeof(st));
  }
  for (size_t i = 0; i < n_op; ++i) {
    DOp op = hp.ops[ob + i];
    if (op.term_end() > op.term_begin) op.term_begin -= tb;
    if (op.n_phase) op.blk_tab -= ab;
    std::memcpy(out.b + h.o_ops + i * sizeof(DOp), &op, sizeof(op));
  }
  for (size_t i = 0; i < n_t; ++i) {
    DTerm d = hp.terms[tb + i];
    if (d.kind != TERM_SIGN) d.tab -= ab;
    std::memcpy(out.b + h.o_terms + i * sizeof(DTerm), &d, sizeof(d));
  }
  std::memcpy(out.b + h.o_mats, p0 + L.o_mats + (size_t)ob * 8 * rb, n_op * 8 * rb);
  std::memcpy(out.b + h.o_tabs, p0 + L.o_tabs + (size_t)ab * 8 * rb, n_tab * 8 * rb);
  return true;
}
}  // namespace

cc_status upload_program(const HostProgram& hp, int arith, DeviceProgram& dp) {
  std::vector<unsigned char> img;
  const ImageLayout L = append_program_image(hp, arith, img);
  void* base = device_alloc_copy(img.data(), img.size());
  if (!base) return fail(CC_ENOMEM, "device allocation of a gate program failed");
  bind_program(dp, hp, static_cast<unsigned char*>(base), L);
  dp.base = base;  // owned
  const size_t rb = arith == GA_F32 ? 4 : 8;
  dp.blobs.resize(hp.passes.size());
  dp.blob_ok.assign(hp.passes.size(), 0);
  for (size_t pi = 0; pi < hp.passes.size(); ++pi)
    dp.blob_ok[pi] = build_pass_blob(hp, (int)pi, img.data() + L.base, L, rb, dp.blobs[pi]);
  return CC_OK;
}

void free_program(DeviceProgram& dp) {
  if (dp.base) cudaFree(dp.base);
  dp = DeviceProgram();
}

}  // namespace cc

using namespace cc;

namespace {
int amp_bytes(int precision) { return precision == CC_C128 ? 16 : 8; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

cc_status sync_status(cudaStream_t s, const char* what) {
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return CC_OK;
}
}  // namespace

extern "C" cc_status cc_simulate_segments(const cc_plan* p, void* seg_buf, uint64_t bytes,
                                          void* stream) {
  if (!p) return fail(CC_EINVAL, "plan is NULL");
  if (!seg_buf) return fail(CC_EINVAL, "seg_buf is NULL");
  if (!aligned16(seg_buf)) return fail(CC_EINVAL, "seg_buf must be 16-byte aligned");
  if (bytes < p->seg_buf_bytes)
    return fail(CC_EBUFSIZE, "seg_buf holds " + std::to_string(bytes) + " bytes, plan needs " +
                                 std::to_string(p->seg_buf_bytes));
  cc_status st = check_device();
  if (st != CC_OK) return st;
  if (seg_launch_per_pass()) {  // one launch per pass and segment
    const int ab = amp_bytes(p->precision);
    for (int i = 0; i < p->n_seg; ++i) {
      char* base = static_cast<char*>(seg_buf) + p->seg_off[i] * ab;
      st = run_program(p->dprog[i], p->arith, base, stream);
      if (st != CC_OK) return st;
    }
    return CC_OK;
  }
  // Default: every pass of every segment in one persistent launch, so the
  // segments' passes overlap instead of running one after another.
  const cudaError_t e = cudaMemsetAsync(p->seg_state, 0, p->seg_state_bytes, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("memset: ") + cudaGetErrorString(e));
  return launch_batch_segments(seg_buf, p->seg_jobs, p->seg_n_jobs, p->seg_n_items, p->seg_done,
                               p->seg_head, nullptr, p->arith, p->seg_block, p->seg_smem,
                               p->seg_grid, stream);
}

extern "C" cc_status cc_merge(const cc_plan* p, const void* seg_buf, uint64_t seg_bytes,
                              void* psi, uint64_t psi_bytes, void* workspace, uint64_t ws_bytes,
                              int32_t form, void* stream) {
  if (!p) return fail(CC_EINVAL, "plan is NULL");
  if (!seg_buf || !psi) return fail(CC_EINVAL, "NULL buffer");
  if (!aligned16(seg_buf) || !aligned16(psi) || (workspace && !aligned16(workspace)))
    return fail(CC_EINVAL, "buffers must be 16-byte aligned");
  if (seg_bytes < p->seg_buf_bytes) return fail(CC_EBUFSIZE, "seg_buf too small");
  if (psi_bytes < p->psi_bytes) return fail(CC_EBUFSIZE, "psi too small");
  if (form < CC_MERGE_AUTO || form > CC_MERGE_F16X3) return fail(CC_EINVAL, "unknown merge form");
  if ((form == CC_MERGE_TF32X3 || form == CC_MERGE_BF16X3 || form == CC_MERGE_F16X3) &&
      p->precision != CC_C64)
    return fail(CC_EINVAL, "tensor-core merge forms need a complex64 plan");
  if (form == CC_MERGE_OZAKI && p->precision != CC_C128)
    return fail(CC_EINVAL, "the Ozaki merge form needs a complex128 plan");
  cc_status st = check_device();
  if (st != CC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int ab = amp_bytes(p->precision);
  const char* sb = static_cast<const char*>(seg_buf);
  if (p->n_seg == 1) {
    const cudaError_t e = cudaMemcpyAsync(psi, sb, p->psi_bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(CC_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
    return CC_OK;
  }
  const int32_t* tables = static_cast<const int32_t*>(p->tables_dev);
  // n >= 3: the stages before the last chain through two workspace buffers;
  // the last stage (Z = 1, the 2^q output) may use a tensor-core form.
  const uint64_t half = p->n_seg >= 3 ? p->chain_ws_amps * ab : 0;
  if (p->n_seg >= 3 && (!workspace || ws_bytes < 2 * half))
    return fail(CC_EBUFSIZE, "workspace too small for the chained merge");
  char* w[2] = {static_cast<char*>(workspace), static_cast<char*>(workspace) + half};
  const void* acc = sb + p->seg_off[0] * ab;
  for (size_t s_i = 0; s_i < p->stages.size(); ++s_i) {
    const auto& sg = p->stages[s_i];
    const bool last = s_i + 1 == p->stages.size();
    void* out = last ? psi : w[s_i & 1];
    MergeStage ms{acc, sb + p->seg_off[sg.seg] * ab, out, sg.qa, sg.qb, sg.K, sg.Z,
                  int64_t(1) << (sg.qa + sg.qb), tables + sg.aidx_off, tables + sg.bidx_off};
    if (!last) {
      st = launch_merge_fma(ms, p->precision, stream);
      if (st != CC_OK) return st;
      acc = out;
      continue;
    }
    // AUTO: the CUDA-core form while the merge is store-bound (K below
    // kAutoTcMinTerms), else 3xFP16 (long K summed in groups of 64 terms, see
    // merge_tc.cu).
    // complex128: the Ozaki tensor-core form wherever it applies.
    int f = form;
    if (f == CC_MERGE_AUTO) {
      if (p->precision == CC_C64)
        f = (sg.K >= kAutoTcMinTerms && sg.qa >= 7 && sg.qb >= 7) ? kAutoTcForm : CC_MERGE_FMA;
      else
        f = (sg.K >= kAutoOzakiMinTerms && sg.qa >= 7 && sg.qb >= 7) ? CC_MERGE_OZAKI
                                                                       : CC_MERGE_FMA;
    }
    if (f != CC_MERGE_FMA) {
      void* tc_ws = workspace ? static_cast<char*>(workspace) + 2 * half : nullptr;
      const uint64_t tc_bytes = ws_bytes > 2 * half ? ws_bytes - 2 * half : 0;
      const uint64_t need = f == CC_MERGE_OZAKI ? merge_ozaki_workspace_bytes(sg.qa, sg.qb, sg.K)
                                                : merge_tc_workspace_bytes(sg.qa, sg.qb, sg.K, f);
      if (!tc_ws || tc_bytes < need) {
        if (form != CC_MERGE_AUTO)
          return fail(CC_EBUFSIZE, "workspace too small for the tensor-core merge");
        f = CC_MERGE_FMA;
      } else {
        st = f == CC_MERGE_OZAKI ? launch_merge_ozaki(ms, tc_ws, tc_bytes, stream)
                                 : launch_merge_tc(ms, f, tc_ws, tc_bytes, stream);
        if (st == CC_OK) return CC_OK;
        if (st != CC_EUNSUPPORTED || form != CC_MERGE_AUTO) return st;
        f = CC_MERGE_FMA;
      }
    }
    return launch_merge_fma(ms, p->precision, stream);
  }
  return CC_OK;
}

extern "C" cc_status cc_simulate_uncut(const cc_uncut* u, void* psi, uint64_t psi_bytes,
                                       void* stream) {
  if (!u) return fail(CC_EINVAL, "uncut plan is NULL");
  if (!psi) return fail(CC_EINVAL, "psi is NULL");
  if (!aligned16(psi)) return fail(CC_EINVAL, "psi must be 16-byte aligned");
  if (psi_bytes < (uint64_t(1) << u->q) * amp_bytes(u->precision))
    return fail(CC_EBUFSIZE, "psi too small");
  cc_status st = check_device();
  if (st != CC_OK) return st;
  return run_program(u->dprog, u->arith, psi, stream);
}

extern "C" cc_status cc_compare(const void* a, const void* b, int64_t n_amp, int32_t precision,
                                double* out, void* stream) {
  if (!a || !b || !out) return fail(CC_EINVAL, "NULL argument");
  if (precision != CC_C64 && precision != CC_C128) return fail(CC_EINVAL, "unknown precision");
  if (n_amp < 0) return fail(CC_EINVAL, "n_amp < 0");
  if (!aligned16(a) || !aligned16(b)) return fail(CC_EINVAL, "buffers must be 16-byte aligned");
  cc_status st = check_device();
  if (st != CC_OK) return st;
  const int n_blocks = num_sms() * 4;
  double* scr = static_cast<double*>(scratch(sizeof(double) * 8 * (n_blocks + 1)));
  if (!scr) return fail(CC_ENOMEM, "scratch allocation failed");
  cudaStream_t s = (cudaStream_t)stream;
  st = launch_compare(a, b, n_amp, precision, scr + 8 * n_blocks, scr, n_blocks, stream);
  if (st != CC_OK) return st;
  double res[8];
  const cudaError_t e = cudaMemcpyAsync(res, scr + 8 * n_blocks, sizeof(res), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
  st = sync_status(s, "cc_compare");
  if (st != CC_OK) return st;
  std::memcpy(out, res, 6 * sizeof(double));
  return CC_OK;
}

extern "C" cc_status cc_gather(const void* psi, int64_t n_amp, int32_t precision,
                               const int64_t* idx, int64_t n_idx, void* out, void* stream) {
  if (!psi || !idx || !out) return fail(CC_EINVAL, "NULL argument");
  if (precision != CC_C64 && precision != CC_C128) return fail(CC_EINVAL, "unknown precision");
  if (n_idx < 0 || n_idx > (int64_t(1) << 20)) return fail(CC_ERANGE, "n_idx must be in 0..2^20");
  for (int64_t i = 0; i < n_idx; ++i)
    if (idx[i] < 0 || idx[i] >= n_amp)
      return fail(CC_ERANGE, "index " + std::to_string(idx[i]) + " outside [0, n_amp)");
  if (n_idx == 0) return CC_OK;
  cc_status st = check_device();
  if (st != CC_OK) return st;
  const int ab = amp_bytes(precision);
  char* scr = static_cast<char*>(scratch(n_idx * (8 + ab) + 16));
  if (!scr) return fail(CC_ENOMEM, "scratch allocation failed");
  int64_t* idx_dev = reinterpret_cast<int64_t*>(scr);
  void* out_dev = scr + ((n_idx * 8 + 15) & ~int64_t(15));
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(idx_dev, idx, n_idx * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
  st = launch_gather(psi, precision, idx_dev, n_idx, out_dev, stream);
  if (st != CC_OK) return st;
  e = cudaMemcpyAsync(out, out_dev, n_idx * ab, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
  return sync_status(s, "cc_gather");
}

extern "C" cc_status cc_sync(void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  cc_status st = sync_status(s, "cc_sync");
  if (st != CC_OK) return st;
  int* flag = device_error_flag();
  if (!flag) return fail(CC_ENOMEM, "device error flag allocation failed");
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h) e = cudaMemset(flag, 0, sizeof(int));
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("cc_sync: ") + cudaGetErrorString(e));
  if (h) return fail(CC_ETIMEOUT, "a bounded device wait expired; results of that call are undefined");
  return CC_OK;
}

extern "C" cc_status cc_copy_to_host(const void* src, void* host, uint64_t bytes, void* stream) {
  if (!src || !host) return fail(CC_EINVAL, "NULL buffer");
  if (bytes == 0) return CC_OK;
  if (!aligned16(src) || !aligned16(host)) return fail(CC_EINVAL, "buffers must be 16-byte aligned");
  cc_status st = check_device();
  if (st != CC_OK) return st;
  void* mapped = nullptr;
  if (cudaHostGetDevicePointer(&mapped, host, 0) != cudaSuccess || !mapped) {
    cudaGetLastError();  // not page-locked and mapped: the copy engines do it
    const cudaError_t e = cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(CC_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
    return CC_OK;
  }
  return launch_copy_to_host(src, mapped, bytes, stream);
}

extern "C" cc_status cc_check_wait_expiry(int32_t polls, void* stream) {
  if (polls < 1 || polls > (1 << 20)) return fail(CC_ERANGE, "polls must be in 1..2^20");
  cc_status st = check_device();
  if (st != CC_OK) return st;
  return launch_expired_wait(polls, stream);
}

extern "C" const char* cc_last_error(void) { return g_error.c_str(); }

extern "C" const char* cc_version(void) { return "cutsim 0.1 (sm_103a)"; }
