// Library-owned plan objects behind the opaque cc_plan / cc_uncut handles.
#pragma once

#include <cmath>
#include <memory>
#include <vector>

#include "internal.h"

namespace cc {
void* device_alloc_copy(const void* host, size_t bytes);  // NULL on failure
void device_free(void* p);
int uncut_tile_bits(int precision);
int seg_tile_bits(int precision);
bool seg_launch_per_pass();  // CUTSIM_SEG_LAUNCH=passes: one launch per segment pass
}  // namespace cc

struct cc_plan;
namespace cc {
// cc_plan_create with an explicit largest segment tile (bits, in
// low_tile_bits + 1 .. max_tile_bits).  host_only: stop after the host work
// (the segment programs and cut bits; no device tables, no device needed).
cc_status create_plan(const cc_gate* gates, int n_gates, int q, const int* seg_sizes, int n_seg,
                      int decomp, int precision, int seg_kmax, cc_plan** out,
                      bool host_only = false);
}  // namespace cc

struct cc_plan {
  struct Cut {
    int q0, q1, kind, s0, s1;
  };
  // Merge stage s: U_s = sum_k U_{s-1}[aidx] (x) seg_s[bidx], batched over z.
  struct Stage {
    int seg = 0;
    int qa = 0, qb = 0;  // log2 sizes of the accumulated factor and of segment s
    int64_t K = 1, Z = 1;
    int64_t aidx_off = 0, bidx_off = 0;  // offsets (int32 entries) into tables_dev
  };

  int q = 0, n_seg = 0, c_total = 0, precision = 0, decomp = 0;
  int arith = 0;  // gate-pass arithmetic (cc::GateArith) the device images are laid out for
  std::vector<int> seg_q, seg_start, seg_c;
  std::vector<int64_t> seg_off;
  struct Bit {
    int cut, s0, s1;  // the cut it belongs to and its two segments
  };
  std::vector<Bit> bits;                      // global cut bits (1 per rank-2 cut, 2 per rank-4)
  std::vector<std::vector<int>> seg_cut_ids;  // per segment: its bits in variant-bit order
  std::vector<Cut> cuts;
  std::vector<cc::HostProgram> hprog;
  std::vector<cc::DeviceProgram> dprog;
  std::vector<Stage> stages;
  void* arena = nullptr;       // the one device allocation holding every table below
  void* tables_dev = nullptr;  // merge index tables (inside arena)
  std::vector<int32_t> host_tables;  // the same tables, kept by host-only plans
  int64_t n_sub = 0;
  uint64_t seg_buf_bytes = 0, psi_bytes = 0, workspace_bytes = 0, table_bytes = 0;
  uint64_t chain_ws_amps = 0;  // amplitudes of one chained-merge intermediate buffer
  // Every segment pass as one job of a persistent launch (inside arena).
  const cc::BJob* seg_jobs = nullptr;
  void* seg_state = nullptr;  // per-run counters, zeroed before each launch
  size_t seg_state_bytes = 0;
  int* seg_done = nullptr;
  unsigned long long* seg_head = nullptr;
  int seg_n_jobs = 0, seg_block = 32, seg_grid = 1;
  int64_t seg_n_items = 0;
  size_t seg_smem = 0;

  ~cc_plan();
};

struct cc_uncut {
  int q = 0, precision = 0;
  int arith = 0;  // gate-pass arithmetic (cc::GateArith)
  cc::HostProgram hprog;
  cc::DeviceProgram dprog;
  ~cc_uncut();
};
