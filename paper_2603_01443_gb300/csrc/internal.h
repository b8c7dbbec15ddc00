// Internal definitions shared by the host runtime and the CUDA kernels.
#pragma once

#include <cstdint>
#include <complex>
#include <string>
#include <vector>

#include "cutsim.h"

namespace cc {

using cd = std::complex<double>;

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
cc_status fail(cc_status s, const std::string& msg);

// ------------------------------------------------------- device programs
// A gate program on an nq-qubit vector is a list of passes.  A pass moves one
// tile of 2^k amplitudes (k "tile bits" of the vector index) into shared
// memory, applies a list of fused operations there and writes it back.
//
// Inside a pass every amplitude carries a "virtual index"
//   v = l | (T << k) | (r << nq)
// where l is its tile-local index, T the tile number (the non-tile index bits
// in increasing order) and r the variant number of the vector.  Diagonal
// factors are functions of two bits of v, so a phase may depend on tile bits,
// on fixed (non-tile) bits and on the variant's cut bits alike.

enum : uint8_t { TERM_SIGN = 0, TERM_TABLE = 1 };

// Diagonal factor of one amplitude with virtual index v:
//   TERM_SIGN : multiply by -1 when bit p0 and bit p1 of v are both set
//   TERM_TABLE: multiply by tab[4*tab + (bit p0) + 2*(bit p1)]
struct DTerm {
  uint8_t kind, p0, p1, pad;
  int32_t tab;
};

enum : int32_t { OP_DENSE = 0, OP_DIAG = 1 };

// OP_DENSE: for every pair (l0, l1 = l0 | 1<<t) apply the terms
//           [term_begin, term_end) to both amplitudes, then the 2x2 matrix
//           mats[8*mat ...] (row-major, interleaved re/im).
// OP_DIAG : apply the terms to every amplitude.
struct DOp {
  int32_t type, t;
  int32_t term_begin, term_sign_end, term_end;  // sign terms first
  int32_t mat;
};

constexpr int MAX_TILE_BITS = 16;
constexpr int MAX_REST_BITS = 40;

struct DPass {
  int32_t nq;         // qubits of the vector
  int32_t k;          // tile bits
  int32_t low;        // tile bits [0, low) are vector bits [0, low)
  int32_t init_zero;  // tile starts as |0...0> instead of being loaded
  int32_t op_begin, op_end;
  int32_t n_rest;     // nq - k
  int8_t tile_bit[MAX_TILE_BITS];  // vector bit of tile bit t
  int8_t rest_bit[MAX_REST_BITS];  // vector bit of the r-th non-tile bit
};

struct HostProgram {
  int nq = 0;
  int var_bits = 0;
  std::vector<DPass> passes;
  std::vector<DOp> ops;
  std::vector<DTerm> terms;
  std::vector<cd> mats;  // 4 per matrix, row-major
  std::vector<cd> tabs;  // 4 per table
};

// One operation of a (segment or uncut) program before pass planning.
enum ItemKind : int { IT_DENSE = 0, IT_DIAG1 = 1, IT_CZ = 2, IT_VAR = 3 };
struct Item {
  int kind = IT_DENSE;
  int a = -1, b = -1;  // qubits (b for IT_CZ)
  cd u[4];             // IT_DENSE: matrix; IT_DIAG1: u[0], u[3] diagonal
  int slot = -1;       // IT_VAR: variant bit
  bool var_sign = false;  // IT_VAR: factor is Z^b (a sign term)
  cd d[2][2];             // IT_VAR: factor d[b][x] for variant bit b, index bit x
};

// Build the program of a list of items on nq qubits with var_bits variant
// bits.  Tiles have at most kmax bits, the lowest `low` of them contiguous.
HostProgram compile_program(const std::vector<Item>& items, int nq, int var_bits, int kmax,
                            int low);

// Gate -> items (CX as H CZ H on the target; diagonal one-qubit gates as IT_DIAG1).
cc_status gate_items(const cc_gate& g, int qoff, std::vector<Item>& out);
cc_status check_gates(const cc_gate* gates, int n_gates, int q);

// Device image of a program: one allocation holding ops, terms, matrices and
// tables, reals converted to the plan's precision.
struct DeviceProgram {
  void* base = nullptr;
  size_t bytes = 0;
  const DOp* ops = nullptr;
  const DTerm* terms = nullptr;
  const void* mats = nullptr;
  const void* tabs = nullptr;
  const void* passes_dev = nullptr;
  std::vector<DPass> passes;
  int n_ops = 0;
};

cc_status upload_program(const HostProgram& hp, int precision, DeviceProgram& dp);
void free_program(DeviceProgram& dp);

// Launch every pass of a program over n_vec vectors of 2^nq amplitudes
// spaced vec_stride amplitudes apart, starting at `state`.
cc_status run_program(const DeviceProgram& dp, int precision, void* state, int64_t n_vec,
                      int64_t vec_stride, void* stream);

// Largest tile (bits) a pass may use: 2^k amplitudes in shared memory.
int max_tile_bits(int precision);
int low_tile_bits(int precision);

// -------------------------------------------------------------- merging
// Batched two-factor merge:
//   out[z*out_stride + y*NA + x] = sum_k A[aidx[z*K+k]*NA + x] * B[bidx[z*K+k]*NB + y]
// with NA = 2^qa, NB = 2^qb, for z < Z.  aidx, bidx are device int32 tables.
struct MergeStage {
  const void* A;
  const void* B;
  void* out;
  int qa, qb;
  int64_t K, Z;
  int64_t out_stride;
  const int32_t* aidx;
  const int32_t* bidx;
};

cc_status launch_merge_fma(const MergeStage& st, int precision, void* stream);

// Tensor-core merge (single stage, Z = 1, identity index tables): returns
// CC_EUNSUPPORTED when the shape does not suit the kernel.
uint64_t merge_tc_workspace_bytes(int qa, int qb, int64_t K, int form);
cc_status launch_merge_tc(const MergeStage& st, int form, void* workspace, uint64_t ws_bytes,
                          void* stream);

// ----------------------------------------------------------- reductions
cc_status launch_compare(const void* a, const void* b, int64_t n, int precision, double* out_dev,
                         double* partials, int n_blocks, void* stream);
cc_status launch_gather(const void* psi, int precision, const int64_t* idx_dev, int64_t n,
                        void* out_dev, void* stream);

// --------------------------------------------------------------- device
cc_status check_device();
int num_sms();
void* scratch(size_t bytes);  // per-device library scratch (grown on demand)
int* device_error_flag();     // per-device int set by kernels whose bounded waits expire

}  // namespace cc
