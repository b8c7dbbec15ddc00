// Internal definitions shared by the host runtime and the CUDA kernels.
#pragma once

#include <cstdint>
#include <complex>
#include <string>
#include <vector>

#include "cutsim.h"

#ifdef __CUDACC__
#define CC_HD __host__ __device__
#else
#define CC_HD
#endif

namespace cc {

using cd = std::complex<double>;

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
cc_status fail(cc_status s, const std::string& msg);

// ------------------------------------------------------- device programs
// A gate program acts on one vector of 2^nq amplitudes.  For a segment the
// vector is the whole block of its 2^{c_i} variants: the variant number
// occupies the index bits above the segment's q_i qubits, so a variant bit is
// a "qubit" that carries no dense gate, only the diagonal cut terms, and many
// small variants share one tile.
//
// The program is a list of passes.  A pass moves tiles of 2^k amplitudes (k
// "tile bits" of the vector index) through shared memory.  Inside a pass every
// amplitude carries a virtual index v = l | (T << k), where l is its tile-local
// index and T the tile number (the non-tile bits in increasing order); every
// diagonal factor is a function of bits of v.
//
// A pass is a list of stages.  In a stage each thread holds 2^rbits amplitudes
// in registers whose tile bits are the stage's register bits; dense one-qubit
// matrices act on register bits only, so a stage runs without touching shared
// memory, and shared memory is used only to re-map bits between stages.

enum : uint8_t { TERM_SIGN = 0, TERM_TABLE = 1, TERM_PBLOCK = 2, TERM_PFIX = 3 };

// Diagonal factor of one amplitude with virtual index v:
//   TERM_SIGN  : multiply by -1 when bit p0 and bit p1 of v are both set
//   TERM_TABLE : multiply by tab[4*tab + (bit p0) + 2*(bit p1)]
//   TERM_PBLOCK: opens a phase block, a product of one-bit phases: with the
//                32 entries T[j] at tab[4*tab], T[j] = K times the product of
//                h_i over the register bits i set in j, it multiplies the
//                amplitude in register slot j by T[j]
//   TERM_PFIX  : inside a phase block, multiply by tab[4*tab] when bit p0 of
//                v (a bit that is not a register bit of the stage) is set
struct DTerm {
  uint8_t kind, p0, p1, pad;
  int32_t tab;
};

// OP_ROT and OP_ROTC are real rotations [[c, -s], [s, c]] in tangent form,
// their scalar factor c (or s) carried by a later phase block:
//   OP_ROT : (a, b) <- (a - t b, b + t a),  t = s / c  (|t| <= 1)
//   OP_ROTC: (a, b) <- (t a - b, a + t b),  t = c / s  (|t| <= 1)
// OP_ROTS applies one such rotation on each register bit i set in its mask t
// (OP_ROTC form where bit i of cot is set) with tangent mats[8*mat + i]; the
// rotations act on distinct bits, so their order does not matter.
enum : int32_t { OP_DENSE = 0, OP_DIAG = 1, OP_ROT = 2, OP_ROTC = 3, OP_ROTS = 4 };

// Before its matrix, an op multiplies each amplitude by (-1)^s with
//   s = popcount(v & (v >> 1) & sign_adj) + sum of the sign terms (bit pairs
//       not adjacent in v)   (mod 2)
// then by its phase block (if any) and every table term.  OP_DENSE then
// applies the 2x2 matrix mats[8*mat ...] (row-major, interleaved re/im) to
// register bit t, OP_ROT / OP_ROTC their rotation with t = mats[8*mat],
// OP_ROTS its rotations on the register bits of the mask t;
// OP_DIAG stops after the diagonal factors.
struct alignas(16) DOp {
  int8_t type, t;
  // terms [term_begin, +n_sign) are sign terms, the next n_phase the phase
  // block (TERM_PBLOCK, then TERM_PFIX), the next n_table table terms
  uint16_t n_sign, n_phase, n_table;
  int32_t term_begin;
  int32_t mat;
  uint64_t sign_adj;  // bit p set: a sign term on (p, p+1)
  uint8_t cot;        // OP_ROTS: register bits whose rotation is in OP_ROTC form
  uint8_t blk_p0;     // copies of the phase block's p0 and tab (when n_phase > 0),
  uint16_t pad;       // so the kernels read the block's table without first
  int32_t blk_tab;    // loading its term
  CC_HD int term_sign_end() const { return term_begin + n_sign; }
  CC_HD int term_phase_end() const { return term_sign_end() + n_phase; }
  CC_HD int term_end() const { return term_phase_end() + n_table; }
};
static_assert(sizeof(DOp) == 32, "two 16-byte loads per op");

struct DStage {
  int32_t op_begin, op_end;
  int8_t rb[8];  // tile bit of register bit i
};

constexpr int MAX_TILE_BITS = 16;
constexpr int MAX_REST_BITS = 48;
constexpr int MAX_REG_BITS = 5;

struct DPass {
  int32_t nq;          // bits of the vector index
  int32_t k;           // tile bits
  int32_t low;         // tile bits [0, low) are vector bits [0, low)
  int32_t init_zero;   // tiles start from |0...0> per variant instead of being loaded
  int32_t stage_begin, stage_end;
  int32_t rbits;       // register bits per thread: 2^rbits amplitudes, 2^(k - rbits) threads
  int32_t n_rest;      // nq - k
  uint32_t zero_tile;  // init: tile bits that are state qubits (must be 0 for amplitude 1)
  uint32_t flags;      // PASS_LAST: the program's last pass
  uint64_t zero_rest;  // init: bits of T that are state qubits
  int8_t tile_bit[MAX_TILE_BITS];  // vector bit of tile bit t
  int8_t rest_bit[MAX_REST_BITS];  // vector bit of the r-th non-tile bit
};

// The last pass of a program stores its vector in the precision's own layout;
// a double-float program's earlier passes store (h, l) pairs.
constexpr uint32_t PASS_LAST = 1u;

// Arithmetic of the gate passes.  Complex64 runs in FP32; complex128 runs in
// double-float pairs on the FP32 pipes (GA_DFL, about 48 significant bits)
// unless CUTSIM_C128_GATES=fp64 selects native FP64.  A program's device
// image holds its reals in the arithmetic's layout: FP32, FP64, or an
// (h, l) float pair in each 8-byte slot.
enum GateArith : int { GA_F32 = 0, GA_F64 = 1, GA_DFL = 2 };
int gate_arith(int precision);

struct HostProgram {
  int nq = 0;       // vector bits (state qubits + variant bits)
  int n_state = 0;  // state qubits (the low bits)
  std::vector<DPass> passes;
  std::vector<DStage> stages;
  std::vector<DOp> ops;
  std::vector<DTerm> terms;
  std::vector<cd> mats;  // 4 per matrix, row-major
  std::vector<cd> tabs;  // 4 per table
};

// One operation of a (segment or uncut) program before pass planning.
enum ItemKind : int { IT_DENSE = 0, IT_DIAG1 = 1, IT_CZ = 2, IT_VAR = 3, IT_DIAG2 = 4 };
struct Item {
  int kind = IT_DENSE;
  int a = -1, b = -1;  // qubits (IT_CZ, IT_DIAG2: the second qubit; IT_VAR: the variant bit)
  cd u[4];             // IT_DENSE: matrix; IT_DIAG1: u[0], u[3] diagonal
  // IT_DENSE from a U3 gate: the angles (theta, phi, lambda), the matrix is
  // built where the item is applied (u3_matrix), on the thread compiling it
  bool u3 = false;
  double ang[3] = {0.0, 0.0, 0.0};
  int slot = -1;       // IT_VAR: variant bit number (b = n_state + slot)
  bool var_sign = false;  // IT_VAR: factor is Z^b (a sign term)
  cd d[2][2];             // IT_VAR: factor d[b][x] for variant bit b, index bit x of a;
                          // IT_DIAG2: factor d[x_b][x_a] on qubits a, b
};

// Build the program of a list of items on an nq-bit vector whose low n_state
// bits are state qubits.  Tiles have at most kmax bits, the lowest `low` of
// them contiguous; stages hold at most rb_max register bits.
HostProgram compile_program(const std::vector<Item>& items, int nq, int n_state, int kmax,
                            int low, int rb_max);
int reg_bits_max(int precision);

// Gate -> items (CX as H CZ H on the target; diagonal one-qubit gates as
// IT_DIAG1; SWAP, ISWAP, CAN as basis changes around diagonal ZZ phases).
cc_status gate_items(const cc_gate& g, int qoff, std::vector<Item>& out);
bool is_two_qubit(int kind);
bool is_rank4(int kind);
// Pauli weights of a rank-4 gate: U = c[0] II + c[1] XX + c[2] YY + c[3] ZZ.
void pauli_weights(const cc_gate& g, cd c[4]);
cc_status check_gates(const cc_gate* gates, int n_gates, int q);

// One pass's part of a program, renumbered from 0 (stages, ops, terms,
// per-op matrices, tables), small enough to travel as the kernel parameter
// of that pass's launch: the kernel then reads its ops and tables through the
// constant bank instead of from global memory.  Layout: a PassBlobHeader,
// then at its offsets the DPass, the DStages, the DOps, the DTerms, the
// matrices (8 reals per op) and the tables (8 reals per table), each 16-byte
// aligned.
constexpr int PASS_BLOB_BYTES = 32 * 1024 - 64;  // kernel parameters: at most 32764 bytes
struct alignas(16) PassBlob {
  unsigned char b[PASS_BLOB_BYTES];
};
struct PassBlobHeader {
  int32_t o_pass, o_stages, o_ops, o_terms, o_mats, o_tabs, pad[2];
};

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
  const DStage* stages = nullptr;
  std::vector<DPass> passes;
  int n_ops = 0;
  // per pass: its blob when it fits (blob_ok), for the parameter-space launch
  std::vector<PassBlob> blobs;
  std::vector<char> blob_ok;
};

// Device image layout of one program inside a larger table buffer.
struct ImageLayout {
  size_t base, o_pass, o_stages, o_ops, o_terms, o_mats, o_tabs, end;
};
// Append hp's image (reals in the layout of the gate arithmetic) to img,
// 256-byte aligned.
ImageLayout append_program_image(const HostProgram& hp, int arith,
                                 std::vector<unsigned char>& img);
// Point dp at an uploaded image (dev_base = device copy of img); dp does not own it.
void bind_program(DeviceProgram& dp, const HostProgram& hp, unsigned char* dev_base,
                  const ImageLayout& L);
cc_status upload_program(const HostProgram& hp, int arith, DeviceProgram& dp);
void free_program(DeviceProgram& dp);

// Launch every pass of a program over the 2^nq-amplitude vector at `state`.
cc_status run_program(const DeviceProgram& dp, int arith, void* state, void* stream);

// Largest tile (bits) a pass may use: 2^k amplitudes in shared memory.
int max_tile_bits(int precision);
int low_tile_bits(int precision);

// ------------------------------------------------------------- batching
// One pass of one segment program inside a batched launch.  The queue of the
// launch is the concatenation of every job's tiles, jobs ordered by pass
// number, so every tile a job waits for sits earlier in the queue.
struct BJob {
  int64_t vec_off;       // amplitude offset of the program's vector in seg_buf
  const DPass* pass;     // device pointers into the program's image
  const DStage* stages;
  const DOp* ops;
  const DTerm* terms;
  const void* mats;
  const void* tabs;
  int64_t tile_begin;    // first queue item of this job
  int64_t n_tiles;
  int32_t dep;           // job whose tiles must all be stored first (-1: none)
  int32_t pad;
};

// Persistent launch over all jobs: CTAs take queue items from *head; done[j]
// counts the stored tiles of job j (both zeroed by the caller).  A wait that
// exceeds its iteration limit sets the device error flag, skips the tile and
// still counts it, so the launch always ends.  stamps (optional) receives the
// %globaltimer value when the first item is taken.
cc_status launch_batch_segments(void* seg_buf, const BJob* jobs, int n_jobs, int64_t n_items,
                                int* done, unsigned long long* head,
                                unsigned long long* stamps, int arith, int block,
                                size_t smem, int grid, void* stream);
// CTAs per SM the batched segment kernel reaches with this block and shared memory.
int batch_segments_occupancy(int arith, int block, size_t smem);

// One merge stage of one circuit inside a batched merge launch; operands are
// offsets (in amplitudes) into one of three caller buffers.
enum : int32_t { BUF_SEG = 0, BUF_WORK = 1, BUF_PSI = 2 };

// CC_MERGE_AUTO (and batches) merge on the tensor cores (3xTF32) from this
// many terms on, where both factors have >= 2^7 amplitudes: at q = 30 the
// CUDA-core form is store-bound through K = 4 and slower from K = 8 on
// (K = 8: 2.03 ms FMA, 1.64 ms 3xTF32).
constexpr int64_t kAutoTcMinTerms = 8;
// The complex64 tensor-core form AUTO and batches use: 3xFP16 with operand
// scales (q = 30: K = 64 1.70 ms against 2.56 ms for 3xTF32, K = 256 7.99
// against 9.00; within 3 % of it at K = 8, 16), also the more accurate
// (q = 30, K = 64: 2.2e-7 against 3.5e-7 of max |psi| on the oracle's samples).
constexpr int kAutoTcForm = CC_MERGE_F16X3;
// CC_MERGE_AUTO merges complex128 plans with the Ozaki tensor-core form from
// this many terms on (both factors >= 2^7 amplitudes).
constexpr int64_t kAutoOzakiMinTerms = 2;
struct BMergeJob {
  int32_t a_buf, b_buf, out_buf, kind;  // kind: 0 tiled, 1 flat
  int64_t a_off, b_off, out_off;
  int32_t qa, qb;
  int64_t K, Z, out_stride;
  const int32_t* aidx;
  const int32_t* bidx;
  int64_t unit_begin, n_units;
  int32_t circ;  // circuit whose output this stage completes (-1: intermediate)
  int32_t pad;
};
// Writes %globaltimer to *out once the stream reaches it.
cc_status launch_stamp(unsigned long long* out, void* stream);
// Work units of a batched merge job for the given tile rows (16 or 32).
int64_t merge_batch_units(int precision, int qa, int qb, int64_t Z, int rows, int32_t* kind);
// One launch over every job of one merge level.  circ_done counts finished
// units per circuit (zeroed by the caller); when a circuit's final stage
// completes, stamps[1 + circ] receives %globaltimer.
cc_status launch_merge_batch(const BMergeJob* jobs, int n_jobs, int64_t n_units, void* seg_buf,
                             void* work, void* psi, int* circ_done, unsigned long long* stamps,
                             int precision, int rows, void* stream);

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

// Complex128 tensor-core merge (Ozaki scheme, merge_ozaki.cu): same shapes as
// the tensor-core merge; returns 0 bytes / CC_EUNSUPPORTED where it does not apply.
uint64_t merge_ozaki_workspace_bytes(int qa, int qb, int64_t K);
cc_status launch_merge_ozaki(const MergeStage& st, void* workspace, uint64_t ws_bytes,
                             void* stream);

// ----------------------------------------------------------- reductions
cc_status launch_compare(const void* a, const void* b, int64_t n, int precision, double* out_dev,
                         double* partials, int n_blocks, void* stream);
// SM-driven copy of `bytes` from device memory to a host buffer's mapped address.
cc_status launch_copy_to_host(const void* src, void* host_mapped, uint64_t bytes, void* stream);
// One bounded wait on a word nothing writes: raises the device error flag.
cc_status launch_expired_wait(int polls, void* stream);
cc_status launch_gather(const void* psi, int precision, const int64_t* idx_dev, int64_t n,
                        void* out_dev, void* stream);

// --------------------------------------------------------------- device
cc_status check_device();
int num_sms();
void* scratch(size_t bytes);  // per-device library scratch (grown on demand)
int* device_error_flag();     // per-device int set by kernels whose bounded waits expire

}  // namespace cc
