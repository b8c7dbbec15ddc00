/*
 * cutsim.h -- C ABI of the GB300 (sm_103a) circuit-cutting state-vector engine.
 *
 * The engine computes, for a circuit C on q qubits and a partition of the
 * qubits into n contiguous segments, the full 2^q-amplitude state C|0...0>
 * in two ways:
 *
 *   cut   : cc_plan_create        -- preprocessing, Algorithm 1 (T_pre)
 *           cc_simulate_segments  -- subcircuit simulation, Algorithm 2 (T_sub)
 *           cc_merge              -- merging, Algorithm 3 (T_merge)
 *   uncut : cc_uncut_create + cc_simulate_uncut   -- T_orig of Eq. 3
 *
 * and verifies results with FP64 device reductions (cc_compare, cc_gather).
 *
 * Conventions (shared by every entry point)
 *   - Amplitude index x = sum_j x_j 2^j: qubit j is bit j (little-endian).
 *   - Segment i holds the contiguous qubits [seg_start[i], seg_start[i]+q_i),
 *     segment 0 the lowest; all (sub)circuits start in |0...0>.
 *   - State vectors are interleaved complex: float2 (CC_C64, 8 bytes per
 *     amplitude) or double2 (CC_C128, 16 bytes per amplitude).
 *   - Every device pointer must be 16-byte aligned device memory of the
 *     current device; `stream` is a cudaStream_t (NULL = legacy default
 *     stream) and every launch is asynchronous on it unless stated otherwise.
 *   - The caller owns every buffer it passes.  The library owns the plan
 *     objects, their small device tables, and a per-device scratch area for
 *     reductions.
 *   - Errors: every call returns a cc_status; nothing throws across the ABI.
 *     Arguments are validated before any launch.  cc_last_error() returns a
 *     thread-local message describing the last failure on the calling thread.
 *
 * Only sm_103 devices are accepted (CC_EDEVICE otherwise): the kernels are
 * compiled for sm_103a alone.
 */
#ifndef CUTSIM_H
#define CUTSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CC_MAX_QUBITS 34   /* 2^34 complex64 = 128 GiB */
#define CC_MAX_SEGMENTS 8
#define CC_MAX_CUTS 24     /* cut bits <= 24, at most 2^24 merge terms */

typedef enum {
  CC_OK = 0,
  CC_EINVAL = 1,        /* malformed argument: NULL pointer, unknown enum, qubit out of range, q0 == q1 */
  CC_ERANGE = 2,        /* size beyond the supported range (q, segment count, c_total, index) */
  CC_EUNSUPPORTED = 3,  /* the cutter cannot decompose the circuit (see cc_plan_create) */
  CC_ENOMEM = 4,        /* host or device allocation of library-owned tables failed */
  CC_EBUFSIZE = 5,      /* a caller buffer is smaller than required */
  CC_ECUDA = 6,         /* a CUDA runtime call or launch failed (see cc_last_error) */
  CC_ETIMEOUT = 7,      /* a bounded device-side wait gave up; outputs are undefined */
  CC_EDEVICE = 8        /* the current device is not an sm_103 GPU */
} cc_status;

typedef enum { CC_C64 = 0, CC_C128 = 1 } cc_precision;

/* Rank-2 decompositions of a cut CZ (Eq. 1 with k = 2).
 * CC_DECOMP_PROJECTOR: CZ = |0><0| (x) I + |1><1| (x) Z, coefficients 1 and 1.
 * CC_DECOMP_S_SDG    : Eq. 2, CZ = [S (x) S + i S^dag (x) S^dag] / (1 + i).
 * A boundary CX is first rewritten as (I (x) H) CZ (I (x) H) (Sec. II.A.2). */
typedef enum { CC_DECOMP_PROJECTOR = 0, CC_DECOMP_S_SDG = 1 } cc_decomp;

/* Merge arithmetic (cc_merge).
 * CC_MERGE_FMA     : complex FMA on CUDA cores in the plan's precision.
 * CC_MERGE_TF32X3  : tcgen05 tensor cores, kind::tf32, each operand split
 *                    x = hi + lo and hi*hi + hi*lo + lo*hi accumulated in FP32,
 *                    at most 64 terms per tensor-core accumulation (longer K
 *                    adds its 64-term partial sums with FP32 tensor
 *                    reduce-add stores) (CC_C64 plans, both factors >= 2^7
 *                    amplitudes; max|dpsi|/max|psi| <= 2e-6).
 * CC_MERGE_BF16X3  : tcgen05 tensor cores, kind::f16 with bf16 operands, the
 *                    same three-product split, FP32 accumulation (CC_C64,
 *                    factors >= 2^7; max|dpsi|/max|psi| <= 5e-5).
 * CC_MERGE_F16X3   : tcgen05 tensor cores, kind::f16 with fp16 operands: each
 *                    operand scaled by a power of two (its largest entry just
 *                    below 1, so no entry leaves fp16's range), split
 *                    x = hi + lo in fp16 and hi*hi + hi*lo + lo*hi accumulated
 *                    in FP32, at most 128 terms per accumulation up to
 *                    K = 256 and 64 beyond (longer K adds the partial sums
 *                    with FP32 tensor reduce-add stores), the two scales
 *                    undone in the epilogue: the significands
 *                    of 3xTF32 (11 bits each) in half the operand bytes at
 *                    twice the tensor rate (CC_C64 plans, both factors >= 2^7
 *                    amplitudes; max|dpsi|/max|psi| <= 2e-6).
 * CC_MERGE_OZAKI   : complex128 on tcgen05 tensor cores (CC_C128 plans, both
 *                    factors >= 2^7 amplitudes): every operand row scaled by a
 *                    power of two and cut into 6 bf16 slices of 9 bits, the
 *                    21 leading slice products accumulated in FP32 (the
 *                    leading levels exactly) and summed exactly in 64-bit
 *                    fixed point, then rounded once to FP64 (the Ozaki
 *                    scheme: Ozaki, Ogita, Oishi, Rump 2012); long K adds its
 *                    64-term groups exactly through the output buffer
 *                    (max|dpsi|/max|psi| <= 1e-12; measured about 2e-13 for
 *                    K <= 64 and 2e-14 beyond).
 * CC_MERGE_AUTO    : complex64: F16X3 where it applies and K >= 8, else FMA;
 *                    complex128: OZAKI where it applies, else FMA.
 * For n_seg >= 3 the form applies to the last (2^q-sized) stage of the chain;
 * the earlier, smaller stages always use FMA. */
typedef enum {
  CC_MERGE_AUTO = 0,
  CC_MERGE_FMA = 1,
  CC_MERGE_TF32X3 = 2,
  CC_MERGE_BF16X3 = 3,
  CC_MERGE_OZAKI = 4,
  CC_MERGE_F16X3 = 5
} cc_merge_form;

typedef enum {
  CC_GATE_U3 = 0,  /* U3(theta,phi,lambda) = [[c, -e^{i l} s], [e^{i p} s, e^{i(p+l)} c]], c=cos(theta/2), s=sin(theta/2) */
  CC_GATE_H = 1,
  CC_GATE_X = 2,
  CC_GATE_Z = 3,
  CC_GATE_S = 4,   /* diag(1, i) */
  CC_GATE_SDG = 5, /* diag(1, -i) */
  CC_GATE_T = 6,   /* diag(1, e^{i pi/4}) */
  CC_GATE_TDG = 7, /* diag(1, e^{-i pi/4}) */
  CC_GATE_CZ = 8,  /* diag(1, 1, 1, -1) on (q0, q1) */
  CC_GATE_CX = 9,  /* control q0, target q1 */
  /* Schmidt rank 4 (Eq. 1 with k = 4), basis |x_q0 x_q1>: */
  CC_GATE_SWAP = 10,  /* exchanges x_q0 and x_q1 */
  CC_GATE_ISWAP = 11, /* SWAP with a factor i on |01> and |10> */
  CC_GATE_CAN = 12    /* exp(-i (tx XX + ty YY + tz ZZ) / 2), (tx, ty, tz) = (theta, phi, lambda) */
} cc_gate_kind;

/* One gate.  q1 = -1 for one-qubit gates; theta, phi, lambda are read for U3
 * and CAN only.  40 bytes, natural alignment. */
typedef struct {
  int32_t kind;
  int32_t q0;
  int32_t q1;
  int32_t reserved;  /* must be 0 */
  double theta, phi, lambda;
} cc_gate;

typedef struct cc_plan cc_plan;    /* opaque, library-owned */
typedef struct cc_uncut cc_uncut;  /* opaque, library-owned */

typedef struct {
  int32_t q, n_seg, c_total, precision, decomp;
  int32_t seg_qubits[CC_MAX_SEGMENTS];  /* q_i */
  int32_t seg_start[CC_MAX_SEGMENTS];   /* first qubit of segment i */
  int32_t seg_cuts[CC_MAX_SEGMENTS];    /* c_i: variant bits of segment i (1 per adjacent rank-2 cut, 2 per rank-4) */
  int32_t seg_passes[CC_MAX_SEGMENTS];  /* gate passes of segment i's program */
  int32_t seg_ops[CC_MAX_SEGMENTS];     /* fused gate operations of segment i */
  int64_t seg_offset[CC_MAX_SEGMENTS];  /* amplitude offset of segment i in seg_buf */
  int64_t n_sub;                        /* N_sub = sum_i 2^{c_i} */
  uint64_t seg_buf_bytes;               /* bytes of seg_buf: sum_i 2^{c_i} 2^{q_i} amplitudes */
  uint64_t psi_bytes;                   /* bytes of the 2^q output */
  uint64_t workspace_bytes;             /* device workspace cc_merge needs (any form) */
  uint64_t table_bytes;                 /* device bytes of the plan's own tables */
  int32_t cut_bits;                     /* merge terms = 2^cut_bits: 1 bit per rank-2 cut, 2 per rank-4 cut */
  int32_t reserved0;
} cc_plan_info_t;

/* cc_plan_create -- preprocessing, Algorithm 1 (T_pre).
 *   gates[n_gates]  host array, read during the call only.
 *   q               1..CC_MAX_QUBITS.
 *   seg_sizes[n_seg] host array, positive, summing to q; n_seg in 1..CC_MAX_SEGMENTS.
 *   decomp          cc_decomp;  precision  cc_precision.
 *   out             receives a plan the caller frees with cc_plan_destroy.
 * Every two-qubit gate whose qubits lie in different segments becomes cut j
 * (j in circuit order).  Segment i gets one shared gate program whose
 * variants differ only in the diagonal local terms selected by the variant's
 * bits for each adjacent cut; the coefficient of cut j is folded into the
 * term on the segment of the gate's first qubit, so merging needs no alpha_m.
 * A CZ or CX cut (rank 2) takes one variant bit.  A SWAP, ISWAP or CAN cut
 * (rank 4) is expanded in Pauli products, sum over (a, b) of w_ab
 * (X^a Z^b) (x) (X^a Z^b), X^a applied as H Z^a H, and takes two variant
 * bits (one when only one of them carries weight).  Inside a segment (or in
 * the uncut program) these gates run as X/Y/Z-basis changes around diagonal
 * ZZ phases.
 * The plan's tables are uploaded to the current device (synchronously).
 * Segments 2..n_seg compile on threads the call starts and joins before it
 * returns (a segment whose thread cannot be started compiles on the calling
 * thread); the programs do not depend on the threads' timing.
 * Errors: CC_EINVAL (NULL, bad enum, bad qubit, sizes not summing to q),
 * CC_ERANGE (q, n_seg or c_total too large, a segment too large to simulate),
 * CC_EUNSUPPORTED (for n_seg >= 3, a cut between non-adjacent segments),
 * CC_ENOMEM, CC_ECUDA, CC_EDEVICE. */
cc_status cc_plan_create(const cc_gate* gates, int32_t n_gates, int32_t q,
                         const int32_t* seg_sizes, int32_t n_seg, int32_t decomp,
                         int32_t precision, cc_plan** out);

/* cc_plan_info -- sizes and counts of a plan (host only, no device work). */
cc_status cc_plan_info(const cc_plan* plan, cc_plan_info_t* info);

/* cc_plan_cut -- the j-th cut: its two qubits (first, second as in the gate),
 * its kind (CC_GATE_CZ or CC_GATE_CX) and the two segments. */
cc_status cc_plan_cut(const cc_plan* plan, int32_t j, int32_t* q0, int32_t* q1,
                      int32_t* kind, int32_t* seg0, int32_t* seg1);

void cc_plan_destroy(cc_plan* plan);

/* cc_simulate_segments -- subcircuit simulation, Algorithm 2 (T_sub).
 * Writes |psi_i^(r)> = S_i^(r)|0> for every segment i and variant r into
 * seg_buf: segment i occupies amplitudes [seg_offset[i], seg_offset[i] +
 * 2^{c_i} 2^{q_i}), variant r at seg_offset[i] + r 2^{q_i}.  Bit t of r
 * selects the term of the t-th cut adjacent to segment i (circuit order).
 * seg_buf_bytes must be >= info.seg_buf_bytes (else CC_EBUFSIZE).
 * All passes of all segments run in one persistent launch (a queue of
 * (pass, tile) items, each pass waiting with a bounded poll for the previous
 * pass of its segment); its per-run counters live in the plan, so calls on
 * one plan must not overlap in time (use one plan per concurrent stream).
 * CUTSIM_SEG_LAUNCH=passes selects one launch per pass instead.
 * Asynchronous on `stream`; an expired wait is reported by cc_sync. */
cc_status cc_simulate_segments(const cc_plan* plan, void* seg_buf, uint64_t seg_buf_bytes,
                               void* stream);

/* cc_merge -- merging, Algorithm 3 (T_merge).
 * psi[x] = sum_m prod_i psi_i^(r_i(m))[x restricted to segment i] over all
 * 2^{c_total} global cut combinations m (bit j of m = term of cut j).
 * n_seg = 2 is one pass over psi; n_seg >= 3 absorbs one segment at a time
 * through `workspace` (>= info.workspace_bytes, may be NULL when that is 0);
 * the tensor-core forms also stage their split operands there.
 * seg_buf is read only; psi (>= info.psi_bytes) is fully overwritten.
 * Errors: CC_EBUFSIZE, CC_EINVAL (form not available for the precision).
 * Asynchronous on `stream`. */
cc_status cc_merge(const cc_plan* plan, const void* seg_buf, uint64_t seg_buf_bytes,
                   void* psi, uint64_t psi_bytes, void* workspace, uint64_t workspace_bytes,
                   int32_t form, void* stream);

/* cc_uncut_create -- pass planning for the uncut simulation of C (host work,
 * tables uploaded synchronously).  Same gate rules as cc_plan_create. */
cc_status cc_uncut_create(const cc_gate* gates, int32_t n_gates, int32_t q, int32_t precision,
                          cc_uncut** out);

/* cc_program_image -- the gate program the uncut simulation of C would run,
 * as a host-side image for inspection and host tests; host work only (no
 * device needed).  Gates as for cc_uncut_create; tile_bits = 0 takes the
 * uncut default, else 2^tile_bits amplitudes per tile (more than the
 * precision's contiguous low tile bits, 4 for CC_C64 and 3 for CC_C128, and
 * at most 14 / 13), which forces more passes on small circuits.
 * words (int64, HOST): version 1, nq, n_state, passes, stages, ops, terms,
 *   mats, tabs; per pass nq, k, low, init_zero, stage_begin, stage_end,
 *   rbits, n_rest, zero_tile, zero_rest, 16 tile bits, 48 rest bits; per
 *   stage op_begin, op_end, 8 register tile bits; per op type, t,
 *   term_begin, n_sign, n_phase, n_table, mat, sign_adj (type 4, a packed
 *   rotation op: t = mask of register bits | mask of those in cotangent form
 *   << 8); per term kind, p0, p1, tab.  reals (double, HOST): the 2x2
 *   matrices (4 complex each; a rotation's t in the first real, a packed
 *   op's tangent of register bit i in real i) then the tables (4 complex
 *   each), re/im interleaved.  The meaning of each field is that of the device program
 *   the gate-pass kernels execute.
 * With words or reals NULL it only stores the sizes in *n_words, *n_reals;
 * CC_EBUFSIZE when the given capacities are too small. */
cc_status cc_program_image(const cc_gate* gates, int32_t n_gates, int32_t q, int32_t precision,
                           int32_t tile_bits, int64_t* words, int64_t* n_words, double* reals,
                           int64_t* n_reals);

/* cc_plan_program_image -- segment `seg`'s gate program of the plan
 * cc_plan_create would build for the same arguments (Algorithm 1's
 * subcircuit generation: one program over the 2^(q_seg + c_seg) amplitudes of
 * all its variants), as a host-side image for inspection and host tests;
 * host work only (no device needed).  tile_bits = 0 takes the segment
 * default, else the limits of cc_program_image.  words and reals as for
 * cc_program_image, followed in words by the plan's number of global cut
 * bits B, the segment's number of variant bits c_seg, and the global bit of
 * each of its variant bits in order (variant bit t of the segment is global
 * bit ids[t]; Algorithm 3 sums over all 2^B global combinations m, taking
 * from segment i the variant whose bit t is bit ids[t] of m), then the merge
 * stages the plan runs: their number and per stage seg, qa, qb, K, Z,
 * aidx_off, bidx_off (stage s: U_s[z][x_s 2^qa + x] = sum_{k < K}
 * U_{s-1}[tab[aidx_off + z K + k]][x] * seg_s[tab[bidx_off + z K + k]][x_s],
 * with U_0 the variants of segment 0), then the length of the index table
 * and its entries. */
cc_status cc_plan_program_image(const cc_gate* gates, int32_t n_gates, int32_t q,
                                const int32_t* seg_sizes, int32_t n_seg, int32_t decomp,
                                int32_t precision, int32_t tile_bits, int32_t seg,
                                int64_t* words, int64_t* n_words, double* reals,
                                int64_t* n_reals);

/* cc_kak_gates -- any two-qubit unitary as gates the library takes (host
 * work, no device).  Eq. 1 makes a general two-qubit gate a Schmidt-rank-4
 * cut; the canonical (Cartan, KAK) factorisation
 *   U = e^{i g} (A1 (x) B1) CAN(tx, ty, tz) (A0 (x) B0)
 * (Khaneja and Glaser 2001; Kraus and Cirac 2001) turns it into one-qubit
 * gates around a CC_GATE_CAN, which the cutter and the simulators take.
 *   u       host array of 32 doubles: the 4x4 unitary on (q0, q1), row-major,
 *           interleaved re/im, basis |x_q0 x_q1> (index 2 x_q0 + x_q1);
 *           read during the call only.
 *   q0, q1  distinct qubits in [0, CC_MAX_QUBITS).
 *   out     host array of at least 9 gates, written: U3 on q0, U3 on q1, CAN on
 *           (q0, q1), U3 on q0, U3 on q1, and (when the global phase is not
 *           0) U3 / X / U3 / X on q0 that multiply by e^{i g}; their product
 *           is u exactly up to rounding (global phase included).
 *   n_out   the number of gates written.
 * Errors: CC_EINVAL for NULL arguments, bad qubits, non-finite entries or a
 * matrix that is not unitary to 1e-10; CC_EUNSUPPORTED if the factorisation
 * fails its own checks (not seen for unitary input). */
#define CC_KAK_MAX_GATES 9
cc_status cc_kak_gates(const double* u, int32_t q0, int32_t q1, cc_gate* out, int32_t* n_out);

/* cc_uncut_info -- number of gate passes over the 2^q vector and of fused ops. */
cc_status cc_uncut_info(const cc_uncut* u, int32_t* n_passes, int32_t* n_ops, int32_t* tile_bits);

/* cc_simulate_uncut -- psi = C|0...0> over the full 2^q vector (T_orig).
 * psi_bytes >= 2^q * amplitude size.  Asynchronous on `stream`.  Complex128
 * gate passes compute in double-float (FP32 pairs, about 48 significant
 * bits; CUTSIM_C128_GATES=fp64 selects native FP64); the vector between
 * passes holds the pairs in the same 16 bytes per amplitude, and the last
 * pass writes complex128. */
cc_status cc_simulate_uncut(const cc_uncut* u, void* psi, uint64_t psi_bytes, void* stream);

void cc_uncut_destroy(cc_uncut* u);

/* cc_compare -- FP64 verification reductions over two device vectors of
 * n_amp amplitudes in `precision`:
 *   out[0] = max_x |a[x] - b[x]|     out[1] = max_x |b[x]|
 *   out[2] = Re <a|b>                out[3] = Im <a|b>
 *   out[4] = <a|a>                   out[5] = <b|b>
 * `out` is host memory.  Uses the library's per-device scratch area and
 * synchronizes `stream` before returning. */
cc_status cc_compare(const void* a, const void* b, int64_t n_amp, int32_t precision,
                     double* out, void* stream);

/* cc_gather -- out[i] = psi[idx[i]] for i < n_idx (the sampled-amplitude
 * check).  idx (int64) and out (n_idx amplitudes of `precision`) are HOST
 * memory; every index must lie in [0, n_amp) (else CC_ERANGE before any
 * launch).  n_idx <= 1<<20.  Synchronizes `stream`. */
cc_status cc_gather(const void* psi, int64_t n_amp, int32_t precision, const int64_t* idx,
                    int64_t n_idx, void* out, void* stream);

/* cc_gather_static -- cc_gather that allocates nothing.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory, such as a process whose GPU memory belongs to another allocator
 * (a framework's caching allocator, a fixed budget reserved at start-up) or a
 * latency-sensitive loop that cannot take the device-wide synchronisation
 * cudaMalloc/cudaFree may imply.  Same arguments, result and errors as
 * cc_gather, except:
 *   - indices and amplitudes are staged in a fixed device array that is part
 *     of the library image (CC_GATHER_STATIC_MAX entries, 1.5 MiB held on
 *     every GPU that loads the library until the process exits); n_idx above
 *     CC_GATHER_STATIC_MAX is rejected with CC_ERANGE before any device work;
 *   - every call looks up that array's device address (cudaGetSymbolAddress)
 *     with the caller's device current; the call synchronizes `stream`, so
 *     it cannot be recorded into a stream capture;
 *   - every call on a device shares the one array: calls whose device work
 *     overlaps (other threads, other streams) race and may return each
 *     other's amplitudes.  A call synchronizes `stream` before it returns, so
 *     calls made one after another from one thread never overlap.
 * It calls no cudaMalloc, cudaFree or other allocating routine. */
#define CC_GATHER_STATIC_MAX 65536
cc_status cc_gather_static(const void* psi, int64_t n_amp, int32_t precision, const int64_t* idx,
                           int64_t n_idx, void* out, void* stream);

/* ------------------------------------------------------------- batching
 * Batched cut simulation of many independent circuits.  The paper runs the
 * subcircuits of one circuit one after another and names running them in
 * parallel as a way to lower the effective threshold further (Sec. VI); it
 * also studies unequal partitions (supplementary Fig. 7).  A batch takes
 * n_circ circuits, each with its own q, gates and contiguous partition
 * (segments may differ in size), and runs
 *   - every pass of every segment program of every circuit in ONE persistent
 *     launch: a device queue of (job, tile) items, jobs ordered by pass
 *     number, each job waiting (bounded) until the pass before it on the same
 *     segment has stored all its tiles;
 *   - then one merge launch per chain level (one for n_seg = 2, two for
 *     n_seg = 3, ...), each over the output tiles of every circuit's stage at
 *     that level, on CUDA cores (CC_MERGE_FMA arithmetic); a circuit's final
 *     stage with K >= 8 terms and both factors >= 2^7 amplitudes (complex64)
 *     runs instead as its own tensor-core merge (3xFP16) after its level, as
 *     CC_MERGE_AUTO would run it (CUTSIM_BATCH_TC=0: all on CUDA cores).
 * The whole sequence can be captured once into a CUDA graph and replayed.
 *
 * Buffers (caller-owned device memory, 16-byte aligned): seg_buf holds every
 * circuit's segment vectors, psi every circuit's 2^q output (circuit i at
 * amplitude psi_offset(i), see cc_batch_circuit), workspace the chained-merge
 * intermediates of circuits with n_seg >= 3.  Sizes come from cc_batch_info.
 */
typedef struct cc_batch cc_batch;  /* opaque, library-owned */

typedef struct {
  int32_t n_circ;
  int32_t precision;
  int32_t tile_bits;       /* largest segment tile (bits) the programs were planned with */
  int32_t merge_rows;      /* output rows per merge tile (16 or 32; complex128 always 32) */
  int32_t n_jobs;          /* segment passes in the persistent launch */
  int32_t merge_levels;    /* merge launches per run */
  int64_t n_items;         /* tiles in the persistent launch's queue */
  int64_t n_sub;           /* subcircuits (variants) over all circuits */
  uint64_t seg_buf_bytes;
  uint64_t psi_bytes;
  uint64_t workspace_bytes;
  int32_t block;           /* threads per CTA of the persistent launch */
  int32_t grid;            /* CTAs of the persistent launch */
} cc_batch_info_t;

/* cc_batch_create -- plan every circuit (Algorithm 1 per circuit) and build
 * the batched launch.
 *   gates             all circuits' gates, circuit i at gates[gate_offset[i] ..
 *                     gate_offset[i+1]); host memory, read during the call.
 *   gate_offset[n_circ+1], q[n_circ], seg_sizes[seg_offset[n_circ]],
 *   seg_offset[n_circ+1]: host arrays; circuit i's segments are
 *                     seg_sizes[seg_offset[i] .. seg_offset[i+1]), at least 2,
 *                     summing to q[i].
 *   tile_bits         0 = the default segment tile, else 5..14 (complex64) or
 *                     4..13 (complex128): the largest tile of a segment pass.
 *   merge_rows        0 = 32, else 16 or 32.
 * Each circuit obeys the rules of cc_plan_create.  n_circ in 1..65536.
 * Errors: those of cc_plan_create (naming the circuit), CC_EINVAL for
 * malformed offsets or a circuit with fewer than 2 segments. */
cc_status cc_batch_create(const cc_gate* gates, const int64_t* gate_offset, int32_t n_circ,
                          const int32_t* q, const int32_t* seg_sizes, const int32_t* seg_offset,
                          int32_t decomp, int32_t precision, int32_t tile_bits,
                          int32_t merge_rows, cc_batch** out);

cc_status cc_batch_info(const cc_batch* b, cc_batch_info_t* info);

/* cc_batch_circuit -- circuit i's output offset in psi (amplitudes), q,
 * c_total and its number of subcircuits. */
cc_status cc_batch_circuit(const cc_batch* b, int32_t i, int64_t* psi_offset, int32_t* q,
                           int32_t* c_total, int64_t* n_sub);

/* cc_batch_run -- simulate and merge every circuit of the batch (asynchronous
 * on `stream`).  stamps: optional device array of n_circ + 1 uint64 that
 * receives %globaltimer (ns) when the persistent launch takes its first tile
 * (stamps[0]) and when the last store of circuit i's output has been issued
 * (stamps[1 + i]; the stores land within their memory latency after it).
 * Stamping costs one counter update per merge tile.
 * Errors: CC_EBUFSIZE, CC_EINVAL; a dependency wait that gives up is
 * reported by cc_sync as CC_ETIMEOUT. */
cc_status cc_batch_run(const cc_batch* b, void* seg_buf, uint64_t seg_buf_bytes, void* psi,
                       uint64_t psi_bytes, void* workspace, uint64_t workspace_bytes,
                       uint64_t* stamps, void* stream);

/* cc_batch_capture -- record cc_batch_run with these buffers into a CUDA
 * graph owned by the batch (replacing any earlier one).  `stream` must be a
 * stream other than the legacy NULL stream; nothing runs during the call.
 * The buffers are baked into the graph and must outlive it. */
cc_status cc_batch_capture(cc_batch* b, void* seg_buf, uint64_t seg_buf_bytes, void* psi,
                           uint64_t psi_bytes, void* workspace, uint64_t workspace_bytes,
                           uint64_t* stamps, void* stream);

/* cc_batch_launch -- replay the captured graph on `stream` (CC_EINVAL if none). */
cc_status cc_batch_launch(const cc_batch* b, void* stream);

/* cc_batch_autotune -- time cc_batch_run on these buffers for every segment
 * tile width in 10..max (complex64 14, complex128 13) and every merge tile
 * height (16, 32; complex128 32 only), re-planning the batch for each, and
 * keep the fastest.  Writes up to max_out candidates (tile bits, merge rows,
 * mean ms over 3 timed runs after one warm-up) and their count to *n_out.
 * Synchronizes `stream`; any captured graph is discarded. */
cc_status cc_batch_autotune(cc_batch* b, void* seg_buf, uint64_t seg_buf_bytes, void* psi,
                            uint64_t psi_bytes, void* workspace, uint64_t workspace_bytes,
                            void* stream, int32_t max_out, int32_t* n_out, int32_t* tile_bits,
                            int32_t* merge_rows, float* ms);

void cc_batch_destroy(cc_batch* b);

/* ------------------------------------------------------ learned planner
 * A small fully connected FP32 network (hand-written forward, backward and
 * Adam kernels) that the planner trains on stage times measured on this GPU
 * and uses to choose cut/no-cut and the segment count; the closed-form
 * thresholds (Eqs. 13-14) are its fallback.  Layers map dims[l] ->
 * dims[l+1], l < n_layers (1..8 layers, widths 1..1024); hidden layers use
 * ReLU, the last is linear.  params (device, float) packs per layer
 * W_l (dims[l+1] x dims[l], row-major) then b_l; inputs x are n x dims[0]
 * row-major, outputs n x dims[n_layers].  work is a device scratch of
 * cc_mlp_work_bytes(dims, n_layers, n) bytes. */
int64_t cc_mlp_param_count(const int32_t* dims, int32_t n_layers);  /* -1 on bad dims */
uint64_t cc_mlp_work_bytes(const int32_t* dims, int32_t n_layers, int64_t n); /* 0 on bad dims */

/* cc_mlp_forward -- y = net(x) for n samples (asynchronous on `stream`). */
cc_status cc_mlp_forward(const int32_t* dims, int32_t n_layers, const float* params,
                         const float* x, int64_t n, float* y, float* work, uint64_t work_bytes,
                         void* stream);

/* cc_mlp_train -- `epochs` full-batch Adam steps (beta1 0.9, beta2 0.999,
 * eps 1e-8, step lr) on the mean squared error between net(x) and the
 * targets t (n x dims[n_layers]).  params, adam_m, adam_v (zero-initialised
 * by the caller for a fresh run) are updated in place; each call counts its
 * steps from 1 for Adam's bias correction; loss (device, may be NULL)
 * receives the loss of every epoch before its update. */
cc_status cc_mlp_train(const int32_t* dims, int32_t n_layers, float* params, float* adam_m,
                       float* adam_v, const float* x, const float* t, int64_t n, int32_t epochs,
                       float lr, float* loss, float* work, uint64_t work_bytes, void* stream);

/* cc_sync -- synchronize `stream`, then report CC_ETIMEOUT if any kernel of
 * this library on the current device gave up a bounded wait since the last
 * cc_sync (the flag is cleared by the call).  Asynchronous entry points
 * cannot return that status themselves. */
cc_status cc_sync(void* stream);

/* cc_copy_to_host -- copy `bytes` from device memory to host memory (a
 * result vector to the caller).  For a page-locked host buffer that is mapped
 * into the device address space (cudaHostAlloc / pinned allocations under
 * unified addressing) the SMs copy it with 16-byte loads and stores through
 * the mapped address, which on a Grace host runs over NVLink-C2C faster than
 * one copy engine; any other host buffer goes through cudaMemcpyAsync.  Both
 * pointers 16-byte aligned.  Asynchronous on `stream`. */
cc_status cc_copy_to_host(const void* src, void* host, uint64_t bytes, void* stream);

/* cc_check_wait_expiry -- exercise the failure path of the bounded device
 * waits without any fault: one thread polls a device word that nothing
 * writes, `polls` times (1..2^20, about 1 us apart), gives up and raises the
 * device error flag exactly as an expired wait in the engine does; the next
 * cc_sync on the stream then returns CC_ETIMEOUT and clears the flag.
 * Asynchronous on `stream`. */
cc_status cc_check_wait_expiry(int32_t polls, void* stream);

/* cc_last_error -- thread-local message of the last failure (never NULL). */
const char* cc_last_error(void);

/* cc_version -- library version string. */
const char* cc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CUTSIM_H */
