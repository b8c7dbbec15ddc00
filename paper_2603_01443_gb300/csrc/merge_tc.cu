// Merging (Algorithm 3) on tcgen05 tensor cores.
//
// The two-factor merge psi[y * NA + x] = sum_k A_k[x] B_k[y] is one real GEMM
//   C[y][n] = sum_kk R[y][kk] * Cop[n][kk],   n = 2x + (0: real, 1: imaginary)
// with kk < K holding real parts and K <= kk < 2K imaginary parts:
//   R[y][k] = Re B_k[y],          R[y][K+k] = Im B_k[y]
//   Cop[2x][k] = Re A_k[x],       Cop[2x][K+k] = -Im A_k[x]
//   Cop[2x+1][k] = Im A_k[x],     Cop[2x+1][K+k] = Re A_k[x]
// so that C, stored row-major in FP32, is psi in interleaved complex64.
// Every operand is split x = hi + lo (bf16 + bf16, or tf32 + tf32) and the
// kernel accumulates hi*hi + hi*lo + lo*hi in FP32 (Markidis et al. 2018,
// "NVIDIA tensor core programmability, performance & precision").
//
// Kernel structure (one CTA per SM, persistent over 128 x 256 output tiles):
//   warp 0      TMA producer: per 128-byte K block, loads R_hi, R_lo (128 rows)
//               and C_hi, C_lo (256 rows) with 128-byte swizzle into one of two
//               96 KB shared-memory stages;
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32 accumulators)
//               and one lane issues the tcgen05.mma instructions;
//   warps 2..5  epilogue: tcgen05.ld of the finished accumulator in 32 x 32
//               blocks, staged through shared memory and written by bulk
//               tensor stores (TMA), then release of the accumulator, so the
//               store of tile i overlaps the MMAs of tile i+1 (3xFP16 with
//               K <= 32: warps 2..9, two per TMEM lane quarter, with K in
//               three 64-byte stages).
// Forms: merge_tc_kernel (the structure above, streaming K in 128-, 64- or
// 32-byte blocks through 2, 4 or 8 stages of the same 192 KB), the default;
// merge_tc_rs_kernel (row operand resident in shared memory), opt-in and
// slower on GB300.  No form shares a load between CTAs: each CTA fetches its
// own operand tiles from L2.
// Every mbarrier wait is bounded: on expiry the kernel raises a device error
// flag (reported as CC_ETIMEOUT by cc_sync), waits a bounded time for its own
// copies and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "tcgen05_util.cuh"

namespace cc {

namespace {

using namespace tcg;

constexpr int BM = 128;            // rows (y) per tile
constexpr int BN = 256;            // real columns per tile (128 complex amplitudes)
constexpr int KB_BYTES = 128;      // bytes of K per stage (one swizzle atom row)
constexpr int STAGES = 2;
constexpr int R_TILE = BM * KB_BYTES;  // 16 KB
constexpr int C_TILE = BN * KB_BYTES;  // 32 KB
constexpr int STAGE_BYTES = 2 * R_TILE + 2 * C_TILE;  // 96 KB
constexpr int STG_BYTES = 32 * 128;  // one epilogue store box: 32 rows x 32 FP32
constexpr int STG_TOTAL = 4 * 2 * STG_BYTES;  // 4 epilogue warps x 2 buffers
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STG_TOTAL + 1024 /*align*/ + 256 /*barriers*/;
constexpr int TMEM_COLS = 512;
constexpr int SMEM_LIMIT = 232448;  // opt-in dynamic shared memory per CTA on sm_103
// 3xTF32 stays within 2e-6 relative while one tensor-core accumulation runs
// over at most 2 x 64 real products; longer K is summed in groups of that length.
constexpr int64_t kTf32GroupTerms = 64;
// 3xFP16 (22-bit operand splits) measured against complex128 results: at
// K = 256 one accumulation over 128 terms errs as little as over 64 (5.9e-7
// and 7.9e-7 of max |psi| at q = 24 and 26) and merges 31 % faster at q = 30;
// at K = 1024 128-term groups err 1.5e-6 against 1.1e-6, so longer K keeps 64.
__host__ __device__ constexpr int64_t f16_group_terms(int64_t K) { return K <= 256 ? 128 : 64; }

// Instruction descriptor: FP32 accumulator, K-major A and B, M = 128, N = 256.
template <int KIND>
__host__ __device__ constexpr uint32_t idesc_value() {
  return (1u << 4)                                            // D format: F32
         | ((KIND == CC_MERGE_F16X3 ? 0u : KIND == CC_MERGE_BF16X3 ? 1u : 2u) << 7)   // A: F16 / BF16 / TF32
         | ((KIND == CC_MERGE_F16X3 ? 0u : KIND == CC_MERGE_BF16X3 ? 1u : 2u) << 10)  // B format
         | ((uint32_t)(BN >> 3) << 17)                        // N / 8
         | ((uint32_t)(BM >> 4) << 24);                       // M / 16
}

// Output tiles are visited in bands of kBand row tiles: inside a band the
// row index runs fastest, so a column-operand tile is used by kBand row tiles
// back to back and the row-operand tiles of the band stay in L2 while the
// band sweeps the columns.  Measured at q = 30 with 3xFP16 (band of 16 ->
// 64): K = 16 1.53 -> 1.37 ms, K = 64 1.61 -> 1.57 ms; 8 and 128 were slower.
constexpr int kBand = 64;
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int& m0, int& n0) {
  const int band = t / (kBand * tiles_n), r = t - band * kBand * tiles_n;
  const int rows = min(kBand, tiles_m - band * kBand);
  m0 = (band * kBand + r % rows) * BM;
  n0 = (r / rows) * BN;
}

// 2^e > the magnitude whose float bits are mb (e = 0 for an all-zero operand).
__device__ __forceinline__ int f16_scale_exp(unsigned int mb) {
  return mb ? (int)((mb >> 23) & 0xFF) - 126 : 0;
}

// Long K runs in groups of group_kb K blocks: each group accumulates into a
// fresh TMEM accumulator and the epilogue writes group 0 with plain tensor
// stores and adds every later group with tensor reduce-add stores (FP32 adds
// in L2, after the warp's earlier stores of the tile have completed), so no
// single tensor-core accumulation runs longer than group_kb K blocks.
//
// KBB bytes of K per stage (the swizzle width) and NST stages: the operand
// buffers hold NST * (2 * BM + 2 * BN) * KBB bytes (192 KB for 128 x 2 and
// 64 x 4); narrower, more numerous stages keep more loads in flight while the
// tensor cores read one.  Every CTA loads its own operand tiles: no load is
// shared between CTAs.
template <int KIND, int KBB, int NST, int EW = 4>
__global__ void __launch_bounds__(64 + 32 * EW, 1)
    merge_tc_kernel(const __grid_constant__ CUtensorMap map_r, const __grid_constant__ CUtensorMap map_c,
                    const __grid_constant__ CUtensorMap map_out, int n_rows, int n_cols,
                    int kblocks, int group_kb, int* err,
                    const unsigned int* __restrict__ f16_maxbits) {
  constexpr int RT = BM * KBB, CT = BN * KBB, STB = 2 * RT + 2 * CT;
  constexpr int STG_ALL = EW * 2 * STG_BYTES;  // epilogue staging: 2 boxes per warp
  static_assert(EW == 4 || EW == 8, "one or two epilogue warps per TMEM lane quarter");
  static_assert(EW == 8 || NST * STB == STAGES * STAGE_BYTES, "operand buffers of 192 KB");
  static_assert(NST * STB + STG_ALL + 1024 + 256 <= SMEM_LIMIT, "shared memory");
  static_assert((2 * NST + 8) * 8 <= 256, "barrier area");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* stg_base = smem + NST * STB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg_base + STG_ALL);
  uint64_t* full = bars;                  // [NST]
  uint64_t* empty = bars + NST;           // [NST]
  uint64_t* tfull = bars + 2 * NST;       // [2]
  uint64_t* tempty = bars + 2 * NST + 2;  // [2]
  uint64_t* drain = bars + 2 * NST + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * NST + 7);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = n_rows / BM, tiles_n = n_cols / BN;
  const int n_tiles = tiles_m * tiles_n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], EW);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_r)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_c)) : "memory");
      int s = 0;
      uint32_t use = 0;  // how many times the stage ring wrapped
      bool issued[NST];
      uint32_t issued_parity[NST];
      for (int i = 0; i < NST; ++i) {
        issued[i] = false;
        issued_parity[i] = 0;
      }
      bool ok = true;
      const int kelem = KIND != CC_MERGE_TF32X3 ? KBB / 2 : KBB / 4;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        int m0, n0;
        tile_coords(t, tiles_m, tiles_n, m0, n0);
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&empty[s], (use & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          unsigned char* st = smem + s * STB;
          const uint32_t fb = smem_u32(&full[s]);
          mbar_expect_tx(&full[s], STB);
          tma_load_2d(smem_u32(st), &map_r, fb, kb * kelem, m0);
          tma_load_2d(smem_u32(st + RT), &map_r, fb, kb * kelem, n_rows + m0);
          tma_load_2d(smem_u32(st + 2 * RT), &map_c, fb, kb * kelem, n0);
          tma_load_2d(smem_u32(st + 2 * RT + CT), &map_c, fb, kb * kelem, n_cols + n0);
          issued[s] = true;
          issued_parity[s] = use & 1;
          if (++s == NST) {
            s = 0;
            ++use;
          }
        }
      }
      if (!ok) {  // let our own copies land before the CTA exits
        for (int i = 0; i < NST; ++i)
          if (issued[i]) mbar_drain(&full[i], issued_parity[i]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_value<KIND>();
      int s = 0;
      uint32_t use = 0;
      int iter = 0;
      bool ok = true;
      bool any_mma = false;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int kb0 = 0; kb0 < kblocks && ok; kb0 += group_kb, ++iter) {
          const int a = iter & 1;
          if (!mbar_wait(&tempty[a], ((iter >> 1) & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dtmem = tmem_base + (uint32_t)(a * BN);
          const int kb1 = min(kblocks, kb0 + group_kb);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&full[s], use & 1, abort_flag, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = smem_u32(smem + s * STB);
            const uint64_t rh = sdesc_sw<KBB>(st), rl = sdesc_sw<KBB>(st + RT);
            const uint64_t ch = sdesc_sw<KBB>(st + 2 * RT), cl = sdesc_sw<KBB>(st + 2 * RT + CT);
#pragma unroll
            for (int k = 0; k < KBB / 32; ++k) {
              const uint64_t adv = (uint64_t)((k * 32) >> 4);
              umma<KIND>(dtmem, rh + adv, ch + adv, idesc, ((kb - kb0) | k) != 0);
              umma<KIND>(dtmem, rh + adv, cl + adv, idesc, 1);
              umma<KIND>(dtmem, rl + adv, ch + adv, idesc, 1);
            }
            any_mma = true;
            umma_commit(&empty[s]);  // frees the stage once these MMAs have read it
            if (++s == NST) {
              s = 0;
              ++use;
            }
          }
          if (!ok) break;
          umma_commit(&tfull[a]);  // accumulator a holds this group's sum
        }
      }
      if (!ok && any_mma) {  // let our own MMAs finish before TMEM is freed
        umma_commit(drain);
        mbar_drain(drain, 0);
      }
    }
  } else {
    // epilogue warps 2..1+EW: TMEM lane quarter = warp % 4 (with EW = 8 two
    // warps per quarter, each over half of the columns).  Each 32 x 32 block
    // of the accumulator goes TMEM -> registers -> a 128-byte-swizzled staging
    // buffer (conflict-free: a lane's row keeps its 16-byte chunks at j ^ (row & 7))
    // -> one bulk tensor store; two buffers keep one store in flight.
    const int quarter = warp & 3;
    const int ew = warp - 2;
    constexpr int CB = BN / 32 / (EW / 4);  // 32-column blocks per warp
    const int cb0 = (ew >> 2) * CB;
    unsigned char* stg = stg_base + ew * 2 * STG_BYTES;
    int buf = 0;
    int iter = 0;
    bool ok_all = true;
    // fp16 operands: the product of the two operand scales, 2^(e_R + e_C)
    const float osc = KIND == CC_MERGE_F16X3
                          ? __uint_as_float((uint32_t)(127 + f16_scale_exp(f16_maxbits[0]) +
                                                       f16_scale_exp(f16_maxbits[1])) << 23)
                          : 1.0f;
    for (int t = blockIdx.x; t < n_tiles && ok_all; t += gridDim.x) {
      int m0, n0;
      tile_coords(t, tiles_m, tiles_n, m0, n0);
      for (int kb0 = 0; kb0 < kblocks; kb0 += group_kb, ++iter) {
        const int a = iter & 1;
        // one lane waits, the warp follows its verdict (tcgen05.ld needs the whole warp)
        int ok = 1;
        if (lane == 0) ok = mbar_wait(&tfull[a], (iter >> 1) & 1, abort_flag, err) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          ok_all = false;
          break;
        }
        tc_fence_after();
        const bool add = kb0 > 0;  // later groups add onto the stored partial sums
        if (add) {
          if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
          __syncwarp();
        }
        const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * BN);
#pragma unroll 1
        for (int c2 = cb0; c2 < cb0 + CB; c2 += 2) {
          uint32_t rr[2][32];
          tmem_ld32x2(tbase + (uint32_t)(c2 * 32), rr[0], rr[1]);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = c2 + h;
            uint32_t(&r)[32] = rr[h];
            if (KIND == CC_MERGE_F16X3) {  // undo the operand scales (exact: a power of two)
#pragma unroll
              for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) * osc);
            }
            unsigned char* sb = stg + buf * STG_BYTES;
            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float4* dst = reinterpret_cast<float4*>(sb + lane * 128 + ((j ^ (lane & 7)) << 4));
              *dst = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                 __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
              if (add)
                asm volatile(
                    "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group"
                    " [%0, {%2, %3}], [%1];" ::"l"(reinterpret_cast<uint64_t>(&map_out)),
                    "r"(smem_u32(sb)), "r"(n0 + c * 32), "r"(m0 + quarter * 32)
                    : "memory");
              else
                asm volatile(
                    "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                        reinterpret_cast<uint64_t>(&map_out)),
                    "r"(smem_u32(sb)), "r"(n0 + c * 32), "r"(m0 + quarter * 32)
                    : "memory");
              asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
            buf ^= 1;
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[a]);
      }
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------- row-operand-stationary form
// For small K the whole row-operand tile (R_hi and R_lo of 128 rows, every K
// block) fits in shared memory.  Each CTA then takes a contiguous run of
// tiles -- runs of tiles_n tiles share one m -- keeps R resident while m is
// unchanged and streams only the column operand, one 32 KB block (C_hi or
// C_lo of one K block) per stage: two thirds of the operand bytes of the
// streaming form per output tile for 3xTF32.
constexpr int RS_C_STAGE = BN * KB_BYTES;  // 32 KB: one K block of C_hi or C_lo
constexpr int RS_MAX_STAGES = 4;

template <int KIND>
__global__ void __launch_bounds__(192, 1)
    merge_tc_rs_kernel(const __grid_constant__ CUtensorMap map_r,
                       const __grid_constant__ CUtensorMap map_c,
                       const __grid_constant__ CUtensorMap map_out, int n_rows, int n_cols,
                       int kblocks, int n_stages, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* r_buf = smem;                               // [2][kblocks][R_TILE]: hi, lo
  unsigned char* c_buf = smem + 2 * kblocks * R_TILE;        // [n_stages][RS_C_STAGE]
  unsigned char* stg_base = c_buf + n_stages * RS_C_STAGE;   // epilogue staging
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg_base + STG_TOTAL);
  uint64_t* full = bars;                        // [RS_MAX_STAGES]
  uint64_t* empty = bars + RS_MAX_STAGES;       // [RS_MAX_STAGES]
  uint64_t* tfull = bars + 2 * RS_MAX_STAGES;   // [2]
  uint64_t* tempty = tfull + 2;                 // [2]
  uint64_t* r_full = tempty + 2;
  uint64_t* r_empty = r_full + 1;
  uint64_t* drain = r_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(drain + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = n_cols / BN;
  const int n_tiles = (n_rows / BM) * tiles_n;
  const int t_begin = (int)(((int64_t)n_tiles * blockIdx.x) / gridDim.x);
  const int t_end = (int)(((int64_t)n_tiles * (blockIdx.x + 1)) / gridDim.x);

  if (threadIdx.x == 0) {
    for (int s = 0; s < n_stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);
    }
    mbar_init(r_full, 1);
    mbar_init(r_empty, 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int kelem = KIND != CC_MERGE_TF32X3 ? KB_BYTES / 2 : KB_BYTES / 4;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_r)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_c)) : "memory");
      int s = 0;
      uint32_t use = 0;
      uint32_t r_use = 0;
      int cur_m = -1;
      bool issued[RS_MAX_STAGES] = {false, false, false, false};
      uint32_t issued_parity[RS_MAX_STAGES] = {0, 0, 0, 0};
      bool r_issued = false;
      uint32_t r_parity = 0;
      bool ok = true;
      for (int t = t_begin; t < t_end && ok; ++t) {
        const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
        if (m0 != cur_m) {
          if (!mbar_wait(r_empty, (r_use & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          const uint32_t rb = smem_u32(r_full);
          mbar_expect_tx(r_full, 2 * kblocks * R_TILE);
          for (int kb = 0; kb < kblocks; ++kb) {
            tma_load_2d(smem_u32(r_buf + kb * R_TILE), &map_r, rb, kb * kelem, m0);
            tma_load_2d(smem_u32(r_buf + (kblocks + kb) * R_TILE), &map_r, rb, kb * kelem,
                        n_rows + m0);
          }
          r_issued = true;
          r_parity = r_use & 1;
          ++r_use;
          cur_m = m0;
        }
        for (int kb = 0; kb < kblocks && ok; ++kb) {
          for (int part = 0; part < 2; ++part) {
            if (!mbar_wait(&empty[s], (use & 1) ^ 1, abort_flag, err)) {
              ok = false;
              break;
            }
            mbar_expect_tx(&full[s], RS_C_STAGE);
            tma_load_2d(smem_u32(c_buf + s * RS_C_STAGE), &map_c, smem_u32(&full[s]), kb * kelem,
                        part ? n_cols + n0 : n0);
            issued[s] = true;
            issued_parity[s] = use & 1;
            if (++s == n_stages) {
              s = 0;
              ++use;
            }
          }
        }
      }
      if (!ok) {  // let our own copies land before the CTA exits
        for (int i = 0; i < n_stages; ++i)
          if (issued[i]) mbar_drain(&full[i], issued_parity[i]);
        if (r_issued) mbar_drain(r_full, r_parity);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_value<KIND>();
      int s = 0;
      uint32_t use = 0, r_use = 0;
      int cur_m = -1;
      int iter = 0;
      bool ok = true;
      bool any_mma = false;
      const uint32_t rh0 = smem_u32(r_buf), rl0 = smem_u32(r_buf + kblocks * R_TILE);
      for (int t = t_begin; t < t_end && ok; ++t, ++iter) {
        const int a = iter & 1;
        const int m0 = (t / tiles_n) * BM;
        if (!mbar_wait(&tempty[a], ((iter >> 1) & 1) ^ 1, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (m0 != cur_m) {
          if (cur_m >= 0) umma_commit(r_empty);  // the old R is free once its MMAs complete
          if (!mbar_wait(r_full, r_use & 1, abort_flag, err)) {
            ok = false;
            break;
          }
          ++r_use;
          cur_m = m0;
          tc_fence_after();
        }
        const uint32_t dtmem = tmem_base + (uint32_t)(a * BN);
        for (int kb = 0; kb < kblocks && ok; ++kb) {
          const uint64_t rh = sdesc(rh0 + kb * R_TILE), rl = sdesc(rl0 + kb * R_TILE);
          for (int part = 0; part < 2; ++part) {
            if (!mbar_wait(&full[s], use & 1, abort_flag, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t cd = sdesc(smem_u32(c_buf + s * RS_C_STAGE));
#pragma unroll
            for (int k = 0; k < KB_BYTES / 32; ++k) {
              const uint64_t adv = (uint64_t)((k * 32) >> 4);
              if (part == 0) {  // C_hi: R_hi * C_hi and R_lo * C_hi
                umma<KIND>(dtmem, rh + adv, cd + adv, idesc, (kb | k) != 0);
                umma<KIND>(dtmem, rl + adv, cd + adv, idesc, 1);
              } else {          // C_lo: R_hi * C_lo
                umma<KIND>(dtmem, rh + adv, cd + adv, idesc, 1);
              }
            }
            any_mma = true;
            umma_commit(&empty[s]);
            if (++s == n_stages) {
              s = 0;
              ++use;
            }
          }
        }
        if (!ok) break;
        umma_commit(&tfull[a]);
      }
      if (!ok && any_mma) {
        umma_commit(drain);
        mbar_drain(drain, 0);
      }
    }
  } else {
    const int quarter = warp & 3;
    unsigned char* stg = stg_base + quarter * 2 * STG_BYTES;
    int buf = 0;
    int iter = 0;
    for (int t = t_begin; t < t_end; ++t, ++iter) {
      const int a = iter & 1;
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&tfull[a], (iter >> 1) & 1, abort_flag, err) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
      const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * BN);
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t r[32];
        tmem_ld32(tbase + (uint32_t)(c * 32), r);
        unsigned char* sb = stg + buf * STG_BYTES;
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float4* dst = reinterpret_cast<float4*>(sb + lane * 128 + ((j ^ (lane & 7)) << 4));
          *dst = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                             __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          asm volatile(
              "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                  reinterpret_cast<uint64_t>(&map_out)),
              "r"(smem_u32(sb)), "r"(n0 + c * 32), "r"(m0 + quarter * 32)
              : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        buf ^= 1;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[a]);
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- operand split
__device__ __forceinline__ void split_store(uint16_t* hi, uint16_t* lo, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
  *hi = __bfloat16_as_ushort(h);
  *lo = __bfloat16_as_ushort(l);
}
__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ void split_store(uint32_t* hi, uint32_t* lo, float v) {
  const uint32_t h = to_tf32(v);
  *hi = h;
  *lo = to_tf32(v - __uint_as_float(h));
}

// fp16 operands carry one power-of-two scale per operand (R, Cop), chosen so
// that the operand's largest entry lies just below 1: every entry is within
// fp16's range (entries below 2^-14 of the largest are subnormal, with an
// absolute error below 2^-25 of it, far inside the complex64 tolerance, which
// is relative to max |psi|).  A first kernel finds the two largest magnitudes
// (atomic maxima of the non-negative float bits), the split kernel then
// writes v 2^-e = hi + lo in fp16, and the epilogue multiplies by 2^(e_R + e_C).

// The largest magnitude of each operand: blockIdx.y = 0 takes the row
// operand's values (the slices B[bidx[k]], k < K), 1 the column operand's (the
// slices A[aidx[k]]; Cop holds the same magnitudes), read in grid-stride
// order so every warp load is contiguous; one atomic maximum per block.
__global__ void __launch_bounds__(256)
    operand_absmax_f16(const float2* __restrict__ A, const float2* __restrict__ B, int qa, int qb,
                       int K, const int32_t* __restrict__ aidx, const int32_t* __restrict__ bidx,
                       unsigned int* __restrict__ maxbits) {
  __shared__ float s_mx[8];
  const bool is_r = blockIdx.y == 0;
  const int qn = is_r ? qb : qa;
  const float2* __restrict__ X = is_r ? B : A;
  const int32_t* __restrict__ idx = is_r ? bidx : aidx;
  const int64_t mask = (int64_t(1) << qn) - 1;
  const int64_t total = (int64_t)K << qn;
  float mx = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = X[((int64_t)idx[i >> qn] << qn) + (i & mask)];
    mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, s_mx[w]);
    if (mx > 0.f) atomicMax(maxbits + (is_r ? 0 : 1), __float_as_uint(mx));
  }
}

// The fp16 split, through a 64 x 64 shared-memory transpose: a block takes
// 64 operand rows (64 rows y of R, or 32 amplitudes x of A giving rows 2x and
// 2x+1 of Cop) and walks the padded K range in chunks of 64; each warp loads
// whole 32-amplitude runs of one slice (contiguous 256-byte reads), and the
// rows go out as contiguous 128-byte runs of hi and of lo.
constexpr int kSplitRows = 64;
__global__ void __launch_bounds__(256)
    split_operands_f16(const float2* __restrict__ A, const float2* __restrict__ B, int qa, int qb,
                       int K, int KR, const int32_t* __restrict__ aidx,
                       const int32_t* __restrict__ bidx, __half* __restrict__ r_ops,
                       __half* __restrict__ c_ops, const unsigned int* __restrict__ maxbits) {
  __shared__ float T[kSplitRows][kSplitRows + 1];
  const int64_t NA = int64_t(1) << qa, NB = int64_t(1) << qb;
  const int64_t r_blocks = NB / kSplitRows;
  const bool is_r = (int64_t)blockIdx.x < r_blocks;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = f16_scale_exp(maxbits[is_r ? 0 : 1]);
  const float down = __uint_as_float((uint32_t)(127 - e) << 23);  // 2^-e
  // first operand row of the block, and the first amplitude it reads
  const int64_t row0 = is_r ? (int64_t)blockIdx.x * kSplitRows
                            : ((int64_t)blockIdx.x - r_blocks) * kSplitRows;
  const int64_t amp0 = is_r ? row0 : row0 / 2;
  __half* const hi = is_r ? r_ops : c_ops;
  __half* const lo = is_r ? r_ops + NB * KR : c_ops + 2 * NA * KR;
  for (int c0 = 0; c0 < KR; c0 += kSplitRows) {
    for (int kl = warp; kl < kSplitRows; kl += 8) {
      const int kk = c0 + kl;
      const bool re = kk < K, used = kk < 2 * K;
      const int k = re ? kk : kk - K;
      if (is_r) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v = 0.f;
          if (used) {
            const float2 b = B[((int64_t)bidx[k] << qb) + amp0 + h * 32 + lane];
            v = re ? b.x : b.y;
          }
          T[h * 32 + lane][kl] = v * down;
        }
      } else {
        float v0 = 0.f, v1 = 0.f;
        if (used) {
          const float2 a = A[((int64_t)aidx[k] << qa) + amp0 + lane];
          v0 = re ? a.x : -a.y;  // row 2x
          v1 = re ? a.y : a.x;   // row 2x + 1
        }
        T[2 * lane][kl] = v0 * down;
        T[2 * lane + 1][kl] = v1 * down;
      }
    }
    __syncthreads();
    for (int r = warp; r < kSplitRows; r += 8) {
      const float v0 = T[r][2 * lane], v1 = T[r][2 * lane + 1];
      const __half h0 = __float2half_rn(v0), h1 = __float2half_rn(v1);
      const __half l0 = __float2half_rn(v0 - __half2float(h0));
      const __half l1 = __float2half_rn(v1 - __half2float(h1));
      const int64_t off = (row0 + r) * KR + c0 + 2 * lane;
      *reinterpret_cast<__half2*>(hi + off) = __halves2half2(h0, h1);
      *reinterpret_cast<__half2*>(lo + off) = __halves2half2(l0, l1);
    }
    __syncthreads();
  }
}

// One warp per operand row; lanes walk the padded K range.  Rows [0, NB) are
// the row operand R, rows [NB, NB + 2 NA) the column operand Cop.
template <typename E>
__global__ void __launch_bounds__(256)
    split_operands(const float2* __restrict__ A, const float2* __restrict__ B, int qa, int qb,
                   int K, int KR, const int32_t* __restrict__ aidx,
                   const int32_t* __restrict__ bidx, E* __restrict__ r_ops, E* __restrict__ c_ops) {
  const int64_t NA = int64_t(1) << qa, NB = int64_t(1) << qb;
  const int64_t rows = NB + 2 * NA;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  if (row < NB) {
    E* hi = r_ops + row * KR;
    E* lo = r_ops + (NB + row) * KR;
    for (int kk = lane; kk < KR; kk += 32) {
      float v = 0.f;
      if (kk < 2 * K) {
        const float2 b = B[(int64_t)bidx[kk % K] * NB + row];
        v = kk < K ? b.x : b.y;
      }
      split_store(hi + kk, lo + kk, v);
    }
  } else {
    const int64_t n = row - NB;
    const int64_t x = n >> 1;
    const int part = (int)(n & 1);
    E* hi = c_ops + n * KR;
    E* lo = c_ops + (2 * NA + n) * KR;
    for (int kk = lane; kk < KR; kk += 32) {
      float v = 0.f;
      if (kk < 2 * K) {
        const float2 a = A[(int64_t)aidx[kk % K] * NA + x];
        if (part == 0) v = kk < K ? a.x : -a.y;
        else v = kk < K ? a.y : a.x;
      }
      split_store(hi + kk, lo + kk, v);
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  }
  return fn;
}

// CUTSIM_TC_STATIONARY=1 selects the row-operand-stationary form where it
// applies.  It reads a third fewer operand bytes but keeps only 2-4 x 32 KB of
// loads in flight per SM against the streaming form's 2 x 96 KB, and on GB300
// the streaming form is faster (3xTF32, K = 64, q = 30: 2.86 vs 3.10 ms), so
// it is the default.
bool tc_stationary_requested() {
  const char* e = std::getenv("CUTSIM_TC_STATIONARY");
  return e && e[0] == '1';
}

// Bytes of K per stage (2, 4 or 8 stages for 128, 64 or 32).  Measured at
// q = 30 with the earlier two-CTA form of this kernel (merge ms, 128-byte /
// 64-byte blocks): a K loop of 4 to 8 128-byte blocks per tile ran faster in
// four 64-byte stages (3xTF32 K = 64: 2.64 / 2.41, K = 128: 4.67 / 4.64;
// split-BF16 K = 128: 2.72 / 2.50); shorter and longer loops ran faster in two
// 128-byte stages (3xTF32 K = 32: 1.55 / 1.62, K = 256: 8.76 / 9.36;
// split-BF16 K = 64: 1.59 / 1.65).  32-byte blocks were slower everywhere.
// CUTSIM_TC_KBLOCK = 128, 64 or 32 overrides.
int tc_kblock(int kblocks128) {
  const char* e = std::getenv("CUTSIM_TC_KBLOCK");
  if (e) {
    const int v = std::atoi(e);
    if (v == 128 || v == 64 || v == 32) return v;
  }
  return kblocks128 >= 4 && kblocks128 <= 8 ? 64 : 128;
}

CUtensorMapSwizzle swizzle_of(int kbb) {
  return kbb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                    : kbb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}

template <int KIND>
void* tc_kernel_ptr(int kbb) {
  if (kbb == 128) return reinterpret_cast<void*>(merge_tc_kernel<KIND, 128, 2>);
  if (kbb == 64) return reinterpret_cast<void*>(merge_tc_kernel<KIND, 64, 4>);
  return reinterpret_cast<void*>(merge_tc_kernel<KIND, 32, 8>);
}

constexpr int kEpi8Smem = 3 * (2 * BM + 2 * BN) * 64 + 8 * 2 * STG_BYTES + 1024 + 256;

// Eight epilogue warps for 3xFP16 merges whose K fits one 128-byte block
// (K <= 32): there the output stream, not the operand stream, sets the pace
// (q = 30, K = 16: 1.60 -> 1.50 ms), while at K = 64 the smaller operand
// stages cost more than the wider epilogue gains (1.60 -> 1.75 ms).
// CUTSIM_TC_EPI8 = 0 / 1 forces the choice.
bool epi8_for(int kr_bytes) {
  if (const char* e = std::getenv("CUTSIM_TC_EPI8")) return e[0] == '1';
  return kr_bytes <= KB_BYTES;
}

int kr_of(int64_t K, int form) {
  const int kelem = form != CC_MERGE_TF32X3 ? KB_BYTES / 2 : KB_BYTES / 4;
  return (int)(((2 * K + kelem - 1) / kelem) * kelem);
}

int elem_bytes(int form) { return form == CC_MERGE_TF32X3 ? 4 : 2; }

}  // namespace

uint64_t merge_tc_workspace_bytes(int qa, int qb, int64_t K, int form) {
  if (qa < 7 || qb < 7 || K < 1 || K > (1 << 20)) return 0;
  const uint64_t kr = (uint64_t)kr_of(K, form);
  const uint64_t rows = 2 * ((uint64_t(1) << qb) + 2 * (uint64_t(1) << qa));
  // fp16: the two operand maxima after the operands (1024-aligned)
  const uint64_t scales = form == CC_MERGE_F16X3 ? 1024 + 1024 : 0;
  return rows * kr * elem_bytes(form) + scales + 1024;
}

cc_status launch_merge_tc(const MergeStage& st, int form, void* workspace, uint64_t ws_bytes,
                          void* stream) {
  if (st.Z != 1) return fail(CC_EUNSUPPORTED, "tensor-core merge handles single-batch stages");
  if (st.qa < 7 || st.qb < 7)
    return fail(CC_EUNSUPPORTED, "tensor-core merge needs both factors of >= 128 amplitudes");
  if (st.qa + st.qb > 40) return fail(CC_ERANGE, "merge output too large");
  const uint64_t need = merge_tc_workspace_bytes(st.qa, st.qb, st.K, form);
  if (need == 0) return fail(CC_EUNSUPPORTED, "tensor-core merge shape unsupported");
  if (ws_bytes < need) return fail(CC_EBUFSIZE, "workspace too small for the tensor-core merge");
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fail(CC_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  int* err = device_error_flag();
  if (!err) return fail(CC_ENOMEM, "device error flag allocation failed");

  const int64_t NA = int64_t(1) << st.qa, NB = int64_t(1) << st.qb;
  const int KR = kr_of(st.K, form);
  const int eb = elem_bytes(form);
  unsigned char* ws =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(workspace) + 1023) & ~uintptr_t(1023));
  unsigned char* r_ops = ws;
  unsigned char* c_ops = ws + (size_t)2 * NB * KR * eb;
  cudaStream_t s = (cudaStream_t)stream;

  const int64_t rows = NB + 2 * NA;
  const unsigned blocks = (unsigned)((rows + 7) / 8);
  unsigned int* f16_maxbits = nullptr;
  if (form == CC_MERGE_F16X3) {
    f16_maxbits = reinterpret_cast<unsigned int*>(
        (reinterpret_cast<uintptr_t>(ws) + (uint64_t)2 * rows * KR * eb + 1023) & ~uintptr_t(1023));
    const cudaError_t me = cudaMemsetAsync(f16_maxbits, 0, 2 * sizeof(unsigned int), s);
    if (me != cudaSuccess) return fail(CC_ECUDA, std::string("memset: ") + cudaGetErrorString(me));
    const int64_t longest = st.K << std::max(st.qa, st.qb);
    const dim3 mgrid((unsigned)std::min<int64_t>((longest + 255) / 256, (int64_t)num_sms() * 8), 2);
    operand_absmax_f16<<<mgrid, 256, 0, s>>>((const float2*)st.A, (const float2*)st.B, st.qa,
                                             st.qb, (int)st.K, st.aidx, st.bidx, f16_maxbits);
    // rows: NB of R and 2 NA of Cop, 64 per block (NB, NA >= 2^7)
    const unsigned sblocks = (unsigned)(NB / kSplitRows + 2 * NA / kSplitRows);
    split_operands_f16<<<sblocks, 256, 0, s>>>(
        (const float2*)st.A, (const float2*)st.B, st.qa, st.qb, (int)st.K, KR, st.aidx, st.bidx,
        (__half*)r_ops, (__half*)c_ops, f16_maxbits);
  } else if (form == CC_MERGE_BF16X3)
    split_operands<uint16_t><<<blocks, 256, 0, s>>>(
        (const float2*)st.A, (const float2*)st.B, st.qa, st.qb, (int)st.K, KR, st.aidx, st.bidx,
        (uint16_t*)r_ops, (uint16_t*)c_ops);
  else
    split_operands<uint32_t><<<blocks, 256, 0, s>>>(
        (const float2*)st.A, (const float2*)st.B, st.qa, st.qb, (int)st.K, KR, st.aidx, st.bidx,
        (uint32_t*)r_ops, (uint32_t*)c_ops);

  CUtensorMap map_r, map_c, map_out;
  const CUtensorMapDataType dt = form == CC_MERGE_BF16X3  ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : form == CC_MERGE_F16X3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint32_t box_k = (cuuint32_t)(KB_BYTES / eb);
  const cuuint32_t estr[2] = {1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)KR, (cuuint64_t)(2 * NB)};
    const cuuint64_t strides[1] = {(cuuint64_t)KR * eb};
    const cuuint32_t box[2] = {box_k, (cuuint32_t)BM};
    if (enc(&map_r, dt, 2, r_ops, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CC_ECUDA, "cuTensorMapEncodeTiled (row operand) failed");
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)KR, (cuuint64_t)(4 * NA)};
    const cuuint64_t strides[1] = {(cuuint64_t)KR * eb};
    const cuuint32_t box[2] = {box_k, (cuuint32_t)BN};
    if (enc(&map_c, dt, 2, c_ops, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CC_ECUDA, "cuTensorMapEncodeTiled (column operand) failed");
  }

  // The streaming form reads K blocks of kbb bytes (its own swizzle width).
  // 3xFP16 with eight epilogue warps (two per TMEM lane quarter) streams K
  // in three 64-byte stages to leave room for their staging buffers
  const bool epi8 = form == CC_MERGE_F16X3 && epi8_for(KR * eb);
  const int kbb = epi8 ? 64 : tc_kblock(KR * eb / KB_BYTES);
  CUtensorMap map_r_k, map_c_k;
  {
    const cuuint64_t dims[2] = {(cuuint64_t)KR, (cuuint64_t)(2 * NB)};
    const cuuint64_t strides[1] = {(cuuint64_t)KR * eb};
    const cuuint32_t box[2] = {(cuuint32_t)(kbb / eb), (cuuint32_t)BM};
    if (enc(&map_r_k, dt, 2, r_ops, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle_of(kbb), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CC_ECUDA, "cuTensorMapEncodeTiled (row operand, K blocks) failed");
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)KR, (cuuint64_t)(4 * NA)};
    const cuuint64_t strides[1] = {(cuuint64_t)KR * eb};
    const cuuint32_t box[2] = {(cuuint32_t)(kbb / eb), (cuuint32_t)BN};
    if (enc(&map_c_k, dt, 2, c_ops, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle_of(kbb), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CC_ECUDA, "cuTensorMapEncodeTiled (column operand, K blocks) failed");
  }

  {
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * NA), (cuuint64_t)NB};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * NA) * 4};
    const cuuint32_t box[2] = {32, 32};
    if (enc(&map_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, st.out, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CC_ECUDA, "cuTensorMapEncodeTiled (output) failed");
  }

  static int attr_done[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    cudaFuncSetAttribute(merge_tc_rs_kernel<CC_MERGE_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    cudaFuncSetAttribute(merge_tc_rs_kernel<CC_MERGE_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    for (int b = 32; b <= 128; b *= 2) {
      cudaFuncSetAttribute(tc_kernel_ptr<CC_MERGE_BF16X3>(b), cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
      cudaFuncSetAttribute(tc_kernel_ptr<CC_MERGE_TF32X3>(b), cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
      cudaFuncSetAttribute(tc_kernel_ptr<CC_MERGE_F16X3>(b), cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    }
    cudaFuncSetAttribute(merge_tc_kernel<CC_MERGE_F16X3, 64, 3, 8>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, kEpi8Smem);
    attr_done[dev] = 1;
  }
  const int n_rows = (int)NB, n_cols = (int)(2 * NA);
  const int n_tiles = (n_rows / BM) * (n_cols / BN);
  const int grid = std::min(n_tiles, num_sms());
  const int kblocks = KR * eb / KB_BYTES;
  // 3xTF32: accumulate at most 2 x kTf32GroupTerms real products per pass
  // through TMEM (the K blocks of 2 x 64 TF32 elements).
  const int group_kb = form == CC_MERGE_TF32X3
                           ? std::max(1, (int)(2 * kTf32GroupTerms * eb / KB_BYTES))
                           : kblocks;
  // Row-operand-stationary form when the 128-row R tile (hi and lo, all K
  // blocks) leaves room for at least two 32 KB column stages.
  const int r_bytes = 2 * kblocks * R_TILE;
  const int rs_stages = std::min(RS_MAX_STAGES, (SMEM_LIMIT - 1024 - 256 - STG_TOTAL - r_bytes) / RS_C_STAGE);
  if (rs_stages >= 2 && kblocks <= group_kb && tc_stationary_requested() &&
      form != CC_MERGE_F16X3) {
    const int smem_rs = r_bytes + rs_stages * RS_C_STAGE + STG_TOTAL + 1024 + 256;
    auto kern = form == CC_MERGE_BF16X3 ? merge_tc_rs_kernel<CC_MERGE_BF16X3>
                                        : merge_tc_rs_kernel<CC_MERGE_TF32X3>;
    kern<<<grid, 192, smem_rs, s>>>(map_r, map_c, map_out, n_rows, n_cols, kblocks, rs_stages, err);
  } else {
    const void* kern = epi8 ? reinterpret_cast<const void*>(merge_tc_kernel<CC_MERGE_F16X3, 64, 3, 8>)
                       : form == CC_MERGE_BF16X3 ? tc_kernel_ptr<CC_MERGE_BF16X3>(kbb)
                       : form == CC_MERGE_F16X3  ? tc_kernel_ptr<CC_MERGE_F16X3>(kbb)
                                                 : tc_kernel_ptr<CC_MERGE_TF32X3>(kbb);
    const int kb_n = KR * eb / kbb;
    // 3xTF32 and 3xFP16 (11-bit significands): at most 64 terms per accumulation
    const int64_t gterms = form == CC_MERGE_F16X3 ? f16_group_terms(st.K) : kTf32GroupTerms;
    const int gkb = form != CC_MERGE_BF16X3 ? std::max(1, (int)(2 * gterms * eb / kbb)) : kb_n;
    int a_rows = n_rows, a_cols = n_cols, a_kb = kb_n, a_gkb = std::min(gkb, kb_n);
    const unsigned int* a_mb = f16_maxbits;
    void* args[] = {&map_r_k, &map_c_k, &map_out, &a_rows, &a_cols, &a_kb, &a_gkb, &err, &a_mb};
    const cudaError_t le = cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(epi8 ? 320 : 192), args,
                                            epi8 ? kEpi8Smem : SMEM_BYTES, s);
    if (le != cudaSuccess)
      return fail(CC_ECUDA, std::string("tensor-core merge launch: ") + cudaGetErrorString(le));
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("tensor-core merge launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

}  // namespace cc
