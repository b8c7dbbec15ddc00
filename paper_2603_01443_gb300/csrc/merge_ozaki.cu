// Complex128 merging (Algorithm 3) on tcgen05 tensor cores: FP64 results
// from bf16 products by the Ozaki scheme (Ozaki, Ogita, Oishi, Rump, "Error-
// free transformations of matrix multiplication by using fast routines of
// matrix multiplication and its applications", Numer. Algorithms 59, 2012).
//
// The two-factor merge is the real GEMM of merge_tc.cu,
//   C[y][n] = sum_kk R[y][kk] * Cop[n][kk],   n = 2x + (0: real, 1: imaginary),
// here with FP64 operands and an FP64 (interleaved complex128) result.
//
// Splitting.  Every operand row is scaled by a power of two 2^e (the row of
// R) or 2^f (the row of Cop) so that its largest entry is below 1 in
// magnitude, and each scaled entry, rounded to 53 fractional bits
// (X = round(v 2^(53 - e))), is written as S = 6 balanced base-2^9 digits,
//   X = sum_i d_i 2^(9 (5 - i)),   |d_i| <= 256,
// so v 2^-e = 2^-8 sum_i d_i 2^(-9 i).  Slice i stores d_i 2^(-9 i) in bf16,
// which holds it exactly (at most 8 significant bits).
//
// Products.  The tensor cores form the slice products (i, j) with
// i + j <= 5 (21 products; the dropped ones are below 2^-50 of the row
// scales' product) and accumulate them in FP32 in four TMEM accumulators:
// level 0 (i + j = 0), level 1, level 2, and levels 3-5 together.  A level-L
// product is an integer times 2^(-9 L), at most 2^16 in magnitude, so over an
// accumulation group of at most 128 real K elements level 0 sums integers
// below 2^23 and level 1 multiples of 2^-9 below 2^15: FP32 holds every
// partial sum exactly.  Level 2 is exact while its partial sums stay below
// 2^24 units (3 x 128 products of at most 2^16; balanced digits make that
// sure in practice); the merged levels 3-5 carry an FP32 rounding error
// below 2^-40 of the scales' product.
//
// Epilogue.  Per output element the four accumulators become one exact
// 64-bit fixed-point integer with 30 fractional bits,
//   I = a0 2^30 + a1 2^30 + a2 2^30 + round(a3 2^30),
// longer K adds the integers of its 128-element groups exactly (the partial
// sum round-trips through the output buffer as int64), and the last group
// converts I 2^(e_y + f_n - 46) to FP64 with one rounding, built from the
// integer bits (no FP64 arithmetic anywhere in the kernel).
//
// Kernel structure (one CTA per SM, persistent over 128 x 128 output tiles,
// bands of 16 row tiles):
//   warp 0      TMA producer: per K block one 3-D load of the 6 row-operand
//               slices (128 rows) and one of the 6 column-operand slices
//               (128 rows) into one of NST shared-memory stages;
//   warp 1      allocates the 512 TMEM columns (4 accumulators of 128) and one
//               lane issues the 21 x (K block / 16) tcgen05.mma of a stage;
//   warps 2..5  epilogue: tcgen05.ld of the four accumulators in 16-column
//               chunks, fixed-point sum, FP64 assembly, 128-byte-swizzled
//               staging and bulk tensor stores.
// Every mbarrier wait is bounded as in merge_tc.cu: on expiry the kernel
// raises the device error flag, drains its own copies and MMAs and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>

#include "internal.h"
#include "tcgen05_util.cuh"

namespace cc {

namespace {

using namespace tcg;

constexpr int OZ_S = 6;           // slices per operand
constexpr int OZ_BETA = 9;        // bits per slice
constexpr int OZ_LEVELS = 6;      // products (i, j) with i + j < OZ_LEVELS
constexpr int OZ_NACC = 4;        // TMEM accumulators: levels 0, 1, 2, 3..5
constexpr int OZ_BM = 128;        // output rows per tile
constexpr int OZ_BN = 128;        // output real columns per tile
constexpr int OZ_GROUP_K = 128;   // real K elements per accumulation group
constexpr int OZ_FIX = 30;        // fraction bits of the epilogue's fixed point
constexpr int OZ_STG_BYTES = 32 * 128;              // one store box: 32 rows x 16 FP64
constexpr int OZ_STG_TOTAL = 4 * 2 * OZ_STG_BYTES;  // 4 epilogue warps x 2 buffers
constexpr int OZ_OPERANDS = 2 * 96 * 1024;          // operand stages: 192 KB
constexpr int OZ_SMEM = OZ_OPERANDS + OZ_STG_TOTAL + 1024 /*align*/ + 256 /*barriers*/;
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_BAND = 16;
static_assert(OZ_NACC * OZ_BN <= OZ_TMEM_COLS, "accumulators fit in TMEM");

// Row exponent of a zero row: every digit is 0 and so is every product.
constexpr int32_t OZ_ZERO_EXP = -4000;

// ---------------------------------------------------------------- splitting
__device__ __forceinline__ double ozaki_operand(const double2* __restrict__ A,
                                                const double2* __restrict__ B, int64_t NA,
                                                int64_t NB, int K, const int32_t* __restrict__ aidx,
                                                const int32_t* __restrict__ bidx, int64_t row,
                                                int kk) {
  if (kk >= 2 * K) return 0.0;
  if (row < NB) {
    const double2 b = B[(int64_t)bidx[kk % K] * NB + row];
    return kk < K ? b.x : b.y;
  }
  const int64_t n = row - NB;
  const double2 a = A[(int64_t)aidx[kk % K] * NA + (n >> 1)];
  if ((n & 1) == 0) return kk < K ? a.x : -a.y;
  return kk < K ? a.y : a.x;
}

// One warp per operand row: rows [0, NB) are R (from the upper factor B),
// rows [NB, NB + 2 NA) are Cop (from the lower factor A).  Writes the row's
// exponent and its 6 slices (slice i of row r at sl[(i * rows_of_operand + r) * KR]).
__global__ void __launch_bounds__(256)
    ozaki_split(const double2* __restrict__ A, const double2* __restrict__ B, int qa, int qb,
                int K, int KR, const int32_t* __restrict__ aidx, const int32_t* __restrict__ bidx,
                __nv_bfloat16* __restrict__ r_sl, __nv_bfloat16* __restrict__ c_sl,
                int32_t* __restrict__ e_row, int32_t* __restrict__ f_col) {
  const int64_t NA = int64_t(1) << qa, NB = int64_t(1) << qb;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= NB + 2 * NA) return;
  // largest magnitude of the row: |v| orders like its bits with the sign cleared
  unsigned long long mx = 0;
  for (int kk = lane; kk < KR; kk += 32) {
    const double v = ozaki_operand(A, B, NA, NB, K, aidx, bidx, row, kk);
    mx = max(mx, (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  // 2^e > max |v|: a normal max = 1.m 2^(E - 1023) < 2^(E - 1022)
  const int32_t e = mx == 0 ? OZ_ZERO_EXP : (int32_t)((mx >> 52) & 0x7FF) - 1022;
  const bool is_r = row < NB;
  const int64_t r = is_r ? row : row - NB;
  const int64_t plane = is_r ? NB : 2 * NA;
  __nv_bfloat16* sl = is_r ? r_sl : c_sl;
  if (lane == 0) {
    if (is_r) e_row[r] = e;
    else f_col[r] = e;
  }
  const float scale[OZ_S] = {1.0f, 0x1p-9f, 0x1p-18f, 0x1p-27f, 0x1p-36f, 0x1p-45f};
  for (int kk = lane; kk < KR; kk += 32) {
    const double v = ozaki_operand(A, B, NA, NB, K, aidx, bidx, row, kk);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ev = (int)((bits >> 52) & 0x7FF);
    long long X = 0;
    if (e != OZ_ZERO_EXP && (bits & 0x7FFFFFFFFFFFFFFFull) != 0) {
      // v = mant 2^(ev - 1075), X = round(v 2^(53 - e)) = round(mant 2^(ev - 1022 - e))
      const unsigned long long mant =
          ev == 0 ? (bits & 0xFFFFFFFFFFFFFull) << 1 : (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const int sh = e + 1022 - ev;  // >= 0 since |v| < 2^e: a right shift
      unsigned long long m = 0;
      if (sh == 0) m = mant;
      else if (sh < 64) m = (mant + (1ull << (sh - 1))) >> sh;
      X = (bits >> 63) ? -(long long)m : (long long)m;
    }
    // balanced base-2^9 digits, most significant first; |d_i| <= 256
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      const int sh = OZ_BETA * (OZ_S - 1 - i);
      long long d = X;
      if (sh > 0) d = (X + (1ll << (sh - 1))) >> sh;
      X -= d << sh;
      sl[((int64_t)i * plane + r) * KR + kk] = __float2bfloat16_rn((float)d * scale[i]);
    }
  }
}

// ------------------------------------------------------------ main kernel
__device__ __forceinline__ void oz_tile_coords(int t, int tiles_m, int tiles_n, int& m0, int& n0) {
  const int band = t / (OZ_BAND * tiles_n), r = t - band * OZ_BAND * tiles_n;
  const int rows = min(OZ_BAND, tiles_m - band * OZ_BAND);
  m0 = (band * OZ_BAND + r % rows) * OZ_BM;
  n0 = (r / rows) * OZ_BN;
}

// Instruction descriptor: FP32 accumulator, bf16 A and B (K-major), M = 128, N = 128.
constexpr uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
         ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// The exact fixed-point value of one output element, in units of 2^-OZ_FIX of
// the level-0 unit: a0, a1, a2 are exact multiples of 1, 2^-9, 2^-18.
__device__ __forceinline__ long long oz_fixed(float a0, float a1, float a2, float a3) {
  const long long i0 = __float2ll_rn(a0);
  const long long i1 = __float2ll_rn(a1 * 0x1p9f);
  const long long i2 = __float2ll_rn(a2 * 0x1p18f);
  const long long i3 = __float2ll_rn(a3 * 0x1p30f);
  return (i0 << OZ_FIX) + (i1 << (OZ_FIX - OZ_BETA)) + (i2 << (OZ_FIX - 2 * OZ_BETA)) + i3;
}

// FP64 bits of I 2^sc, rounded to nearest even, from the integer alone.
__device__ __forceinline__ unsigned long long oz_to_f64(long long I, int sc) {
  if (I == 0) return 0ull;
  const unsigned long long sign = I < 0 ? (1ull << 63) : 0ull;
  const unsigned long long m = I < 0 ? (unsigned long long)(-I) : (unsigned long long)I;
  const int lz = __clzll((long long)m);
  const unsigned long long mn = m << lz;  // leading one at bit 63
  unsigned long long mant = mn >> 11;     // 53 bits, implicit one at bit 52
  const unsigned long long rest = mn & 0x7FFull;
  mant += (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
  const int E = 1023 + (63 - lz) + sc;  // biased exponent of the leading one
  if (E <= 0) return sign;              // below the normal range (never for state vectors)
  if (E >= 2047) return sign | 0x7FF0000000000000ull;
  // the implicit one of mant adds 1 to E - 1; a rounding carry to 2^53 adds one more
  return sign | ((((unsigned long long)(E - 1)) << 52) + mant);
}

template <int KBB, int NST>
__global__ void __launch_bounds__(192, 1)
    merge_ozaki_kernel(const __grid_constant__ CUtensorMap map_r,
                       const __grid_constant__ CUtensorMap map_c,
                       const __grid_constant__ CUtensorMap map_out,
                       const int32_t* __restrict__ e_row, const int32_t* __restrict__ f_col,
                       const double* out, int n_rows, int n_cols, int kblocks, int group_kb,
                       int* err) {
  constexpr int KEL = KBB / 2;                  // bf16 elements of K per stage
  constexpr int AS = OZ_BM * KBB, BS = OZ_BN * KBB;  // one slice of each operand
  constexpr int STB = OZ_S * (AS + BS);
  static_assert(NST * STB == OZ_OPERANDS, "operand stages of 192 KB");
  static_assert((2 * NST + 6) * 8 <= 256, "barrier area");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* stg_base = smem + NST * STB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg_base + OZ_STG_TOTAL);
  uint64_t* full = bars;                // [NST]
  uint64_t* empty = bars + NST;         // [NST]
  uint64_t* tfull = bars + 2 * NST;     // the accumulators hold a finished group
  uint64_t* tempty = bars + 2 * NST + 1;  // the epilogue has read them
  uint64_t* drain = bars + 2 * NST + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * NST + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = n_rows / OZ_BM, tiles_n = n_cols / OZ_BN;
  const int n_tiles = tiles_m * tiles_n;
  const int n_groups = (kblocks + group_kb - 1) / group_kb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 4);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
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
      uint32_t use = 0;
      bool issued[NST];
      uint32_t issued_parity[NST];
      for (int i = 0; i < NST; ++i) {
        issued[i] = false;
        issued_parity[i] = 0;
      }
      bool ok = true;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        int m0, n0;
        oz_tile_coords(t, tiles_m, tiles_n, m0, n0);
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&empty[s], (use & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          unsigned char* st = smem + s * STB;
          const uint32_t fb = smem_u32(&full[s]);
          mbar_expect_tx(&full[s], STB);
          tma_load_3d(smem_u32(st), &map_r, fb, kb * KEL, m0, 0);
          tma_load_3d(smem_u32(st + OZ_S * AS), &map_c, fb, kb * KEL, n0, 0);
          issued[s] = true;
          issued_parity[s] = use & 1;
          if (++s == NST) {
            s = 0;
            ++use;
          }
        }
      }
      if (!ok) {
        for (int i = 0; i < NST; ++i)
          if (issued[i]) mbar_drain(&full[i], issued_parity[i]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = oz_idesc();
      int s = 0;
      uint32_t use = 0;
      int iter = 0;
      bool ok = true;
      bool any_mma = false;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int kb0 = 0; kb0 < kblocks && ok; kb0 += group_kb, ++iter) {
          if (!mbar_wait(tempty, (iter & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          uint32_t fresh = (1u << OZ_NACC) - 1;  // accumulators not yet written in this group
          const int kb1 = min(kblocks, kb0 + group_kb);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&full[s], use & 1, abort_flag, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = smem_u32(smem + s * STB);
#pragma unroll
            for (int k = 0; k < KBB / 32; ++k) {
              const uint64_t adv = (uint64_t)((k * 32) >> 4);
#pragma unroll
              for (int i = 0; i < OZ_S; ++i) {
                const uint64_t a = sdesc_sw<KBB>(st + i * AS) + adv;
#pragma unroll
                for (int j = 0; j < OZ_LEVELS - i; ++j) {
                  const int acc = min(i + j, OZ_NACC - 1);
                  const uint64_t b = sdesc_sw<KBB>(st + OZ_S * AS + j * BS) + adv;
                  const uint32_t accumulate = (fresh >> acc) & 1u ? 0u : 1u;
                  fresh &= ~(1u << acc);
                  umma<CC_MERGE_BF16X3>(tmem_base + (uint32_t)(acc * OZ_BN), a, b, idesc,
                                        accumulate);
                }
              }
            }
            any_mma = true;
            umma_commit(&empty[s]);
            if (++s == NST) {
              s = 0;
              ++use;
            }
          }
          if (!ok) break;
          umma_commit(tfull);
        }
      }
      if (!ok && any_mma) {
        umma_commit(drain);
        mbar_drain(drain, 0);
      }
    }
  } else {
    // epilogue warps 2..5: TMEM lane quarter = warp % 4, one output row per lane
    const int quarter = warp & 3;
    unsigned char* stg = stg_base + quarter * 2 * OZ_STG_BYTES;
    int buf = 0;
    int iter = 0;
    bool ok_all = true;
    for (int t = blockIdx.x; t < n_tiles && ok_all; t += gridDim.x) {
      int m0, n0;
      oz_tile_coords(t, tiles_m, tiles_n, m0, n0);
      const int y = m0 + quarter * 32 + lane;
      const int ey = e_row[y] - 2 * (OZ_BETA - 1) - OZ_FIX;  // exponent of one fixed-point unit
      const long long* orow = reinterpret_cast<const long long*>(out) + (int64_t)y * n_cols + n0;
      for (int g = 0; g < n_groups; ++g, ++iter) {
        int ok = 1;
        if (lane == 0) ok = mbar_wait(tfull, iter & 1, abort_flag, err) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          ok_all = false;
          break;
        }
        tc_fence_after();
        if (g > 0) {  // the earlier groups' partial sums of this tile must have landed
          if (lane == 0) {
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
            asm volatile("fence.proxy.async.global;" ::: "memory");
          }
          __syncwarp();
        }
        const bool last = g == n_groups - 1;
        const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < OZ_BN / 16; ++c) {
          uint32_t r0[16], r1[16], r2[16], r3[16];
          tmem_ld16(tbase + 0 * OZ_BN + c * 16, r0);
          tmem_ld16(tbase + 1 * OZ_BN + c * 16, r1);
          tmem_ld16(tbase + 2 * OZ_BN + c * 16, r2);
          tmem_ld16(tbase + 3 * OZ_BN + c * 16, r3);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          long long v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            v[j] = oz_fixed(__uint_as_float(r0[j]), __uint_as_float(r1[j]),
                            __uint_as_float(r2[j]), __uint_as_float(r3[j]));
          if (g > 0) {  // add the earlier groups' exact sums, read through L2
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
              long long p0, p1;
              asm volatile("ld.global.cg.v2.s64 {%0, %1}, [%2];"
                           : "=l"(p0), "=l"(p1)
                           : "l"(orow + c * 16 + j));
              v[j] += p0;
              v[j + 1] += p1;
            }
          }
          unsigned long long w[16];
          if (last) {
            const int4* fp = reinterpret_cast<const int4*>(f_col + n0 + c * 16);
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
              const int4 f = __ldg(fp + q4);
              w[4 * q4 + 0] = oz_to_f64(v[4 * q4 + 0], ey + f.x);
              w[4 * q4 + 1] = oz_to_f64(v[4 * q4 + 1], ey + f.y);
              w[4 * q4 + 2] = oz_to_f64(v[4 * q4 + 2], ey + f.z);
              w[4 * q4 + 3] = oz_to_f64(v[4 * q4 + 3], ey + f.w);
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = (unsigned long long)v[j];
          }
          unsigned char* sb = stg + buf * OZ_STG_BYTES;
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          __syncwarp();
          // 128-byte swizzle: the 16-byte chunk h of row `lane` sits at h ^ (lane & 7)
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            ulonglong2* dst = reinterpret_cast<ulonglong2*>(sb + lane * 128 + ((h ^ (lane & 7)) << 4));
            *dst = make_ulonglong2(w[2 * h], w[2 * h + 1]);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            asm volatile(
                "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                    reinterpret_cast<uint64_t>(&map_out)),
                "r"(smem_u32(sb)), "r"(n0 + c * 16), "r"(m0 + quarter * 32)
                : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
          buf ^= 1;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty);
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
                 "r"(OZ_TMEM_COLS)
                 : "memory");
  }
}

typedef CUresult (*OzEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                               const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                               const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

OzEncodeFn oz_encode_fn() {
  static OzEncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<OzEncodeFn>(p);
    cudaGetLastError();
  }
  return fn;
}

// Bytes of K per stage: 64 (two 96 KB stages, the default) or 32 (four 48 KB
// stages); CUTSIM_OZ_KBLOCK overrides.
int oz_kblock() {
  const char* e = std::getenv("CUTSIM_OZ_KBLOCK");
  return e && std::atoi(e) == 32 ? 32 : 64;
}

int oz_kr(int64_t K) { return (int)(((2 * K + 31) / 32) * 32); }

uint64_t align1k(uint64_t x) { return (x + 1023) & ~uint64_t(1023); }

struct OzLayout {
  uint64_t r_sl, c_sl, e_row, f_col, end;
};

OzLayout oz_layout(int qa, int qb, int64_t K) {
  const uint64_t NA = uint64_t(1) << qa, NB = uint64_t(1) << qb, KR = (uint64_t)oz_kr(K);
  OzLayout L;
  L.r_sl = 0;
  L.c_sl = align1k(L.r_sl + OZ_S * NB * KR * 2);
  L.e_row = align1k(L.c_sl + OZ_S * 2 * NA * KR * 2);
  L.f_col = align1k(L.e_row + NB * 4);
  L.end = align1k(L.f_col + 2 * NA * 4);
  return L;
}

}  // namespace

uint64_t merge_ozaki_workspace_bytes(int qa, int qb, int64_t K) {
  if (qa < 7 || qb < 7 || K < 1 || K > (1 << 20)) return 0;
  return oz_layout(qa, qb, K).end + 1024;
}

cc_status launch_merge_ozaki(const MergeStage& st, void* workspace, uint64_t ws_bytes,
                             void* stream) {
  if (st.Z != 1) return fail(CC_EUNSUPPORTED, "Ozaki merge handles single-batch stages");
  if (st.qa < 7 || st.qb < 7)
    return fail(CC_EUNSUPPORTED, "Ozaki merge needs both factors of >= 128 amplitudes");
  if (st.qa + st.qb > 40) return fail(CC_ERANGE, "merge output too large");
  const uint64_t need = merge_ozaki_workspace_bytes(st.qa, st.qb, st.K);
  if (need == 0) return fail(CC_EUNSUPPORTED, "Ozaki merge shape unsupported");
  if (ws_bytes < need) return fail(CC_EBUFSIZE, "workspace too small for the Ozaki merge");
  if ((reinterpret_cast<uintptr_t>(st.out) & 15u) != 0)
    return fail(CC_EINVAL, "Ozaki merge output must be 16-byte aligned");
  OzEncodeFn enc = oz_encode_fn();
  if (!enc) return fail(CC_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  int* err = device_error_flag();
  if (!err) return fail(CC_ENOMEM, "device error flag allocation failed");

  const int64_t NA = int64_t(1) << st.qa, NB = int64_t(1) << st.qb;
  const int KR = oz_kr(st.K);
  const OzLayout L = oz_layout(st.qa, st.qb, st.K);
  unsigned char* ws = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(workspace) + 1023) & ~uintptr_t(1023));
  __nv_bfloat16* r_sl = reinterpret_cast<__nv_bfloat16*>(ws + L.r_sl);
  __nv_bfloat16* c_sl = reinterpret_cast<__nv_bfloat16*>(ws + L.c_sl);
  int32_t* e_row = reinterpret_cast<int32_t*>(ws + L.e_row);
  int32_t* f_col = reinterpret_cast<int32_t*>(ws + L.f_col);
  cudaStream_t s = (cudaStream_t)stream;

  const int64_t rows = NB + 2 * NA;
  ozaki_split<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(
      (const double2*)st.A, (const double2*)st.B, st.qa, st.qb, (int)st.K, KR, st.aidx, st.bidx,
      r_sl, c_sl, e_row, f_col);

  const int kbb = oz_kblock();
  const int kel = kbb / 2;
  const CUtensorMapSwizzle sw = kbb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
  CUtensorMap map_r, map_c, map_out;
  const cuuint32_t estr3[3] = {1, 1, 1};
  {
    const cuuint64_t dims[3] = {(cuuint64_t)KR, (cuuint64_t)NB, (cuuint64_t)OZ_S};
    const cuuint64_t strides[2] = {(cuuint64_t)KR * 2, (cuuint64_t)NB * KR * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kel, (cuuint32_t)OZ_BM, (cuuint32_t)OZ_S};
    if (enc(&map_r, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, r_sl, dims, strides, box, estr3,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CC_ECUDA, "cuTensorMapEncodeTiled (Ozaki row slices) failed");
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)KR, (cuuint64_t)(2 * NA), (cuuint64_t)OZ_S};
    const cuuint64_t strides[2] = {(cuuint64_t)KR * 2, (cuuint64_t)(2 * NA) * KR * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kel, (cuuint32_t)OZ_BN, (cuuint32_t)OZ_S};
    if (enc(&map_c, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, c_sl, dims, strides, box, estr3,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CC_ECUDA, "cuTensorMapEncodeTiled (Ozaki column slices) failed");
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * NA), (cuuint64_t)NB};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * NA) * 8};
    const cuuint32_t box[2] = {16, 32};
    const cuuint32_t estr2[2] = {1, 1};
    if (enc(&map_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, st.out, dims, strides, box, estr2,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CC_ECUDA, "cuTensorMapEncodeTiled (Ozaki output) failed");
  }

  static int attr_done[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    cudaFuncSetAttribute(merge_ozaki_kernel<64, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    cudaFuncSetAttribute(merge_ozaki_kernel<32, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    attr_done[dev] = 1;
  }
  const int n_rows = (int)NB, n_cols = (int)(2 * NA);
  const int n_tiles = (n_rows / OZ_BM) * (n_cols / OZ_BN);
  const int grid = std::min(n_tiles, num_sms());
  const int kblocks = KR / kel;
  const int group_kb = OZ_GROUP_K / kel;
  const double* outp = static_cast<const double*>(st.out);
  if (kbb == 64)
    merge_ozaki_kernel<64, 2><<<grid, 192, OZ_SMEM, s>>>(map_r, map_c, map_out, e_row, f_col, outp,
                                                         n_rows, n_cols, kblocks, group_kb, err);
  else
    merge_ozaki_kernel<32, 4><<<grid, 192, OZ_SMEM, s>>>(map_r, map_c, map_out, e_row, f_col, outp,
                                                         n_rows, n_cols, kblocks, group_kb, err);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("Ozaki merge launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

}  // namespace cc
