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
// scales' product) and accumulate them in FP32 in TMEM, one accumulator per
// level L = i + j for the leading levels and one for the remaining levels
// together.  A level-L product is an integer times 2^(-9 L), at most 2^16 in
// magnitude, so over an accumulation group of at most 128 real K elements
// level 0 sums integers below 2^23 and level 1 multiples of 2^-9 below 2^15:
// FP32 holds every partial sum exactly.  Levels 2 and 3 are exact while their
// partial sums stay below 2^24 units ((L + 1) x 128 products of at most 2^16;
// balanced digits keep them near 2^20 in practice).  Only the merged
// accumulator rounds: with four accumulators (levels 0, 1, 2, then 3-5) its
// rounding reaches a few 1e-13 of max |psi| by 256 terms; with five (levels
// 0-3, then 4-5) it stays near 2e-14 at any K.
//
// Epilogue.  Per output element the accumulators become one exact 64-bit
// fixed-point integer (30 or 33 fraction bits below the level-0 unit),
// longer K adds the integers of its 128-element groups exactly (the partial
// sum round-trips through the output buffer as int64), and the last group
// rounds I 2^(e_y + f_n - 16 - fraction bits) to FP64 once.
//
// Kernel structure (one CTA per SM, persistent over 128 x BN output tiles,
// bands of 16 row tiles):
//   warp 0      TMA producer: per K block one 3-D load of the 6 row-operand
//               slices (128 rows) and one of the 6 column-operand slices
//               (BN rows) into one of NST shared-memory stages;
//   warp 1      allocates TMEM (NACC accumulators of BN columns, one or two
//               sets) and one lane issues the 21 x (K block / 16) tcgen05.mma
//               of a stage;
//   warps 2..   epilogue (4 or 8 warps): tcgen05.ld of the accumulators in
//               16-column chunks, fixed-point sum, FP64 conversion,
//               128-byte-swizzled staging and bulk tensor stores; with two
//               accumulator sets the epilogue of one tile overlaps the MMAs
//               of the next.
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
constexpr int OZ_BM = 128;        // output rows per tile
constexpr int OZ_GROUP_K = 128;   // real K elements per accumulation group
constexpr int OZ_STG_BYTES = 32 * 128;              // one store box: 32 rows x 16 FP64
constexpr int OZ_BAND = 16;

// Row exponent of a zero row: every digit is 0 and so is every product.
constexpr int32_t OZ_ZERO_EXP = -4000;

// ---------------------------------------------------------------- splitting
// v = X 2^(e - 53) with X rounded to an integer (|v| < 2^e), cut into OZ_S
// balanced base-2^9 digits, most significant first (|d_i| <= 256); out[i] is
// d_i 2^(-9 i), exact in bf16.
__device__ __forceinline__ void ozaki_digits(double v, int32_t e, float (&out)[OZ_S]) {
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
  const float scale[OZ_S] = {1.0f, 0x1p-9f, 0x1p-18f, 0x1p-27f, 0x1p-36f, 0x1p-45f};
#pragma unroll
  for (int i = 0; i < OZ_S; ++i) {
    const int sh = OZ_BETA * (OZ_S - 1 - i);
    long long d = X;
    if (sh > 0) d = (X + (1ll << (sh - 1))) >> sh;
    X -= d << sh;
    out[i] = (float)d * scale[i];
  }
}

// The split through a shared-memory transpose.  A block takes 64 operand
// rows: 64 rows y of R (from the upper factor B), or 32 amplitudes x of A,
// giving rows 2x and 2x+1 of Cop.  First each row's exponent, from the
// largest |re| and |im| of its amplitude over the K slices (2^e > that
// maximum); then the padded K range in chunks of 32, each warp loading
// contiguous 32-amplitude runs of one slice, and the rows' digits written as
// contiguous runs of each slice (slice i of row r at
// sl[(i * rows_of_operand + r) * KR]).
constexpr int kOzRows = 64, kOzChunk = 32;
__global__ void __launch_bounds__(256)
    ozaki_split(const double2* __restrict__ A, const double2* __restrict__ B, int qa, int qb,
                int K, int KR, const int32_t* __restrict__ aidx, const int32_t* __restrict__ bidx,
                __nv_bfloat16* __restrict__ r_sl, __nv_bfloat16* __restrict__ c_sl,
                int32_t* __restrict__ e_row, int32_t* __restrict__ f_col) {
  __shared__ double T[kOzRows][kOzChunk + 1];
  __shared__ unsigned long long s_mx[8][kOzRows];
  __shared__ int32_t s_e[kOzRows];
  const int64_t NA = int64_t(1) << qa, NB = int64_t(1) << qb;
  const int64_t r_blocks = NB / kOzRows;
  const bool is_r = (int64_t)blockIdx.x < r_blocks;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = is_r ? (int64_t)blockIdx.x * kOzRows
                            : ((int64_t)blockIdx.x - r_blocks) * kOzRows;
  const int64_t amp0 = is_r ? row0 : row0 / 2;
  const int qn = is_r ? qb : qa;
  const double2* __restrict__ X = is_r ? B : A;
  const int32_t* __restrict__ idx = is_r ? bidx : aidx;
  const int64_t plane = is_r ? NB : 2 * NA;
  __nv_bfloat16* const sl = is_r ? r_sl : c_sl;
  // |v| orders like its bits with the sign cleared
  const unsigned long long abs_mask = 0x7FFFFFFFFFFFFFFFull;
  unsigned long long m0 = 0, m1 = 0;
  for (int k = warp; k < K; k += 8) {
    const int64_t base = ((int64_t)idx[k] << qn) + amp0;
    const double2 v0 = X[base + lane];
    m0 = max(m0, max((unsigned long long)__double_as_longlong(v0.x) & abs_mask,
                     (unsigned long long)__double_as_longlong(v0.y) & abs_mask));
    if (is_r) {
      const double2 v1 = X[base + 32 + lane];
      m1 = max(m1, max((unsigned long long)__double_as_longlong(v1.x) & abs_mask,
                       (unsigned long long)__double_as_longlong(v1.y) & abs_mask));
    }
  }
  s_mx[warp][lane] = m0;
  s_mx[warp][32 + lane] = m1;
  __syncthreads();
  const int n_amp = is_r ? 64 : 32;
  if ((int)threadIdx.x < n_amp) {
    unsigned long long mx = 0;
    for (int w = 0; w < 8; ++w) mx = max(mx, s_mx[w][threadIdx.x]);
    // 2^e > max |v|: a normal max = 1.m 2^(E - 1023) < 2^(E - 1022)
    const int32_t e = mx == 0 ? OZ_ZERO_EXP : (int32_t)((mx >> 52) & 0x7FF) - 1022;
    if (is_r) {
      s_e[threadIdx.x] = e;
      e_row[row0 + threadIdx.x] = e;
    } else {
      s_e[2 * threadIdx.x] = s_e[2 * threadIdx.x + 1] = e;
      f_col[row0 + 2 * threadIdx.x] = e;
      f_col[row0 + 2 * threadIdx.x + 1] = e;
    }
  }
  __syncthreads();
  for (int c0 = 0; c0 < KR; c0 += kOzChunk) {
    for (int kl = warp; kl < kOzChunk; kl += 8) {
      const int kk = c0 + kl;
      const bool used = kk < 2 * K, re = kk < K;
      const int k = re ? kk : kk - K;
      if (is_r) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          double v = 0.0;
          if (used) {
            const double2 b = B[((int64_t)bidx[k] << qb) + amp0 + h * 32 + lane];
            v = re ? b.x : b.y;
          }
          T[h * 32 + lane][kl] = v;
        }
      } else {
        double v0 = 0.0, v1 = 0.0;
        if (used) {
          const double2 a = A[((int64_t)aidx[k] << qa) + amp0 + lane];
          v0 = re ? a.x : -a.y;  // row 2x
          v1 = re ? a.y : a.x;   // row 2x + 1
        }
        T[2 * lane][kl] = v0;
        T[2 * lane + 1][kl] = v1;
      }
    }
    __syncthreads();
    for (int r = warp; r < kOzRows; r += 8) {
      float d[OZ_S];
      ozaki_digits(T[r][lane], s_e[r], d);
#pragma unroll
      for (int i = 0; i < OZ_S; ++i)
        sl[((int64_t)i * plane + row0 + r) * KR + c0 + lane] = __float2bfloat16_rn(d[i]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ main kernel
// A kernel configuration: K bytes per stage KBB, NST stages, BN output
// columns per tile, NACC TMEM accumulators (levels 0 .. NACC - 2 each in
// its own, exact; the remaining levels merged in the last), NBUF sets of
// them (2: the epilogue of one tile overlaps the MMAs of the next).
template <int KBB, int NST, int BN, int NACC, int NBUF, int EW>
struct OzCfg {
  static constexpr int KEL = KBB / 2;                  // bf16 elements of K per stage
  static constexpr int AS = OZ_BM * KBB;               // one row-operand slice per stage
  static constexpr int BS = BN * KBB;                  // one column-operand slice per stage
  static constexpr int STB = OZ_S * (AS + BS);         // one stage
  static constexpr int STG = EW * 2 * OZ_STG_BYTES;     // epilogue staging: 2 boxes per warp
  static constexpr int SMEM = NST * STB + STG + 1024 + 256;
  static constexpr int THREADS = 64 + 32 * EW;
  static constexpr int COLS_PER_WARP = BN / (EW / 4);  // each TMEM lane quarter split EW / 4 ways
  static constexpr int COLS = NACC * BN * NBUF;
  static constexpr int TMEM = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128
                            : COLS <= 256 ? 256 : 512;
  // fixed-point fraction bits: the exact levels' units down to 2^-(9 (NACC - 2)),
  // plus a margin for the merged level's rounding
  static constexpr int FIX = NACC == 4 ? 30 : 33;
  static_assert(COLS <= 512, "accumulators fit in TMEM");
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static_assert(NACC == 4 || NACC == 5, "4 or 5 accumulators");
  static_assert((EW == 4 || EW == 8) && COLS_PER_WARP % 16 == 0, "epilogue warps");
};

__device__ __forceinline__ void oz_tile_coords(int t, int tiles_m, int tiles_n, int bn, int& m0,
                                               int& n0) {
  const int band = t / (OZ_BAND * tiles_n), r = t - band * OZ_BAND * tiles_n;
  const int rows = min(OZ_BAND, tiles_m - band * OZ_BAND);
  m0 = (band * OZ_BAND + r % rows) * OZ_BM;
  n0 = (r / rows) * bn;
}

// Instruction descriptor: FP32 accumulator, bf16 A and B (K-major), M = 128, N = BN.
template <int BN>
constexpr uint32_t oz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
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

__device__ __forceinline__ long long mad_wide(int a, int b, long long c) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

// The fixed-point value of one output element in units of 2^-FIX of the
// level-0 unit.  Level L < NACC - 1 holds an integer times 2^(-9 L) below
// 2^25 units; each converts to int32 exactly, the merged last level rounds.
// The sum is formed with 32 x 32 -> 64-bit multiply-adds by powers of two.
template <int NACC, int FIX>
__device__ __forceinline__ long long oz_fixed(const float (&a)[NACC]) {
  long long I = (long long)__float2int_rn(a[NACC - 1] * __int_as_float((127 + FIX) << 23));
#pragma unroll
  for (int L = NACC - 2; L >= 1; --L)
    I = mad_wide(__float2int_rn(a[L] * __int_as_float((127 + OZ_BETA * L) << 23)),
                 1 << (FIX - OZ_BETA * L), I);
  // level 0: i0 2^FIX, FIX >= 30
  const int i0 = __float2int_rn(a[0]);
  return mad_wide(i0 << (FIX - 30), 1 << 30, I);
}

// FP64 bits of I 2^sc, rounded to nearest even, from the integer alone.
__device__ __forceinline__ unsigned long long oz_to_f64(long long I, int sc) {
  if (I == 0) return 0ull;
  const unsigned long long sign = (unsigned long long)I & (1ull << 63);
  const unsigned long long m = I < 0 ? 0ull - (unsigned long long)I : (unsigned long long)I;
  const int lz = __clzll((long long)m);
  const unsigned long long mn = m << lz;  // leading one at bit 63
  unsigned long long mant = mn >> 11;     // 53 bits, implicit one at bit 52
  const unsigned int rest = (unsigned int)mn & 0x7FFu;
  mant += (rest > 0x400u || (rest == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  const int E = 1023 + (63 - lz) + sc;  // biased exponent of the leading one
  if (E <= 0) return sign;              // below the normal range (never for state vectors)
  if (E >= 2047) return sign | 0x7FF0000000000000ull;
  // the implicit one of mant adds 1 to E - 1; a rounding carry to 2^53 adds one more
  return sign | ((((unsigned long long)(E - 1)) << 52) + mant);
}

// The same value through the hardware conversion: I to FP64 (rounded to
// nearest even), then 2^sc added to the exponent field (exact: the results
// of a state-vector merge lie far inside the normal range).
__device__ __forceinline__ unsigned long long oz_to_f64_cvt(long long I, int sc) {
  if (I == 0) return 0ull;
  double d;
  asm("cvt.rn.f64.s64 %0, %1;" : "=d"(d) : "l"(I));
  return (unsigned long long)__double_as_longlong(d) + ((unsigned long long)(long long)sc << 52);
}

template <int KBB, int NST, int BN, int NACC, int NBUF, int EW, int CVT>
__global__ void __launch_bounds__(64 + 32 * EW, 1)
    merge_ozaki_kernel(const __grid_constant__ CUtensorMap map_r,
                       const __grid_constant__ CUtensorMap map_c,
                       const __grid_constant__ CUtensorMap map_out,
                       const int32_t* __restrict__ e_row, const int32_t* __restrict__ f_col,
                       const double* out, int n_rows, int n_cols, int kblocks, int group_kb,
                       int* err) {
  using Cfg = OzCfg<KBB, NST, BN, NACC, NBUF, EW>;
  constexpr int KEL = Cfg::KEL, AS = Cfg::AS, BS = Cfg::BS, STB = Cfg::STB;
  constexpr int FIX = Cfg::FIX;
  static_assert((2 * NST + 2 * NBUF + 3) * 8 <= 256, "barrier area");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* stg_base = smem + NST * STB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg_base + Cfg::STG);
  uint64_t* full = bars;                        // [NST]
  uint64_t* empty = bars + NST;                 // [NST]
  uint64_t* tfull = bars + 2 * NST;             // [NBUF] accumulator set holds a finished group
  uint64_t* tempty = bars + 2 * NST + NBUF;     // [NBUF] the epilogue has read it
  uint64_t* drain = bars + 2 * NST + 2 * NBUF;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(drain + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = n_rows / OZ_BM, tiles_n = n_cols / BN;
  const int n_tiles = tiles_m * tiles_n;
  const int n_groups = (kblocks + group_kb - 1) / group_kb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EW);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(Cfg::TMEM)
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
        oz_tile_coords(t, tiles_m, tiles_n, BN, m0, n0);
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
      constexpr uint32_t idesc = oz_idesc<BN>();
      int s = 0;
      uint32_t use = 0;
      int iter = 0;
      bool ok = true;
      bool any_mma = false;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int kb0 = 0; kb0 < kblocks && ok; kb0 += group_kb, ++iter) {
          const int ab = iter % NBUF;
          if (!mbar_wait(&tempty[ab], ((iter / NBUF) & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dbase = tmem_base + (uint32_t)(ab * NACC * BN);
          uint32_t fresh = (1u << NACC) - 1;  // accumulators not yet written in this group
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
                  const int acc = min(i + j, NACC - 1);
                  const uint64_t b = sdesc_sw<KBB>(st + OZ_S * AS + j * BS) + adv;
                  const uint32_t accumulate = (fresh >> acc) & 1u ? 0u : 1u;
                  fresh &= ~(1u << acc);
                  umma<CC_MERGE_BF16X3>(dbase + (uint32_t)(acc * BN), a, b, idesc, accumulate);
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
          umma_commit(&tfull[ab]);
        }
      }
      if (!ok && any_mma) {
        umma_commit(drain);
        mbar_drain(drain, 0);
      }
    }
  } else {
    // epilogue warps 2 .. EW + 1: TMEM lane quarter = warp % 4, one output row
    // per lane; the EW / 4 warps of a quarter split the tile's columns
    const int quarter = warp & 3;
    const int part = (warp - 2) >> 2;
    const int c_begin = part * (Cfg::COLS_PER_WARP / 16);
    const int c_end = c_begin + Cfg::COLS_PER_WARP / 16;
    unsigned char* stg = stg_base + (warp - 2) * 2 * OZ_STG_BYTES;
    int buf = 0;
    int iter = 0;
    bool ok_all = true;
    for (int t = blockIdx.x; t < n_tiles && ok_all; t += gridDim.x) {
      int m0, n0;
      oz_tile_coords(t, tiles_m, tiles_n, BN, m0, n0);
      const int y = m0 + quarter * 32 + lane;
      const int ey = e_row[y] - 2 * (OZ_BETA - 1) - FIX;  // exponent of one fixed-point unit
      const long long* orow = reinterpret_cast<const long long*>(out) + (int64_t)y * n_cols + n0;
      for (int g = 0; g < n_groups; ++g, ++iter) {
        const int ab = iter % NBUF;
        int ok = 1;
        if (lane == 0) ok = mbar_wait(&tfull[ab], (iter / NBUF) & 1, abort_flag, err) ? 1 : 0;
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
        const uint32_t tbase =
            tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * NACC * BN);
#pragma unroll 1
        for (int c = c_begin; c < c_end; ++c) {
          uint32_t r[NACC][16];
#pragma unroll
          for (int L = 0; L < NACC; ++L) tmem_ld16(tbase + L * BN + c * 16, r[L]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (c == c_end - 1) {  // every accumulator value is in registers: free the set
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[ab]);
          }
          long long v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float a[NACC];
#pragma unroll
            for (int L = 0; L < NACC; ++L) a[L] = __uint_as_float(r[L][j]);
            v[j] = oz_fixed<NACC, FIX>(a);
          }
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
              if (CVT) {
                w[4 * q4 + 0] = oz_to_f64_cvt(v[4 * q4 + 0], ey + f.x);
                w[4 * q4 + 1] = oz_to_f64_cvt(v[4 * q4 + 1], ey + f.y);
                w[4 * q4 + 2] = oz_to_f64_cvt(v[4 * q4 + 2], ey + f.z);
                w[4 * q4 + 3] = oz_to_f64_cvt(v[4 * q4 + 3], ey + f.w);
              } else {
                w[4 * q4 + 0] = oz_to_f64(v[4 * q4 + 0], ey + f.x);
                w[4 * q4 + 1] = oz_to_f64(v[4 * q4 + 1], ey + f.y);
                w[4 * q4 + 2] = oz_to_f64(v[4 * q4 + 2], ey + f.z);
                w[4 * q4 + 3] = oz_to_f64(v[4 * q4 + 3], ey + f.w);
              }
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
                 "r"(Cfg::TMEM)
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

// Kernel configurations (K bytes per stage, stages, columns per tile,
// accumulators, accumulator sets, epilogue warps, FP64 conversion).
// Measured at q = 30 (merge ms for K = 4 / 64 / 256 terms):
//   0  64-column tiles, 4 accumulators, 2 sets, 8 epilogue warps, hardware
//      int64 -> FP64 conversion: 7.3 / 11.8 / 49.3 (max|dpsi|/max|psi| up to
//      4.4e-13 at K = 256, 1.6e-12 at K = 4096: the merged levels' rounding
//      grows with K);
//   1  the same with 5 accumulators (levels 0-3 exact, 4-5 merged), 1 set:
//      8.4 / 15.6 / 64.9, errors near 2e-14 at every K;
//   2  128-column tiles, 4 accumulators, 1 set, 4 epilogue warps, integer
//      conversion: 15.7 / 19.7 / 64.8;
//   3  configuration 0 with the integer conversion: 9.9 / 13.0 / 50.1.
// The default takes 0 while K <= 64 (one accumulation group) and 1 beyond;
// CUTSIM_OZ_CFG selects one by index.
struct OzChoice {
  int kbb, nst, bn, nacc, nbuf, ew, cvt;
  const void* fn;
  int smem, threads;
};
template <int KBB, int NST, int BN, int NACC, int NBUF, int EW, int CVT>
OzChoice oz_choice() {
  using Cfg = OzCfg<KBB, NST, BN, NACC, NBUF, EW>;
  return {KBB, NST, BN, NACC, NBUF, EW, CVT,
          reinterpret_cast<const void*>(merge_ozaki_kernel<KBB, NST, BN, NACC, NBUF, EW, CVT>),
          Cfg::SMEM, Cfg::THREADS};
}
const OzChoice* oz_choices(int* n) {
  static const OzChoice c[] = {
      oz_choice<64, 2, 64, 4, 2, 8, 1>(),   // 0
      oz_choice<64, 2, 64, 5, 1, 8, 1>(),   // 1
      oz_choice<64, 2, 128, 4, 1, 4, 0>(),  // 2
      oz_choice<64, 2, 64, 4, 2, 8, 0>(),   // 3
  };
  *n = (int)(sizeof(c) / sizeof(c[0]));
  return c;
}
int oz_choice_for(int64_t K) {
  const char* e = std::getenv("CUTSIM_OZ_CFG");
  int n = 0;
  oz_choices(&n);
  if (e) {
    const int v = std::atoi(e);
    if (v >= 0 && v < n) return v;
  }
  return K <= OZ_GROUP_K / 2 ? 0 : 1;
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

  // 64 operand rows per block: NB of R and 2 NA of Cop (NB, NA >= 2^7)
  const int64_t blocks = NB / kOzRows + 2 * NA / kOzRows;
  ozaki_split<<<(unsigned)blocks, 256, 0, s>>>(
      (const double2*)st.A, (const double2*)st.B, st.qa, st.qb, (int)st.K, KR, st.aidx, st.bidx,
      r_sl, c_sl, e_row, f_col);

  int n_choices = 0;
  const OzChoice& cfg = oz_choices(&n_choices)[oz_choice_for(st.K)];
  const int kbb = cfg.kbb;
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
    const cuuint32_t box[3] = {(cuuint32_t)kel, (cuuint32_t)cfg.bn, (cuuint32_t)OZ_S};
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
    const OzChoice* all = oz_choices(&n_choices);
    for (int i = 0; i < n_choices; ++i)
      cudaFuncSetAttribute(all[i].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, all[i].smem);
    attr_done[dev] = 1;
  }
  const int n_rows = (int)NB, n_cols = (int)(2 * NA);
  const int n_tiles = (n_rows / OZ_BM) * (n_cols / cfg.bn);
  const int grid = std::min(n_tiles, num_sms());
  int kblocks = KR / kel;
  int group_kb = OZ_GROUP_K / kel;
  const double* outp = static_cast<const double*>(st.out);
  void* args[] = {&map_r, &map_c, &map_out, &e_row, &f_col, &outp, (void*)&n_rows, (void*)&n_cols,
                  &kblocks, &group_kb, &err};
  const cudaError_t le = cudaLaunchKernel(cfg.fn, dim3((unsigned)grid), dim3((unsigned)cfg.threads), args,
                                          (size_t)cfg.smem, s);
  if (le != cudaSuccess)
    return fail(CC_ECUDA, std::string("Ozaki merge launch: ") + cudaGetErrorString(le));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("Ozaki merge launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

}  // namespace cc
