// Merging (Algorithm 3) on CUDA cores.
//
// For two factors the sum over cut combinations is a complex outer-product
// sum: with x the index of the lower factor (NA = 2^qa amplitudes) and y that
// of the upper one, out[y * NA + x] = sum_k A_k[x] * B_k[y].  The output is
// written exactly once, so for few terms this is a pure store stream; the
// factors (K * (NA + NB) amplitudes) stay in L2.
//
// Tiled form: a CTA owns a 32 x 128 (complex64) or 32 x 64 (complex128) block
// of the output, stages chunks of the factors' rows in shared memory and keeps
// an 8 x 2 (8 x 1) register block of accumulators per thread; stores are
// 16-byte streaming stores, each warp writing 512 contiguous bytes per row.
// The wide form (complex64, K <= 8, a small lower factor) drops the staging:
// 8 x 512 tiles read straight from L2 and written with no barrier.  The flat
// form (one output per thread) covers factors too short for a tile.  The
// tiled and flat forms take per-term row tables so that one kernel also
// serves the batched stages of the chained merge for three or more segments.
//
// Accumulation (complex64): terms are summed in FP32 chunks of KC; when there
// is more than one chunk, each chunk total is added to a running (hi, lo)
// pair with Knuth's TwoSum, so the rounding error grows with the chunk length
// and the number of chunks instead of with K.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "internal.h"

namespace cc {

namespace {

constexpr int KC = 32;  // terms staged per chunk

__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// Knuth's TwoSum: hi + lo += x with the rounding error of the add kept in lo.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}
__device__ __forceinline__ void two_sum_add(float2& hi, float2& lo, float2 x) {
  two_sum_add(hi.x, lo.x, x.x);
  two_sum_add(hi.y, lo.y, x.y);
}

__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// complex64 tile: 4*RPT rows (y) x 128 columns (x) of out_z (the output of
// one batch entry z); 256 threads = 64 column pairs x 4 row groups of RPT rows.
template <bool COMP, int RPT>
__device__ __forceinline__ void tile_c64(const float2* __restrict__ A, const float2* __restrict__ B,
                                         float2* __restrict__ out_z, int64_t NA, int64_t NB,
                                         int64_t K, const int32_t* __restrict__ ai,
                                         const int32_t* __restrict__ bi, int64_t y0, int64_t x0,
                                         float2 (*As)[128], float2 (*Bs)[4 * RPT]) {
  const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
  float2 acc[RPT][2], hi[COMP ? RPT : 1][2], lo[COMP ? RPT : 1][2];
#pragma unroll
  for (int i = 0; i < (COMP ? RPT : 1); ++i)
    hi[i][0] = hi[i][1] = lo[i][0] = lo[i][1] = make_float2(0.f, 0.f);
  for (int64_t k0 = 0; k0 < K; k0 += KC) {
    const int kc = (int)((K - k0) < KC ? (K - k0) : KC);
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
    for (int e = tid; e < kc * 64; e += 256) {
      const int kk = e >> 6, c = e & 63;
      const float4 v = *reinterpret_cast<const float4*>(A + (int64_t)ai[k0 + kk] * NA + x0 + 2 * c);
      *reinterpret_cast<float4*>(&As[kk][2 * c]) = v;
    }
    for (int e = tid; e < kc * 2 * RPT; e += 256) {
      const int kk = e / (2 * RPT), c = e % (2 * RPT);
      const float4 v = *reinterpret_cast<const float4*>(B + (int64_t)bi[k0 + kk] * NB + y0 + 2 * c);
      *reinterpret_cast<float4*>(&Bs[kk][2 * c]) = v;
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][2 * tx]);
      const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
#pragma unroll
      for (int i = 0; i < RPT; i += 2) {
        const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][ty * RPT + i]);
        const float2 b0 = make_float2(b.x, b.y), b1 = make_float2(b.z, b.w);
        cfma(acc[i][0], a0, b0);
        cfma(acc[i][1], a1, b0);
        cfma(acc[i + 1][0], a0, b1);
        cfma(acc[i + 1][1], a1, b1);
      }
    }
    __syncthreads();
    if (COMP) {
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        two_sum_add(hi[i][0], lo[i][0], acc[i][0]);
        two_sum_add(hi[i][1], lo[i][1], acc[i][1]);
      }
    }
  }
  if (COMP) {
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      acc[i][0] = make_float2(hi[i][0].x + lo[i][0].x, hi[i][0].y + lo[i][0].y);
      acc[i][1] = make_float2(hi[i][1].x + lo[i][1].x, hi[i][1].y + lo[i][1].y);
    }
  }
  float2* o = out_z + (y0 + ty * RPT) * NA + x0 + 2 * tx;
#pragma unroll
  for (int i = 0; i < RPT; ++i)
    __stcs(reinterpret_cast<float4*>(o + i * NA),
           make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y));
}

// Few terms (K <= 8): a pure store stream.  A CTA owns 8 rows x 512 columns
// of the output (each row a 4 KB contiguous run), each thread 2 columns of
// every row; the factors' values come straight from L2 (the lower factor's
// two values per term with one 16-byte load, the upper factor's eight row
// values with warp-uniform loads), so there is no shared-memory staging and
// no barrier between tiles.
constexpr int kWideRows = 8;
constexpr int kWideCols = 512;
template <int K>  // 1, 2, 4 or 8: the term loop unrolls and its loads issue together
__global__ void __launch_bounds__(256)
    merge_wide_c64(const float2* __restrict__ A, const float2* __restrict__ B,
                   float2* __restrict__ out, int qa, int qb,
                   const int32_t* __restrict__ aidx, const int32_t* __restrict__ bidx) {
  const int64_t NA = int64_t(1) << qa, NB = int64_t(1) << qb;
  const int64_t tiles_x = NA / kWideCols, n_tiles = tiles_x * (NB / kWideRows);
  const int t = threadIdx.x;
  for (int64_t w = blockIdx.x; w < n_tiles; w += gridDim.x) {
    const int64_t y0 = (w / tiles_x) * kWideRows, x0 = (w % tiles_x) * kWideCols + 2 * t;
    float2 acc[kWideRows][2];
#pragma unroll
    for (int r = 0; r < kWideRows; ++r) acc[r][0] = acc[r][1] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(A + (int64_t)aidx[k] * NA + x0));
      const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
      const float4* brow = reinterpret_cast<const float4*>(B + (int64_t)bidx[k] * NB + y0);
#pragma unroll
      for (int r = 0; r < kWideRows; r += 2) {
        const float4 b = __ldg(brow + r / 2);
        const float2 b0 = make_float2(b.x, b.y), b1 = make_float2(b.z, b.w);
        cfma(acc[r][0], a0, b0);
        cfma(acc[r][1], a1, b0);
        cfma(acc[r + 1][0], a0, b1);
        cfma(acc[r + 1][1], a1, b1);
      }
    }
    float2* o = out + y0 * NA + x0;
#pragma unroll
    for (int r = 0; r < kWideRows; ++r)
      __stcs(reinterpret_cast<float4*>(o + r * NA),
             make_float4(acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y));
  }
}

template <bool COMP>
__global__ void __launch_bounds__(256)
    merge_tile_c64(const float2* __restrict__ A, const float2* __restrict__ B,
                   float2* __restrict__ out, int qa, int qb, int64_t K, int64_t Z,
                   int64_t out_stride, const int32_t* __restrict__ aidx,
                   const int32_t* __restrict__ bidx) {
  __shared__ __align__(16) float2 As[KC][128];
  __shared__ __align__(16) float2 Bs[KC][32];
  const int64_t NA = int64_t(1) << qa, NB = int64_t(1) << qb;
  const int64_t tiles_x = NA >> 7, tiles_y = NB >> 5;
  const int64_t n_tiles = tiles_x * tiles_y * Z;
  for (int64_t w = blockIdx.x; w < n_tiles; w += gridDim.x) {
    const int64_t z = w / (tiles_x * tiles_y);
    const int64_t rem = w - z * tiles_x * tiles_y;
    const int64_t y0 = (rem / tiles_x) << 5, x0 = (rem % tiles_x) << 7;
    tile_c64<COMP, 8>(A, B, out + z * out_stride, NA, NB, K, aidx + z * K, bidx + z * K, y0, x0,
                      As, Bs);
  }
}

// complex128 tile: 32 rows x 64 columns; 256 threads = 64 columns x 4 row groups.
__device__ __forceinline__ void tile_c128(const double2* __restrict__ A,
                                          const double2* __restrict__ B,
                                          double2* __restrict__ out_z, int64_t NA, int64_t NB,
                                          int64_t K, const int32_t* __restrict__ ai,
                                          const int32_t* __restrict__ bi, int64_t y0, int64_t x0,
                                          double2 (*As)[64], double2 (*Bs)[32]) {
  const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
  double2 acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = make_double2(0.0, 0.0);
  for (int64_t k0 = 0; k0 < K; k0 += KC) {
    const int kc = (int)((K - k0) < KC ? (K - k0) : KC);
    for (int e = tid; e < kc * 64; e += 256) {
      const int kk = e >> 6, c = e & 63;
      As[kk][c] = A[(int64_t)ai[k0 + kk] * NA + x0 + c];
    }
    for (int e = tid; e < kc * 32; e += 256) {
      const int kk = e >> 5, c = e & 31;
      Bs[kk][c] = B[(int64_t)bi[k0 + kk] * NB + y0 + c];
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      const double2 a = As[kk][tx];
#pragma unroll
      for (int i = 0; i < 8; ++i) cfma(acc[i], a, Bs[kk][ty * 8 + i]);
    }
    __syncthreads();
  }
  double2* o = out_z + (y0 + ty * 8) * NA + x0 + tx;
#pragma unroll
  for (int i = 0; i < 8; ++i) __stcs(o + i * NA, acc[i]);
}

__global__ void __launch_bounds__(256)
    merge_tile_c128(const double2* __restrict__ A, const double2* __restrict__ B,
                    double2* __restrict__ out, int qa, int qb, int64_t K, int64_t Z,
                    int64_t out_stride, const int32_t* __restrict__ aidx,
                    const int32_t* __restrict__ bidx) {
  __shared__ __align__(16) double2 As[KC][64];
  __shared__ __align__(16) double2 Bs[KC][32];
  const int64_t NA = int64_t(1) << qa, NB = int64_t(1) << qb;
  const int64_t tiles_x = NA >> 6, tiles_y = NB >> 5;
  const int64_t n_tiles = tiles_x * tiles_y * Z;
  for (int64_t w = blockIdx.x; w < n_tiles; w += gridDim.x) {
    const int64_t z = w / (tiles_x * tiles_y);
    const int64_t rem = w - z * tiles_x * tiles_y;
    const int64_t y0 = (rem / tiles_x) << 5, x0 = (rem % tiles_x) << 6;
    tile_c128(A, B, out + z * out_stride, NA, NB, K, aidx + z * K, bidx + z * K, y0, x0, As, Bs);
  }
}

__device__ __forceinline__ void add_chunk(float2& hi, float2& lo, float2 x) { two_sum_add(hi, lo, x); }
__device__ __forceinline__ void add_chunk(double2& hi, double2&, double2 x) {
  hi.x += x.x;
  hi.y += x.y;
}

// One output amplitude per thread, any factor sizes.
template <typename C>
__global__ void __launch_bounds__(256)
    merge_flat(const C* __restrict__ A, const C* __restrict__ B, C* __restrict__ out, int qa,
               int qb, int64_t K, int64_t Z, int64_t out_stride, const int32_t* __restrict__ aidx,
               const int32_t* __restrict__ bidx) {
  const int64_t NA = int64_t(1) << qa, NB = int64_t(1) << qb;
  const int64_t per = NA * NB, total = per * Z;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = f / per, e = f - z * per;
    const int64_t x = e & (NA - 1), y = e >> qa;
    C hi, lo;
    hi.x = hi.y = lo.x = lo.y = 0;
    for (int64_t k0 = 0; k0 < K; k0 += KC) {
      const int64_t k1 = (K - k0) < KC ? K : k0 + KC;
      C acc;
      acc.x = acc.y = 0;
      for (int64_t k = k0; k < k1; ++k)
        cfma(acc, A[(int64_t)aidx[z * K + k] * NA + x], B[(int64_t)bidx[z * K + k] * NB + y]);
      add_chunk(hi, lo, acc);
    }
    hi.x += lo.x;
    hi.y += lo.y;
    out[z * out_stride + e] = hi;
  }
}

// One output amplitude of a merge stage, any factor sizes.
template <typename C>
__device__ __forceinline__ C flat_one(const C* __restrict__ A, const C* __restrict__ B, int qa,
                                      int64_t NA, int64_t NB, int64_t K,
                                      const int32_t* __restrict__ ai,
                                      const int32_t* __restrict__ bi, int64_t e) {
  const int64_t x = e & (NA - 1), y = e >> qa;
  C hi, lo;
  hi.x = hi.y = lo.x = lo.y = 0;
  for (int64_t k0 = 0; k0 < K; k0 += KC) {
    const int64_t k1 = (K - k0) < KC ? K : k0 + KC;
    C acc;
    acc.x = acc.y = 0;
    for (int64_t k = k0; k < k1; ++k) cfma(acc, A[(int64_t)ai[k] * NA + x], B[(int64_t)bi[k] * NB + y]);
    add_chunk(hi, lo, acc);
  }
  hi.x += lo.x;
  hi.y += lo.y;
  return hi;
}

__device__ __forceinline__ unsigned long long merge_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Batched merge: the units (output tiles, or runs of 256 amplitudes for
// factors too short for a tile) of many stage jobs in one grid-stride loop.
template <typename C, int RPT>
__global__ void __launch_bounds__(256)
    merge_batch_kernel(const BMergeJob* __restrict__ jobs, int n_jobs, long long n_units,
                       C* seg, C* work, C* psi, int* __restrict__ circ_done,
                       unsigned long long* __restrict__ stamps) {
  constexpr bool F32 = sizeof(C) == 8;
  constexpr int TX = F32 ? 128 : 64, TY = F32 ? 4 * RPT : 32;
  __shared__ __align__(16) C As[KC][TX];
  __shared__ __align__(16) C Bs[KC][TY];
  for (long long w = blockIdx.x; w < n_units; w += gridDim.x) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].unit_begin <= w) lo = mid; else hi = mid - 1;
    }
    const BMergeJob& J = jobs[lo];
    C* const bufs[3] = {seg, work, psi};
    const C* A = bufs[J.a_buf] + J.a_off;
    const C* B = bufs[J.b_buf] + J.b_off;
    C* out = bufs[J.out_buf] + J.out_off;
    const int64_t NA = int64_t(1) << J.qa, NB = int64_t(1) << J.qb;
    const int64_t u = w - J.unit_begin;
    if (J.kind == 0) {
      const int64_t tiles_x = NA / TX, tiles_y = NB / TY;
      const int64_t z = u / (tiles_x * tiles_y);
      const int64_t rem = u - z * tiles_x * tiles_y;
      const int64_t y0 = (rem / tiles_x) * TY, x0 = (rem % tiles_x) * TX;
      if constexpr (F32) {
        if (J.K > KC)
          tile_c64<true, RPT>(A, B, out + z * J.out_stride, NA, NB, J.K, J.aidx + z * J.K,
                              J.bidx + z * J.K, y0, x0, As, Bs);
        else
          tile_c64<false, RPT>(A, B, out + z * J.out_stride, NA, NB, J.K, J.aidx + z * J.K,
                               J.bidx + z * J.K, y0, x0, As, Bs);
      } else {
        tile_c128(A, B, out + z * J.out_stride, NA, NB, J.K, J.aidx + z * J.K, J.bidx + z * J.K,
                  y0, x0, As, Bs);
      }
    } else {
      const int64_t per = NA * NB, f = u * 256 + threadIdx.x;
      if (f < per * J.Z) {
        const int64_t z = f / per, e = f - z * per;
        out[z * J.out_stride + e] =
            flat_one<C>(A, B, J.qa, NA, NB, J.K, J.aidx + z * J.K, J.bidx + z * J.K, e);
      }
    }
    if (J.circ >= 0 && stamps) {
      // counts units whose stores were issued; no fence, so the stamp may
      // precede the last stores' arrival in memory by their latency
      __syncthreads();
      if (threadIdx.x == 0) {
        const int v = atomicAdd(circ_done + J.circ, 1);
        if (v + 1 == J.n_units) stamps[1 + J.circ] = merge_timer();
      }
    }
  }
}

}  // namespace

cc_status launch_merge_fma(const MergeStage& st, int precision, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t NA = int64_t(1) << st.qa, NB = int64_t(1) << st.qb;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (precision == CC_C64) {
    const char* wide_env = std::getenv("CUTSIM_MERGE_WIDE");
    const bool wide_ok = !(wide_env && wide_env[0] == '0');
    // the wide form re-reads the lower factor once per 8 output rows (the
    // tile form once per 32), so it is taken while the lower factor's K terms
    // are small: q = 30 K = 4 1.81 -> 1.62 ms, K = 2 1.46 -> 1.26 ms; the
    // last stage of an n = 3 chain with K * NA = 2^22 ran 1.86 -> 1.93 ms
    if (wide_ok && st.Z == 1 && (st.K == 1 || st.K == 2 || st.K == 4 || st.K == 8) &&
        st.qa >= 9 && st.qb >= 3 && st.K * NA <= (int64_t(1) << 21)) {
      const int64_t tiles = (NA / kWideCols) * (NB / kWideRows);
      auto kern = st.K == 1 ? merge_wide_c64<1> : st.K == 2 ? merge_wide_c64<2>
                : st.K == 4 ? merge_wide_c64<4> : merge_wide_c64<8>;
      kern<<<(unsigned)std::min(tiles, cap), 256, 0, s>>>(
          (const float2*)st.A, (const float2*)st.B, (float2*)st.out, st.qa, st.qb, st.aidx,
          st.bidx);
    } else if (st.qa >= 7 && st.qb >= 5) {
      const int64_t tiles = (NA >> 7) * (NB >> 5) * st.Z;
      auto kern = st.K > KC ? merge_tile_c64<true> : merge_tile_c64<false>;
      kern<<<(unsigned)std::min(tiles, cap), 256, 0, s>>>(
          (const float2*)st.A, (const float2*)st.B, (float2*)st.out, st.qa, st.qb, st.K, st.Z,
          st.out_stride, st.aidx, st.bidx);
    } else {
      const int64_t blocks = std::min((NA * NB * st.Z + 255) / 256, cap);
      merge_flat<float2><<<(unsigned)blocks, 256, 0, s>>>(
          (const float2*)st.A, (const float2*)st.B, (float2*)st.out, st.qa, st.qb, st.K, st.Z,
          st.out_stride, st.aidx, st.bidx);
    }
  } else {
    if (st.qa >= 6 && st.qb >= 5) {
      const int64_t tiles = (NA >> 6) * (NB >> 5) * st.Z;
      merge_tile_c128<<<(unsigned)std::min(tiles, cap), 256, 0, s>>>(
          (const double2*)st.A, (const double2*)st.B, (double2*)st.out, st.qa, st.qb, st.K, st.Z,
          st.out_stride, st.aidx, st.bidx);
    } else {
      const int64_t blocks = std::min((NA * NB * st.Z + 255) / 256, cap);
      merge_flat<double2><<<(unsigned)blocks, 256, 0, s>>>(
          (const double2*)st.A, (const double2*)st.B, (double2*)st.out, st.qa, st.qb, st.K, st.Z,
          st.out_stride, st.aidx, st.bidx);
    }
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("merge launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

}  // namespace cc

namespace cc {

int64_t merge_batch_units(int precision, int qa, int qb, int64_t Z, int rows, int32_t* kind) {
  const int64_t NA = int64_t(1) << qa, NB = int64_t(1) << qb;
  const int tx = precision == CC_C64 ? 128 : 64;
  const int ty = precision == CC_C64 ? rows : 32;
  if (NA >= tx && NB >= ty) {
    if (kind) *kind = 0;
    return (NA / tx) * (NB / ty) * Z;
  }
  if (kind) *kind = 1;
  return (NA * NB * Z + 255) / 256;
}

namespace {
__global__ void stamp_kernel(unsigned long long* out) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *out = t;
}
}  // namespace

cc_status launch_stamp(unsigned long long* out, void* stream) {
  stamp_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("stamp launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

cc_status launch_merge_batch(const BMergeJob* jobs, int n_jobs, int64_t n_units, void* seg_buf,
                             void* work, void* psi, int* circ_done, unsigned long long* stamps,
                             int precision, int rows, void* stream) {
  if (n_units <= 0 || n_jobs <= 0) return CC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t grid = std::min<int64_t>(n_units, (int64_t)num_sms() * 8);
  if (precision == CC_C128) {
    merge_batch_kernel<double2, 8><<<(unsigned)grid, 256, 0, s>>>(
        jobs, n_jobs, n_units, (double2*)seg_buf, (double2*)work, (double2*)psi, circ_done, stamps);
  } else if (rows == 16) {
    merge_batch_kernel<float2, 4><<<(unsigned)grid, 256, 0, s>>>(
        jobs, n_jobs, n_units, (float2*)seg_buf, (float2*)work, (float2*)psi, circ_done, stamps);
  } else {
    merge_batch_kernel<float2, 8><<<(unsigned)grid, 256, 0, s>>>(
        jobs, n_jobs, n_units, (float2*)seg_buf, (float2*)work, (float2*)psi, circ_done, stamps);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(CC_ECUDA, std::string("batched merge launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

}  // namespace cc
