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
// The flat form (one output per thread) covers factors too short for a tile.
// Both take per-term row tables so that one kernel also serves the batched
// stages of the chained merge for three or more segments.
//
// Accumulation (complex64): terms are summed in FP32 chunks of KC; when there
// is more than one chunk, each chunk total is added to a running (hi, lo)
// pair with Knuth's TwoSum, so the rounding error grows with the chunk length
// and the number of chunks instead of with K.
#include <cuda_runtime.h>

#include <algorithm>

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

// complex64 tile: 32 rows (y) x 128 columns (x); 256 threads = 64 column pairs x 4 row groups.
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
  const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
  for (int64_t w = blockIdx.x; w < n_tiles; w += gridDim.x) {
    const int64_t z = w / (tiles_x * tiles_y);
    const int64_t rem = w - z * tiles_x * tiles_y;
    const int64_t y0 = (rem / tiles_x) << 5, x0 = (rem % tiles_x) << 7;
    const int32_t* ai = aidx + z * K;
    const int32_t* bi = bidx + z * K;
    float2 acc[8][2], hi[COMP ? 8 : 1][2], lo[COMP ? 8 : 1][2];
#pragma unroll
    for (int i = 0; i < (COMP ? 8 : 1); ++i)
      hi[i][0] = hi[i][1] = lo[i][0] = lo[i][1] = make_float2(0.f, 0.f);
    for (int64_t k0 = 0; k0 < K; k0 += KC) {
      const int kc = (int)((K - k0) < KC ? (K - k0) : KC);
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
      for (int e = tid; e < kc * 64; e += 256) {
        const int kk = e >> 6, c = e & 63;
        const float4 v = *reinterpret_cast<const float4*>(A + (int64_t)ai[k0 + kk] * NA + x0 + 2 * c);
        *reinterpret_cast<float4*>(&As[kk][2 * c]) = v;
      }
      for (int e = tid; e < kc * 16; e += 256) {
        const int kk = e >> 4, c = e & 15;
        const float4 v = *reinterpret_cast<const float4*>(B + (int64_t)bi[k0 + kk] * NB + y0 + 2 * c);
        *reinterpret_cast<float4*>(&Bs[kk][2 * c]) = v;
      }
      __syncthreads();
      for (int kk = 0; kk < kc; ++kk) {
        const float4 a = *reinterpret_cast<const float4*>(&As[kk][2 * tx]);
        const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][ty * 8 + i]);
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
        for (int i = 0; i < 8; ++i) {
          two_sum_add(hi[i][0], lo[i][0], acc[i][0]);
          two_sum_add(hi[i][1], lo[i][1], acc[i][1]);
        }
      }
    }
    if (COMP) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        acc[i][0] = make_float2(hi[i][0].x + lo[i][0].x, hi[i][0].y + lo[i][0].y);
        acc[i][1] = make_float2(hi[i][1].x + lo[i][1].x, hi[i][1].y + lo[i][1].y);
      }
    }
    float2* o = out + z * out_stride + (y0 + ty * 8) * NA + x0 + 2 * tx;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      __stcs(reinterpret_cast<float4*>(o + i * NA),
             make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y));
  }
}

// complex128 tile: 32 rows x 64 columns; 256 threads = 64 columns x 4 row groups.
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
  const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
  for (int64_t w = blockIdx.x; w < n_tiles; w += gridDim.x) {
    const int64_t z = w / (tiles_x * tiles_y);
    const int64_t rem = w - z * tiles_x * tiles_y;
    const int64_t y0 = (rem / tiles_x) << 5, x0 = (rem % tiles_x) << 6;
    const int32_t* ai = aidx + z * K;
    const int32_t* bi = bidx + z * K;
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
    double2* o = out + z * out_stride + (y0 + ty * 8) * NA + x0 + tx;
#pragma unroll
    for (int i = 0; i < 8; ++i) __stcs(o + i * NA, acc[i]);
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

}  // namespace

cc_status launch_merge_fma(const MergeStage& st, int precision, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t NA = int64_t(1) << st.qa, NB = int64_t(1) << st.qb;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (precision == CC_C64) {
    if (st.qa >= 7 && st.qb >= 5) {
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
