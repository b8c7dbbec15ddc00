// FP64 verification reductions (max |a - b|, max |b|, <a|b>, <a|a>, <b|b>) and
// the sampled-amplitude gather.  complex128 inputs: every product and sum in
// FP64.  complex64 inputs: exact FP32 products, double-float runs, FP64
// across runs (see compare_partial_c64).
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace cc {

namespace {

constexpr int RB = 256;  // threads per reduction block

struct Acc6 {
  double d2, b2, re, im, na, nb;  // max |a-b|^2, max |b|^2, Re<a|b>, Im<a|b>, <a|a>, <b|b>
};

__device__ __forceinline__ void combine(Acc6& x, const Acc6& y) {
  x.d2 = fmax(x.d2, y.d2);
  x.b2 = fmax(x.b2, y.b2);
  x.re += y.re;
  x.im += y.im;
  x.na += y.na;
  x.nb += y.nb;
}

__device__ __forceinline__ Acc6 shfl_xor(const Acc6& a, int m) {
  Acc6 r;
  r.d2 = __shfl_xor_sync(0xffffffffu, a.d2, m);
  r.b2 = __shfl_xor_sync(0xffffffffu, a.b2, m);
  r.re = __shfl_xor_sync(0xffffffffu, a.re, m);
  r.im = __shfl_xor_sync(0xffffffffu, a.im, m);
  r.na = __shfl_xor_sync(0xffffffffu, a.na, m);
  r.nb = __shfl_xor_sync(0xffffffffu, a.nb, m);
  return r;
}

__device__ Acc6 block_reduce(Acc6 v) {
  __shared__ Acc6 sh[RB / 32];
  for (int m = 16; m >= 1; m >>= 1) combine(v, shfl_xor(v, m));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < RB / 32) ? sh[lane] : Acc6{0, 0, 0, 0, 0, 0};
    for (int m = 16; m >= 1; m >>= 1) combine(v, shfl_xor(v, m));
  }
  return v;
}

// Double-float accumulator (hi + lo, two FP32): exact products via FMA
// (Dekker's TwoProduct) added with Knuth's TwoSum, so a run of R products
// carries a relative error of about R * 2^-48 instead of R * 2^-24.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ void df_add_prod(DF& s, float x, float y) {
  const float p = x * y;
  const float e = fmaf(x, y, -p);  // x*y = p + e exactly
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}
__device__ __forceinline__ double df_value(const DF& s) { return (double)s.hi + (double)s.lo; }

constexpr int kRun = 64;  // elements per thread between FP64 accumulations

// One element of the complex64 comparison: the maxima in FP32, the four
// sums as exact products added in double-float.
__device__ __forceinline__ void cmp_elem(float ar, float ai, float br, float bi, float& d2,
                                         float& b2, DF& re, DF& im, DF& na, DF& nb) {
  const float dr = ar - br, di = ai - bi;
  d2 = fmaxf(d2, fmaf(dr, dr, di * di));
  b2 = fmaxf(b2, fmaf(br, br, bi * bi));
  df_add_prod(re, ar, br);  // Re conj(a) b = ar br + ai bi
  df_add_prod(re, ai, bi);
  df_add_prod(im, ar, bi);  // Im conj(a) b = ar bi - ai br
  df_add_prod(im, -ai, br);
  df_add_prod(na, ar, ar);
  df_add_prod(na, ai, ai);
  df_add_prod(nb, br, br);
  df_add_prod(nb, bi, bi);
}

// complex64 inputs: the products are formed exactly in FP32 and summed in
// double-float over runs of kRun elements per thread; each run's sum is then
// added in FP64.  GB300's FP64 rate (1/64 of FP32) would otherwise bound the
// pass at ~20 FP64 operations per element, far below the HBM rate.  The
// maxima are taken in FP32 (the differences of nearby FP32 values are
// exact; the squares carry 2^-24 relative error).  Each thread reads two
// amplitudes per 16-byte load (the buffers are 16-byte aligned) with kLoads
// loads of each vector in flight before any arithmetic; an odd last
// amplitude is added by thread 0 of block 0.
constexpr int kLoads = 4;
__global__ void __launch_bounds__(RB)
    compare_partial_c64(const float2* __restrict__ a, const float2* __restrict__ b, int64_t n,
                        double* __restrict__ partials) {
  Acc6 v{0, 0, 0, 0, 0, 0};
  float d2 = 0.f, b2 = 0.f;
  const float4* __restrict__ a4 = reinterpret_cast<const float4*>(a);
  const float4* __restrict__ b4 = reinterpret_cast<const float4*>(b);
  const int64_t n2 = n >> 1;
  const int64_t stride = (int64_t)gridDim.x * RB;
  int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x;
  while (i < n2) {
    DF re{0.f, 0.f}, im{0.f, 0.f}, na{0.f, 0.f}, nb{0.f, 0.f};
#pragma unroll 1
    for (int r = 0; r < kRun / (2 * kLoads) && i < n2; ++r, i += kLoads * stride) {
      float4 x[kLoads], y[kLoads];
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        const int64_t j = i + u * stride;
        if (j < n2) {
          x[u] = __ldcs(a4 + j);
          y[u] = __ldcs(b4 + j);
        } else {  // zeros add nothing to any sum or maximum
          x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          y[u] = x[u];
        }
      }
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        cmp_elem(x[u].x, x[u].y, y[u].x, y[u].y, d2, b2, re, im, na, nb);
        cmp_elem(x[u].z, x[u].w, y[u].z, y[u].w, d2, b2, re, im, na, nb);
      }
    }
    v.re += df_value(re);
    v.im += df_value(im);
    v.na += df_value(na);
    v.nb += df_value(nb);
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    DF re{0.f, 0.f}, im{0.f, 0.f}, na{0.f, 0.f}, nb{0.f, 0.f};
    const float2 x = a[n - 1], y = b[n - 1];
    cmp_elem(x.x, x.y, y.x, y.y, d2, b2, re, im, na, nb);
    v.re += df_value(re);
    v.im += df_value(im);
    v.na += df_value(na);
    v.nb += df_value(nb);
  }
  v.d2 = d2;
  v.b2 = b2;
  v = block_reduce(v);
  if (threadIdx.x == 0) {
    double* p = partials + 8 * blockIdx.x;
    p[0] = v.d2; p[1] = v.b2; p[2] = v.re; p[3] = v.im; p[4] = v.na; p[5] = v.nb;
  }
}

template <typename C>
__global__ void __launch_bounds__(RB)
    compare_partial(const C* __restrict__ a, const C* __restrict__ b, int64_t n,
                    double* __restrict__ partials) {
  Acc6 v{0, 0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) {
    const C x = a[i], y = b[i];
    const double ar = x.x, ai = x.y, br = y.x, bi = y.y;
    const double dr = ar - br, di = ai - bi;
    v.d2 = fmax(v.d2, dr * dr + di * di);
    v.b2 = fmax(v.b2, br * br + bi * bi);
    v.re += ar * br + ai * bi;  // conj(a) b
    v.im += ar * bi - ai * br;
    v.na += ar * ar + ai * ai;
    v.nb += br * br + bi * bi;
  }
  v = block_reduce(v);
  if (threadIdx.x == 0) {
    double* p = partials + 8 * blockIdx.x;
    p[0] = v.d2; p[1] = v.b2; p[2] = v.re; p[3] = v.im; p[4] = v.na; p[5] = v.nb;
  }
}

__global__ void __launch_bounds__(RB) compare_final(const double* __restrict__ partials,
                                                    int n_blocks, double* __restrict__ out) {
  Acc6 v{0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < n_blocks; i += RB) {
    const double* p = partials + 8 * i;
    combine(v, Acc6{p[0], p[1], p[2], p[3], p[4], p[5]});
  }
  v = block_reduce(v);
  if (threadIdx.x == 0) {
    out[0] = sqrt(v.d2);
    out[1] = sqrt(v.b2);
    out[2] = v.re;
    out[3] = v.im;
    out[4] = v.na;
    out[5] = v.nb;
  }
}

template <typename C>
__global__ void gather_kernel(const C* __restrict__ psi, const int64_t* __restrict__ idx,
                              int64_t n, C* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = psi[idx[i]];
}

// Device -> host copy by the SMs themselves: 16-byte loads from HBM and
// 16-byte stores through the host buffer's mapped address (NVLink-C2C on a
// Grace host), four vectors in flight per thread.
__global__ void __launch_bounds__(256) copy_to_host_kernel(const int4* __restrict__ src,
                                                           int4* __restrict__ dst, int64_t n16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const int4 a = __ldcs(src + i), b = __ldcs(src + i + stride);
    const int4 c = __ldcs(src + i + 2 * stride), d = __ldcs(src + i + 3 * stride);
    dst[i] = a;
    dst[i + stride] = b;
    dst[i + 2 * stride] = c;
    dst[i + 3 * stride] = d;
  }
  for (; i < n16; i += stride) dst[i] = __ldcs(src + i);
}

// Polls a device word that nothing writes, `polls` times ~1 us apart, then
// raises the error flag the way an expired wait in the engine does.
__global__ void expired_wait_kernel(const int* __restrict__ never_set, int polls,
                                    int* __restrict__ err) {
  int seen = 0;
  for (int i = 0; i < polls && !seen; ++i) {
    seen = *(volatile const int*)never_set;
    __nanosleep(1000);
  }
  if (!seen) atomicExch(err, 1);
}

}  // namespace

cc_status launch_copy_to_host(const void* src, void* host_mapped, uint64_t bytes, void* stream) {
  const int64_t n16 = (int64_t)(bytes / 16);
  cudaStream_t s = (cudaStream_t)stream;
  if (n16 > 0) {
    const int64_t grid = std::min<int64_t>((n16 + 255) / 256, (int64_t)num_sms() * 8);
    copy_to_host_kernel<<<(unsigned)grid, 256, 0, s>>>(static_cast<const int4*>(src),
                                                       static_cast<int4*>(host_mapped), n16);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CC_ECUDA, std::string("copy launch: ") + cudaGetErrorString(e));
  }
  const uint64_t tail = bytes - (uint64_t)n16 * 16;
  if (tail) {
    const cudaError_t e = cudaMemcpyAsync(static_cast<char*>(host_mapped) + n16 * 16,
                                          static_cast<const char*>(src) + n16 * 16, tail,
                                          cudaMemcpyDefault, s);
    if (e != cudaSuccess) return fail(CC_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
  }
  return CC_OK;
}

cc_status launch_expired_wait(int polls, void* stream) {
  int* err = device_error_flag();
  if (!err) return fail(CC_ENOMEM, "device error flag allocation failed");
  int* word = static_cast<int*>(scratch(sizeof(int)));
  if (!word) return fail(CC_ENOMEM, "scratch allocation failed");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(word, 0, sizeof(int), s);
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("memset: ") + cudaGetErrorString(e));
  expired_wait_kernel<<<1, 1, 0, s>>>(word, polls, err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("wait probe launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

cc_status launch_compare(const void* a, const void* b, int64_t n, int precision, double* out_dev,
                         double* partials, int n_blocks, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == CC_C128)
    compare_partial<double2><<<n_blocks, RB, 0, s>>>((const double2*)a, (const double2*)b, n, partials);
  else
    compare_partial_c64<<<n_blocks, RB, 0, s>>>((const float2*)a, (const float2*)b, n, partials);
  compare_final<<<1, RB, 0, s>>>(partials, n_blocks, out_dev);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("compare launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

cc_status launch_gather(const void* psi, int precision, const int64_t* idx_dev, int64_t n,
                        void* out_dev, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)((n + 255) / 256);
  if (precision == CC_C128)
    gather_kernel<double2><<<blocks, 256, 0, s>>>((const double2*)psi, idx_dev, n, (double2*)out_dev);
  else
    gather_kernel<float2><<<blocks, 256, 0, s>>>((const float2*)psi, idx_dev, n, (float2*)out_dev);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CC_ECUDA, std::string("gather launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

}  // namespace cc
