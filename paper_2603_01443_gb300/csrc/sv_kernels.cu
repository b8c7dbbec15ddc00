// Gate passes over batched state vectors (subcircuit simulation, Algorithm 2,
// and the uncut simulation T_orig).
//
// One CTA owns one tile of 2^k amplitudes of one vector at a time: it loads
// the tile into shared memory with 16-byte vector loads (the lowest tile bits
// are contiguous vector bits, so every load is part of a >= 128-byte run),
// applies the pass's fused operations in shared memory, and stores the tile
// back in place.  The first pass of a program starts from |0...0> and reads
// nothing.  When the whole vector fits one tile (segments of up to 14 qubits
// in complex64, 13 in complex128) the program is a single pass and every
// variant of a segment is one CTA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "internal.h"

namespace cc {

template <typename R>
struct CT;
template <>
struct CT<float> {
  using C = float2;
  using V = float4;
  static constexpr int PV = 2;  // amplitudes per 16-byte vector
};
template <>
struct CT<double> {
  using C = double2;
  using V = double2;
  static constexpr int PV = 1;
};

template <typename R>
__device__ __forceinline__ void cmul(R& xr, R& xi, R yr, R yi) {
  const R t = xr * yr - xi * yi;
  xi = xr * yi + xi * yr;
  xr = t;
}

// Multiply amplitude a (virtual index v) by the diagonal factors of an op.
template <typename R>
__device__ __forceinline__ void apply_terms(typename CT<R>::C& a, uint64_t v,
                                            const DTerm* __restrict__ terms, int tb, int tse,
                                            int te, const R* __restrict__ tabs) {
  uint32_t sign = 0;
  for (int i = tb; i < tse; ++i) {
    const DTerm d = terms[i];
    sign ^= (uint32_t)((v >> d.p0) & (v >> d.p1)) & 1u;
  }
  if (te > tse) {
    R fr = R(1), fi = R(0);
    for (int i = tse; i < te; ++i) {
      const DTerm d = terms[i];
      const int idx = (int)((v >> d.p0) & 1u) | ((int)((v >> d.p1) & 1u) << 1);
      const R* t = tabs + 8 * d.tab + 2 * idx;
      cmul(fr, fi, t[0], t[1]);
    }
    cmul(a.x, a.y, fr, fi);
  }
  if (sign) {
    a.x = -a.x;
    a.y = -a.y;
  }
}

// Vector offset of tile row h (the tile bits above the contiguous low run).
__device__ __forceinline__ int64_t tile_row_offset(uint32_t h, const int8_t* __restrict__ hi_bits) {
  int64_t g = 0;
  for (int t = 0; h; ++t, h >>= 1)
    if (h & 1u) g |= int64_t(1) << hi_bits[t];
  return g;
}

template <typename R>
__global__ void __launch_bounds__(1024)
    pass_kernel(typename CT<R>::C* __restrict__ state, int64_t vec_stride,
                const DPass* __restrict__ pass, const DOp* __restrict__ ops,
                const DTerm* __restrict__ terms, const R* __restrict__ mats,
                const R* __restrict__ tabs, int64_t n_work, int64_t tiles_per_vec) {
  using C = typename CT<R>::C;
  using V = typename CT<R>::V;
  constexpr int PV = CT<R>::PV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const DPass P = *pass;
  const uint32_t n = 1u << P.k;
  const uint32_t half = n >> 1;
  const uint32_t nt = blockDim.x, tid = threadIdx.x;
  const uint32_t low_mask = (P.low >= 32) ? 0xffffffffu : ((1u << P.low) - 1u);
  const int8_t* __restrict__ hi_bits = pass->tile_bit + P.low;

  for (int64_t w = blockIdx.x; w < n_work; w += gridDim.x) {
    const int64_t r = w / tiles_per_vec;
    const int64_t T = w - r * tiles_per_vec;
    C* vec = state + r * vec_stride;
    const uint64_t vbase = ((uint64_t)T << P.k) | ((uint64_t)r << P.nq);
    int64_t gbase = 0;
    for (int b = 0; b < P.n_rest; ++b) gbase |= ((T >> b) & 1) << pass->rest_bit[b];

    if (P.init_zero) {
      for (uint32_t l = tid; l < n; l += nt) {
        C z;
        z.x = (T == 0 && l == 0) ? R(1) : R(0);
        z.y = R(0);
        s[l] = z;
      }
    } else {
      for (uint32_t u = tid; u < n / PV; u += nt) {
        const uint32_t l = u * PV;
        const int64_t g = gbase | (l & low_mask) | tile_row_offset(l >> P.low, hi_bits);
        *reinterpret_cast<V*>(s + l) = *reinterpret_cast<const V*>(vec + g);
      }
    }
    __syncthreads();

    for (int o = P.op_begin; o < P.op_end; ++o) {
      const DOp op = ops[o];
      if (op.type == OP_DENSE) {
        const R* m = mats + 8 * op.mat;
        const R u0r = m[0], u0i = m[1], u1r = m[2], u1i = m[3];
        const R u2r = m[4], u2i = m[5], u3r = m[6], u3i = m[7];
        const int t = op.t;
        const uint32_t lo = (1u << t) - 1u;
        const bool has_terms = op.term_end > op.term_begin;
        for (uint32_t p = tid; p < half; p += nt) {
          const uint32_t l0 = ((p & ~lo) << 1) | (p & lo);
          const uint32_t l1 = l0 | (1u << t);
          C a0 = s[l0], a1 = s[l1];
          if (has_terms) {
            apply_terms<R>(a0, vbase | l0, terms, op.term_begin, op.term_sign_end, op.term_end, tabs);
            apply_terms<R>(a1, vbase | l1, terms, op.term_begin, op.term_sign_end, op.term_end, tabs);
          }
          C b0, b1;
          b0.x = u0r * a0.x - u0i * a0.y + u1r * a1.x - u1i * a1.y;
          b0.y = u0r * a0.y + u0i * a0.x + u1r * a1.y + u1i * a1.x;
          b1.x = u2r * a0.x - u2i * a0.y + u3r * a1.x - u3i * a1.y;
          b1.y = u2r * a0.y + u2i * a0.x + u3r * a1.y + u3i * a1.x;
          s[l0] = b0;
          s[l1] = b1;
        }
      } else {
        for (uint32_t l = tid; l < n; l += nt) {
          C a = s[l];
          apply_terms<R>(a, vbase | l, terms, op.term_begin, op.term_sign_end, op.term_end, tabs);
          s[l] = a;
        }
      }
      __syncthreads();
    }

    for (uint32_t u = tid; u < n / PV; u += nt) {
      const uint32_t l = u * PV;
      const int64_t g = gbase | (l & low_mask) | tile_row_offset(l >> P.low, hi_bits);
      *reinterpret_cast<V*>(vec + g) = *reinterpret_cast<const V*>(s + l);
    }
    __syncthreads();
  }
}

namespace {

int threads_for(int k) {
  const int pairs = 1 << std::max(k - 1, 0);
  return std::min(1024, std::max(32, pairs / 4));
}

template <typename R>
cc_status launch_pass_t(const DeviceProgram& dp, int pi, void* state, int64_t n_vec,
                        int64_t vec_stride, cudaStream_t stream) {
  using C = typename CT<R>::C;
  const DPass& P = dp.passes[pi];
  const int64_t tiles_per_vec = int64_t(1) << (P.nq - P.k);
  const int64_t n_work = n_vec * tiles_per_vec;
  if (n_work <= 0) return CC_OK;
  const size_t smem = sizeof(C) << P.k;
  const int nt = threads_for(P.k);
  auto kern = pass_kernel<R>;
  static int attr_done[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_done[dev] = 1;
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, smem);
  occ = std::max(occ, 1);
  const int64_t cap = (int64_t)num_sms() * occ;
  const int64_t grid = std::min(n_work, cap);
  const DPass* dpass = reinterpret_cast<const DPass*>(
      reinterpret_cast<const char*>(dp.passes_dev) + sizeof(DPass) * pi);
  kern<<<(unsigned)grid, nt, smem, stream>>>(
      reinterpret_cast<C*>(state), vec_stride, dpass, dp.ops, dp.terms,
      reinterpret_cast<const R*>(dp.mats), reinterpret_cast<const R*>(dp.tabs), n_work,
      tiles_per_vec);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(CC_ECUDA, std::string("pass kernel launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

}  // namespace

cc_status run_program(const DeviceProgram& dp, int precision, void* state, int64_t n_vec,
                      int64_t vec_stride, void* stream) {
  for (int pi = 0; pi < (int)dp.passes.size(); ++pi) {
    const cc_status st =
        precision == CC_C128
            ? launch_pass_t<double>(dp, pi, state, n_vec, vec_stride, (cudaStream_t)stream)
            : launch_pass_t<float>(dp, pi, state, n_vec, vec_stride, (cudaStream_t)stream);
    if (st != CC_OK) return st;
  }
  return CC_OK;
}

}  // namespace cc
