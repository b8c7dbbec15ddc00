// Gate passes over state vectors (subcircuit simulation, Algorithm 2, and the
// uncut simulation T_orig).
//
// One CTA owns one tile of 2^k amplitudes at a time.  It loads the tile into
// shared memory with 16-byte vector loads (the lowest tile bits are
// contiguous vector bits, so every load is part of a >= 128-byte run) -- or,
// in a program's first pass, starts from |0...0> and reads nothing -- then
// runs the pass's stages and stores the tile back in place.
//
// Stage: thread tau holds the 2^RB amplitudes whose tile index has its RB
// register bits free and its other bits equal to tau's bits (deposited in
// increasing order), so the 32 lanes of a warp cover low tile bits.  Each
// fused op multiplies every held amplitude by its diagonal factors and then
// applies a 2x2 matrix to one register bit, entirely in registers.  Between
// stages the tile goes through shared memory, whose layout XORs the low four
// index bits with higher ones to spread a warp's accesses over the banks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <cstring>

#include "dfloat.cuh"
#include "internal.h"

namespace cc {

// Amplitude types of the three gate-pass arithmetics: C is one amplitude in
// registers and shared memory, V the 16-byte vector moved to and from HBM,
// PV the amplitudes per vector.
template <typename R>
struct CT;
template <>
struct CT<float> {
  using C = float2;
  using V = float4;
  static constexpr int PV = 2;
};
template <>
struct CT<double> {
  using C = double2;
  using V = double2;
  static constexpr int PV = 1;
};
template <>
struct CT<dfl> {
  using C = cdfl;
  using V = float4;  // (re.h, re.l, im.h, im.l)
  static constexpr int PV = 1;
};

template <typename R>
constexpr bool is_f32() { return std::is_same<R, float>::value; }
template <typename R>
constexpr bool is_dfl() { return std::is_same<R, dfl>::value; }

// y + t x in the pass's arithmetic (FP32 and FP64 contract it to one FMA)
__device__ __forceinline__ float mad(float t, float x, float y) { return __fmaf_rn(t, x, y); }
__device__ __forceinline__ double mad(double t, double x, double y) { return __fma_rn(t, x, y); }
__device__ __forceinline__ dfl mad(dfl t, dfl x, dfl y) { return dfma(t, x, y); }

// Read-only load of program data: through the non-coherent global path, or
// (PM, the parameter-space launch) a plain load, which the compiler serves
// from the constant bank.
template <bool PM, typename T>
__device__ __forceinline__ T ldro(const T* p) {
  if constexpr (PM)
    return *p;
  else
    return __ldg(p);
}

namespace {

__device__ __forceinline__ uint32_t swz(uint32_t l) {
  return l ^ (((l >> 4) ^ (l >> 8) ^ (l >> 12)) & 15u);
}

// Vector offset of tile row h (the tile bits above the contiguous low run).
__device__ __forceinline__ int64_t tile_row_offset(uint32_t h, const int8_t* __restrict__ hi_bits) {
  int64_t g = 0;
  for (int t = 0; h; ++t, h >>= 1)
    if (h & 1u) g |= int64_t(1) << hi_bits[t];
  return g;
}

template <int N>
constexpr int ilog2() {
  if constexpr (N <= 1) return 0;
  else return 1 + ilog2<N / 2>();
}

// Where a thread's load/store vectors sit.  Thread tau (< n_active) moves the
// vectors l = (tau + it * n_active) * PV, it < NV.  The map from a tile index
// to its vector offset, (l & low_mask) | tile_row_offset(l >> low), and the
// shared-memory swizzle are both GF(2)-linear in l, and tau's bits and it's
// bits are disjoint, so each address is the thread's part XOR the
// iteration's part, the latter combined from one term per bit of it.
template <int NVB>
struct TileMap {
  int64_t g_t;            // vector offset of l = tau * PV
  uint32_t p_t;           // swizzled position of l = tau * PV
  int64_t g_b[NVB > 0 ? NVB : 1];   // offset of l = 2^b * n_active * PV
  uint32_t p_b[NVB > 0 ? NVB : 1];  // swizzled position of the same
};

__device__ __forceinline__ int64_t tile_addr(uint32_t l, uint32_t low_mask, int low,
                                             const int8_t* __restrict__ hi_bits) {
  return (int64_t)(l & low_mask) | tile_row_offset(l >> low, hi_bits);
}

template <int PV, int NVB>
__device__ __forceinline__ TileMap<NVB> make_tile_map(const DPass& P, const DPass* __restrict__ pass,
                                                      uint32_t n_active) {
  TileMap<NVB> m;
  const uint32_t low_mask = (P.low >= 32) ? 0xffffffffu : ((1u << P.low) - 1u);
  const int8_t* __restrict__ hi_bits = pass->tile_bit + P.low;
  const uint32_t lt = threadIdx.x * PV;
  m.g_t = tile_addr(lt, low_mask, P.low, hi_bits);
  m.p_t = swz(lt);
#pragma unroll
  for (int b = 0; b < NVB; ++b) {
    const uint32_t lb = (n_active * PV) << b;
    m.g_b[b] = tile_addr(lb, low_mask, P.low, hi_bits);
    m.p_b[b] = swz(lb);
  }
  return m;
}

// The per-iteration parts g_b, p_b are the same for every thread of the
// CTA: the kernels keep them in shared memory (written by thread 0 before a
// barrier) and read them at each tile's load and store.  The volatile reads
// keep the compiler from holding all of them in registers across the stage
// loop, where the register-bound pass needs every register.
__device__ __forceinline__ int64_t shared_map_g(const int64_t* s_tg, int b) {
  return *(volatile const int64_t*)(s_tg + b);
}
__device__ __forceinline__ uint32_t shared_map_p(const uint32_t* s_tp, int b) {
  return *(volatile const uint32_t*)(s_tp + b);
}
template <int NVB>
__device__ __forceinline__ void publish_tile_map(const TileMap<NVB>& tm, int64_t* s_tg,
                                                 uint32_t* s_tp) {
  static_assert(NVB <= 4, "at most four per-iteration terms");
  if (threadIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < NVB; ++b) {
      s_tg[b] = tm.g_b[b];
      s_tp[b] = tm.p_b[b];
    }
  }
}

template <typename R>
__device__ __forceinline__ void cmul(R& xr, R& xi, R yr, R yi) {
  const R t = xr * yr - xi * yi;
  xi = xr * yi + xi * yr;
  xr = t;
}
__device__ __forceinline__ void cmul(dfl& xr, dfl& xi, dfl yr, dfl yi) {
  const dfl t = dfma(xr, yr, -(xi * yi));
  xi = dfma(xr, yi, xi * yr);
  xr = t;
}

// Slots j < 2^RB whose register bit i is set (i < 5).
__host__ __device__ constexpr uint32_t slot_pattern(int i) {
  return i == 0 ? 0xAAAAAAAAu : i == 1 ? 0xCCCCCCCCu : i == 2 ? 0xF0F0F0F0u
       : i == 3 ? 0xFF00FF00u : 0xFFFF0000u;
}

// Per-stage view of where the register bits sit in the tile index.
template <int RB>
struct StageRegs {
  int rb[RB];          // tile bit of register bit i (ascending)
  uint32_t rmask;      // tile bits held in registers
  uint32_t cons;       // bit i: register bits i and i+1 are adjacent tile bits
  __device__ __forceinline__ int index_of(int p) const {  // -1 if tile bit p is not a register bit
    return (p < 32 && ((rmask >> p) & 1u)) ? __popc(rmask & ((1u << p) - 1u)) : -1;
  }
};

// Apply a phase block: slot j gets Phi T[j], with T the block's 32
// precomputed products (the host folds the block's constant K into them) and
// Phi the product of the ratios of the TERM_PFIX terms whose bit is set in
// the thread's fixed index bits c (1 when there are none): one complex
// product per amplitude however many phases the block holds.  Phi is the same
// for all of the thread's amplitudes, so it commutes with every op of the
// stage: it multiplies into the thread's deferred factor F (hasF set), which
// the stage applies once before its store.  The complex128 kernels skip slot
// 0 where T[0] = 1.
template <typename R, int RB, bool PM>
__device__ __forceinline__ void apply_phase(typename CT<R>::C (&a)[1 << RB], const DOp& op,
                                            uint64_t c, const DTerm* __restrict__ terms,
                                            const R* __restrict__ tabs, typename CT<R>::C& F,
                                            bool& hasF) {
  constexpr int N = 1 << RB;
  const R* tb = tabs + 8 * op.blk_tab;  // the block term's tab, copied into the op
  const bool skip0 = !is_f32<R>() && !(op.blk_p0 & 1u);
  R pr = R(1), pi = R(0);
  const bool fixed = op.term_phase_end() > op.term_sign_end() + 1;
  if (fixed) {
    for (int t = op.term_sign_end() + 1; t < op.term_phase_end(); ++t) {
      const DTerm d = terms[t];
      if ((c >> d.p0) & 1u) {
        const R* f = tabs + 8 * d.tab;
        cmul(pr, pi, f[0], f[1]);
      }
    }
    cmul(F.x, F.y, pr, pi);
    hasF = true;
  }
  if constexpr (is_f32<R>()) {
    const float4* t4 = reinterpret_cast<const float4*>(tb);
#pragma unroll
    for (int j2 = 0; j2 < N / 2; ++j2) {
      const float4 f = ldro<PM>(t4 + j2);
      cmul(a[2 * j2].x, a[2 * j2].y, f.x, f.y);
      cmul(a[2 * j2 + 1].x, a[2 * j2 + 1].y, f.z, f.w);
    }
  } else if constexpr (is_dfl<R>()) {
    const float4* t4 = reinterpret_cast<const float4*>(tb);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (j == 0 && skip0) continue;
      const float4 f = ldro<PM>(t4 + j);
      cmul(a[j].x, a[j].y, dfl(f.x, f.y), dfl(f.z, f.w));
    }
  } else {
    const double2* t2 = reinterpret_cast<const double2*>(tb);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (j == 0 && skip0) continue;
      const double2 f = ldro<PM>(t2 + j);
      cmul(a[j].x, a[j].y, f.x, f.y);
    }
  }
}

// x with its sign bit flipped where bit 31 of m is set: x ^ (m & 0x80000000).
__device__ __forceinline__ uint32_t xor_sign(uint32_t x, uint32_t m) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x78;" : "=r"(d) : "r"(x), "r"(m), "r"(0x80000000u));
  return d;
}

// Multiply the thread's 2^RB amplitudes by an op's diagonal factors.  With
// v = c | r (c: the thread's fixed index bits, r: register bits, disjoint),
// the CZ-type sign (-1)^{popcount(v & (v>>1) & adj)} splits into a constant,
// a part linear in r and a part quadratic in adjacent register bits, which
// gives the sign of every slot at once as a 32-bit mask over slots.
template <typename R, int RB, bool PM>
__device__ __forceinline__ void apply_diag(typename CT<R>::C (&a)[1 << RB], const DOp& op,
                                           uint64_t c, const StageRegs<RB>& sr,
                                           const DTerm* __restrict__ terms,
                                           const R* __restrict__ tabs, typename CT<R>::C& F,
                                           bool& hasF) {
  constexpr int N = 1 << RB;
  constexpr uint32_t ALL = N >= 32 ? 0xFFFFFFFFu : ((1u << N) - 1u);
  uint32_t smask = 0;
  if (op.sign_adj) {
    const uint64_t adj = op.sign_adj;
    const uint64_t lin = ((c & adj) << 1) ^ ((c >> 1) & adj);
    if (__popcll(c & (c >> 1) & adj) & 1) smask = ALL;
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      if ((lin >> sr.rb[i]) & 1u) smask ^= slot_pattern(i);
      if (i + 1 < RB && ((sr.cons >> i) & 1u) && ((adj >> sr.rb[i]) & 1u))
        smask ^= slot_pattern(i) & slot_pattern(i + 1 < RB ? i + 1 : i);
    }
  }
  for (int t = op.term_begin; t < op.term_sign_end(); ++t) {
    const DTerm d = terms[t];
    const int i0 = sr.index_of(d.p0), i1 = sr.index_of(d.p1);
    const uint32_t c0 = (uint32_t)(c >> d.p0) & 1u, c1 = (uint32_t)(c >> d.p1) & 1u;
    uint32_t pa = 0, pb = 0;
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      if (i == i0) pa = slot_pattern(i);
      if (i == i1) pb = slot_pattern(i);
    }
    if (i0 < 0) pa = c0 ? ALL : 0u;
    if (i1 < 0) pb = c1 ? ALL : 0u;
    smask ^= pa & pb;
  }
  smask &= ALL;
  if (smask) {
    // slot j's sign is bit j of smask moved to bit 31: one shift per slot and
    // one three-input logic op (x ^ (m & 0x80000000)) per float
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const uint32_t m = smask << (31 - j);
      if constexpr (is_f32<R>()) {
        a[j].x = __uint_as_float(xor_sign(__float_as_uint(a[j].x), m));
        a[j].y = __uint_as_float(xor_sign(__float_as_uint(a[j].y), m));
      } else if constexpr (is_dfl<R>()) {
        a[j].x = dfl(__uint_as_float(xor_sign(__float_as_uint(a[j].x.h), m)),
                     __uint_as_float(xor_sign(__float_as_uint(a[j].x.l), m)));
        a[j].y = dfl(__uint_as_float(xor_sign(__float_as_uint(a[j].y.h), m)),
                     __uint_as_float(xor_sign(__float_as_uint(a[j].y.l), m)));
      } else {
        const long long hx = __double_as_longlong(a[j].x);
        const long long hy = __double_as_longlong(a[j].y);
        a[j].x = __hiloint2double((int)xor_sign((uint32_t)(hx >> 32), m), (int)(uint32_t)hx);
        a[j].y = __hiloint2double((int)xor_sign((uint32_t)(hy >> 32), m), (int)(uint32_t)hy);
      }
    }
  }
  if (op.term_phase_end() > op.term_sign_end())
    apply_phase<R, RB, PM>(a, op, c, terms, tabs, F, hasF);
  for (int t = op.term_phase_end(); t < op.term_end(); ++t) {
    const DTerm d = terms[t];
    const int i0 = sr.index_of(d.p0), i1 = sr.index_of(d.p1);
    const int c0 = (int)((c >> d.p0) & 1u), c1 = (int)((c >> d.p1) & 1u);
    const R* tb = tabs + 8 * d.tab;
    const R f0r = tb[0], f0i = tb[1], f1r = tb[2], f1i = tb[3];
    const R f2r = tb[4], f2i = tb[5], f3r = tb[6], f3i = tb[7];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int x0 = i0 >= 0 ? (j >> i0) & 1 : c0;
      const int x1 = i1 >= 0 ? (j >> i1) & 1 : c1;
      const int idx = x0 | (x1 << 1);
      const R fr = idx == 0 ? f0r : idx == 1 ? f1r : idx == 2 ? f2r : f3r;
      const R fi = idx == 0 ? f0i : idx == 1 ? f1i : idx == 2 ? f2i : f3i;
      cmul(a[j].x, a[j].y, fr, fi);
    }
  }
}

// Tile index of register slot j: lo[j & (2^L - 1)] | hi[j >> L], where the
// low L = min(RB, 2) register bits index `lo` (which also carries the
// thread's own bits) and the others index `hi`.
template <int RB>
struct SlotIndex {
  static constexpr int L = RB < 2 ? RB : 2;
  static constexpr int H = RB - L;
  uint32_t lo[1 << L];
  uint32_t hi[1 << H];
  __device__ __forceinline__ uint32_t operator()(int j) const {
    return lo[j & ((1 << L) - 1)] | hi[j >> L];
  }
};

// An op's 2x2 matrix (row-major, interleaved re/im), loaded with 16-byte loads.
template <typename R>
struct Mat {
  R v[8];
};
template <typename R, bool PM>
__device__ __forceinline__ Mat<R> load_mat(const R* __restrict__ p) {
  Mat<R> m;
  if constexpr (is_f32<R>()) {
    const float4 x = ldro<PM>(reinterpret_cast<const float4*>(p));
    const float4 y = ldro<PM>(reinterpret_cast<const float4*>(p) + 1);
    m.v[0] = x.x; m.v[1] = x.y; m.v[2] = x.z; m.v[3] = x.w;
    m.v[4] = y.x; m.v[5] = y.y; m.v[6] = y.z; m.v[7] = y.w;
  } else if constexpr (is_dfl<R>()) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 x = ldro<PM>(reinterpret_cast<const float4*>(p) + i);
      m.v[2 * i] = dfl(x.x, x.y);
      m.v[2 * i + 1] = dfl(x.z, x.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 x = ldro<PM>(reinterpret_cast<const double2*>(p) + i);
      m.v[2 * i] = x.x;
      m.v[2 * i + 1] = x.y;
    }
  }
  return m;
}

// 2x2 matrix on register bit RHO of every held pair.
template <typename R, int RB, int RHO>
__device__ __forceinline__ void dense_mat(typename CT<R>::C (&a)[1 << RB], const Mat<R>& mm) {
  const R* m = mm.v;
  using C = typename CT<R>::C;
  constexpr int N = 1 << RB;
  const R u0r = m[0], u0i = m[1], u1r = m[2], u1i = m[3];
  const R u2r = m[4], u2i = m[5], u3r = m[6], u3i = m[7];
#pragma unroll
  for (int p = 0; p < N / 2; ++p) {
    constexpr int lo = (1 << RHO) - 1;
    const int j0 = ((p & ~lo) << 1) | (p & lo);
    const int j1 = j0 | (1 << RHO);
    const C a0 = a[j0], a1 = a[j1];
    C b0, b1;
    if constexpr (is_dfl<R>()) {
      b0.x = mad(u0r, a0.x, mad(-u0i, a0.y, mad(u1r, a1.x, -(u1i * a1.y))));
      b0.y = mad(u0r, a0.y, mad(u0i, a0.x, mad(u1r, a1.y, u1i * a1.x)));
      b1.x = mad(u2r, a0.x, mad(-u2i, a0.y, mad(u3r, a1.x, -(u3i * a1.y))));
      b1.y = mad(u2r, a0.y, mad(u2i, a0.x, mad(u3r, a1.y, u3i * a1.x)));
    } else {
      b0.x = u0r * a0.x - u0i * a0.y + u1r * a1.x - u1i * a1.y;
      b0.y = u0r * a0.y + u0i * a0.x + u1r * a1.y + u1i * a1.x;
      b1.x = u2r * a0.x - u2i * a0.y + u3r * a1.x - u3i * a1.y;
      b1.y = u2r * a0.y + u2i * a0.x + u3r * a1.y + u3i * a1.x;
    }
    a[j0] = b0;
    a[j1] = b1;
  }
}

// x + (-0), exact for every x (signed zeros, infinities and NaNs included).
// Both outputs of a rotation need both inputs, so one of them is computed
// into a fresh register and copied back into its slot's register; written
// as this add, the copy issues on the FMA pipe instead of the ALU pipe, which
// the pass's integer and logic work keeps the busier of the two.
__device__ __forceinline__ float fma_pipe_copy(float x) {
  float r;
  asm("add.rn.f32 %0, %1, 0f80000000;" : "=f"(r) : "f"(x));
  return r;
}

// Real rotation in tangent form on register bit RHO of every held pair:
// (a, b) <- (a - t b, b + t a), or with COT (a, b) <- (t a - b, a + t b);
// two multiply-adds per amplitude.
template <typename R, int RB, int RHO, bool COT>
__device__ __forceinline__ void rot_mat(typename CT<R>::C (&a)[1 << RB], R t) {
  using C = typename CT<R>::C;
  constexpr int N = 1 << RB;
#pragma unroll
  for (int p = 0; p < N / 2; ++p) {
    constexpr int lo = (1 << RHO) - 1;
    const int j0 = ((p & ~lo) << 1) | (p & lo);
    const int j1 = j0 | (1 << RHO);
    const C a0 = a[j0], a1 = a[j1];
    C b0, b1;
    if constexpr (is_dfl<R>()) {
      if (COT) {
        b0.x = mad(t, a0.x, -a1.x);
        b0.y = mad(t, a0.y, -a1.y);
        b1.x = mad(t, a1.x, a0.x);
        b1.y = mad(t, a1.y, a0.y);
      } else {
        b0.x = mad(-t, a1.x, a0.x);
        b0.y = mad(-t, a1.y, a0.y);
        b1.x = mad(t, a0.x, a1.x);
        b1.y = mad(t, a0.y, a1.y);
      }
    } else if (COT) {
      b0.x = t * a0.x - a1.x;
      b0.y = t * a0.y - a1.y;
      b1.x = t * a1.x + a0.x;
      b1.y = t * a1.y + a0.y;
    } else {
      b0.x = a0.x - t * a1.x;
      b0.y = a0.y - t * a1.y;
      b1.x = a1.x + t * a0.x;
      b1.y = a1.y + t * a0.y;
    }
    if constexpr (is_f32<R>()) {
      b0.x = fma_pipe_copy(b0.x);
      b0.y = fma_pipe_copy(b0.y);
    }
    a[j0] = b0;
    a[j1] = b1;
  }
}

// The rotations of an OP_ROTS op: register bit RHO.. in turn, each in its
// tangent (or cotangent) form with its own tangent.
template <typename R, int RB, int RHO>
__device__ __forceinline__ void rot_run(typename CT<R>::C (&a)[1 << RB], uint32_t bits,
                                        uint32_t cot, const Mat<R>& m) {
  if constexpr (RHO < RB) {
    if ((bits >> RHO) & 1u) {
      if ((cot >> RHO) & 1u)
        rot_mat<R, RB, RHO, true>(a, m.v[RHO]);
      else
        rot_mat<R, RB, RHO, false>(a, m.v[RHO]);
    }
    rot_run<R, RB, RHO + 1>(a, bits, cot, m);
  }
}

template <typename V>
__device__ __forceinline__ V swap_pair(V v) {  // (a, b) -> (b, a) for a float4 of two complex64
  float4 f = reinterpret_cast<float4&>(v);
  f = make_float4(f.z, f.w, f.x, f.y);
  return reinterpret_cast<V&>(f);
}

// Load, transform and store tile T of one pass.  n_active threads (a power
// of two, 2^(k - RB)) take part; each moves 2^RB amplitudes in NV 16-byte
// vectors per phase.  CG loads through L2 only, for vectors that other CTAs
// of the same launch wrote.
template <typename R, int RB, bool CG, bool PM = false>
__device__ __forceinline__ void run_tile(typename CT<R>::C* __restrict__ vec, const DPass& P,
                                         const DStage* __restrict__ stages,
                                         const DOp* __restrict__ ops,
                                         const DTerm* __restrict__ terms,
                                         const R* __restrict__ mats, const R* __restrict__ tabs,
                                         const int8_t* __restrict__ rest_bit, int64_t T,
                                         typename CT<R>::C* s, uint32_t n_active,
                                         const TileMap<ilog2<(1 << RB) / CT<R>::PV>()>& tm,
                                         const int64_t* s_tg, const uint32_t* s_tp) {
  using C = typename CT<R>::C;
  using V = typename CT<R>::V;
  constexpr int PV = CT<R>::PV;
  constexpr int N = 1 << RB;
  constexpr int NV = N / PV;
  constexpr int NVB = ilog2<NV>();
  const uint32_t n = 1u << P.k;
  const uint32_t tid = threadIdx.x;
  const uint32_t kmask = n - 1u;
  const bool active = tid < n_active;

  const uint64_t vbase = (uint64_t)T << P.k;
  int64_t gbase = 0;
  for (int b = 0; b < P.n_rest; ++b) gbase |= ((T >> b) & 1) << rest_bit[b];
  const bool rest_zero = (((uint64_t)T) & P.zero_rest) == 0;
  const int64_t g0 = gbase | tm.g_t;

  if (!P.init_zero) {
    if (active) {
      V val[NV];
#pragma unroll
      for (int it = 0; it < NV; ++it) {
        int64_t g = g0;
#pragma unroll
        for (int b = 0; b < NVB; ++b)
          if ((it >> b) & 1) g ^= shared_map_g(s_tg, b);
        val[it] = CG ? __ldcg(reinterpret_cast<const V*>(vec + g)) : *reinterpret_cast<const V*>(vec + g);
      }
#pragma unroll
      for (int it = 0; it < NV; ++it) {
        uint32_t pl = tm.p_t;
#pragma unroll
        for (int b = 0; b < NVB; ++b)
          if ((it >> b) & 1) pl ^= shared_map_p(s_tp, b);
        V v = val[it];
        if (PV == 2 && (pl & 1u)) v = swap_pair(v);  // the swizzle swapped the pair
        *reinterpret_cast<V*>(s + (pl & ~uint32_t(PV - 1))) = v;
      }
    }
    __syncthreads();
  }

  for (int si = P.stage_begin; si < P.stage_end; ++si) {
    if (active) {
      const DStage st = stages[si];
      StageRegs<RB> sr;
      sr.rmask = 0;
      sr.cons = 0;
      SlotIndex<RB> dep;
#pragma unroll
      for (int j = 0; j < (1 << SlotIndex<RB>::L); ++j) dep.lo[j] = 0;
#pragma unroll
      for (int j = 0; j < (1 << SlotIndex<RB>::H); ++j) dep.hi[j] = 0;
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        sr.rb[i] = st.rb[i];
        const uint32_t b = 1u << st.rb[i];
        sr.rmask |= b;
        if (i + 1 < RB && st.rb[i + 1 < RB ? i + 1 : i] == st.rb[i] + 1) sr.cons |= 1u << i;
        if (i < SlotIndex<RB>::L) {
#pragma unroll
          for (int j = 0; j < (1 << SlotIndex<RB>::L); ++j)
            if (j & (1 << i)) dep.lo[j] |= b;
        } else {
#pragma unroll
          for (int j = 0; j < (1 << SlotIndex<RB>::H); ++j)
            if (j & (1 << (i - SlotIndex<RB>::L))) dep.hi[j] |= b;
        }
      }
      uint32_t base = 0;
      {
        uint32_t free_bits = kmask & ~sr.rmask, t = tid;
        while (free_bits) {
          const uint32_t p = __ffs(free_bits) - 1;
          free_bits &= free_bits - 1;
          base |= (t & 1u) << p;
          t >>= 1;
        }
      }
#pragma unroll
      for (int j = 0; j < (1 << SlotIndex<RB>::L); ++j) dep.lo[j] |= base;
      const uint64_t cfix = vbase | base;  // the thread's fixed index bits in this stage
      // swz is GF(2)-linear and dep.lo, dep.hi have disjoint bits:
      // swz(dep(j)) = swz(dep.lo[.]) ^ swz(dep.hi[.])
      SlotIndex<RB> sp;
#pragma unroll
      for (int j = 0; j < (1 << SlotIndex<RB>::L); ++j) sp.lo[j] = swz(dep.lo[j]);
#pragma unroll
      for (int j = 0; j < (1 << SlotIndex<RB>::H); ++j) sp.hi[j] = swz(dep.hi[j]);
#define CC_SLOT_POS(j) (sp.lo[(j) & ((1 << SlotIndex<RB>::L) - 1)] ^ sp.hi[(j) >> SlotIndex<RB>::L])

      C a[N];
      if (P.init_zero && si == P.stage_begin) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          a[j].x = (rest_zero && (dep(j) & P.zero_tile) == 0) ? R(1) : R(0);
          a[j].y = R(0);
        }
      } else {
#pragma unroll
        for (int j = 0; j < N; ++j) a[j] = s[CC_SLOT_POS(j)];
      }

      // op o's matrix sits at mats + 8 o (the image stores one per op), so
      // the descriptor and the matrix load independently.  F: the deferred
      // per-thread phase factor of the stage's TERM_PFIX terms.
      C F;
      F.x = R(1);
      F.y = R(0);
      bool hasF = false;
      for (int o = st.op_begin; o < st.op_end; ++o) {
        const DOp op = ops[o];
        const Mat<R> m = load_mat<R, PM>(mats + 8 * o);
        if (op.sign_adj != 0 || op.term_end() > op.term_begin)
          apply_diag<R, RB, PM>(a, op, cfix, sr, terms, tabs, F, hasF);
#define CC_OP_SWITCH(CALL)                                     \
  switch (op.t) {                                              \
    case 0: CALL(0); break;                                    \
    case 1: if (RB > 1) CALL((RB > 1 ? 1 : 0)); break;         \
    case 2: if (RB > 2) CALL((RB > 2 ? 2 : 0)); break;         \
    case 3: if (RB > 3) CALL((RB > 3 ? 3 : 0)); break;         \
    default: if (RB > 4) CALL((RB > 4 ? 4 : 0)); break;        \
  }
#define CC_DENSE(RHO) dense_mat<R, RB, RHO>(a, m)
#define CC_ROT(RHO) rot_mat<R, RB, RHO, false>(a, m.v[0])
#define CC_ROTC(RHO) rot_mat<R, RB, RHO, true>(a, m.v[0])
        if (op.type == OP_DENSE) {
          CC_OP_SWITCH(CC_DENSE)
        } else if (op.type == OP_ROT) {
          CC_OP_SWITCH(CC_ROT)
        } else if (op.type == OP_ROTC) {
          CC_OP_SWITCH(CC_ROTC)
        } else if (op.type == OP_ROTS) {
          rot_run<R, RB, 0>(a, (uint32_t)op.t, op.cot, m);
        }
#undef CC_DENSE
#undef CC_ROT
#undef CC_ROTC
#undef CC_OP_SWITCH
      }

      if (hasF) {
#pragma unroll
        for (int j = 0; j < N; ++j) cmul(a[j].x, a[j].y, F.x, F.y);
      }
#pragma unroll
      for (int j = 0; j < N; ++j) s[CC_SLOT_POS(j)] = a[j];
#undef CC_SLOT_POS
    }
    __syncthreads();
  }

  if (active) {
#pragma unroll
    for (int it = 0; it < NV; ++it) {
      int64_t g = g0;
      uint32_t pl = tm.p_t;
#pragma unroll
      for (int b = 0; b < NVB; ++b)
        if ((it >> b) & 1) {
          g ^= shared_map_g(s_tg, b);
          pl ^= shared_map_p(s_tp, b);
        }
      V v = *reinterpret_cast<const V*>(s + (pl & ~uint32_t(PV - 1)));
      if (PV == 2 && (pl & 1u)) v = swap_pair(v);
      if constexpr (is_dfl<R>()) {
        if (P.flags & PASS_LAST) {  // h + l is exact in FP64
          const float4 f = reinterpret_cast<const float4&>(v);
          *reinterpret_cast<double2*>(vec + g) =
              make_double2((double)f.x + (double)f.y, (double)f.z + (double)f.w);
          continue;
        }
      }
      *reinterpret_cast<V*>(vec + g) = v;
    }
  }
  __syncthreads();
}

template <typename R, int RB>
__global__ void __launch_bounds__(512)
    stage_kernel(typename CT<R>::C* __restrict__ vec, const DPass* __restrict__ pass,
                 const DStage* __restrict__ stages, const DOp* __restrict__ ops,
                 const DTerm* __restrict__ terms, const R* __restrict__ mats,
                 const R* __restrict__ tabs, int64_t n_tiles) {
  using C = typename CT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const DPass P = *pass;
  constexpr int NVB = ilog2<(1 << RB) / CT<R>::PV>();
  __shared__ int64_t s_tg[4];
  __shared__ uint32_t s_tp[4];
  const TileMap<NVB> tm = make_tile_map<CT<R>::PV, NVB>(P, pass, blockDim.x);
  publish_tile_map<NVB>(tm, s_tg, s_tp);
  __syncthreads();
  for (int64_t T = blockIdx.x; T < n_tiles; T += gridDim.x)
    run_tile<R, RB, false>(vec, P, stages, ops, terms, mats, tabs, pass->rest_bit, T, s,
                           blockDim.x, tm, s_tg, s_tp);
}

// The same pass with its part of the program as the kernel parameter (a
// PassBlob): ops, matrices and tables are read through the constant bank,
// loads that are the same for every thread of the warp.
template <typename R, int RB>
__global__ void __launch_bounds__(512)
    stage_kernel_p(typename CT<R>::C* __restrict__ vec, const __grid_constant__ PassBlob blob,
                   int64_t n_tiles) {
  using C = typename CT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const PassBlobHeader* h = reinterpret_cast<const PassBlobHeader*>(blob.b);
  const DPass* pass = reinterpret_cast<const DPass*>(blob.b + h->o_pass);
  const DStage* stages = reinterpret_cast<const DStage*>(blob.b + h->o_stages);
  const DOp* ops = reinterpret_cast<const DOp*>(blob.b + h->o_ops);
  const DTerm* terms = reinterpret_cast<const DTerm*>(blob.b + h->o_terms);
  const R* mats = reinterpret_cast<const R*>(blob.b + h->o_mats);
  const R* tabs = reinterpret_cast<const R*>(blob.b + h->o_tabs);
  const DPass P = *pass;
  constexpr int NVB = ilog2<(1 << RB) / CT<R>::PV>();
  __shared__ int64_t s_tg[4];
  __shared__ uint32_t s_tp[4];
  const TileMap<NVB> tm = make_tile_map<CT<R>::PV, NVB>(P, pass, blockDim.x);
  publish_tile_map<NVB>(tm, s_tg, s_tp);
  __syncthreads();
  for (int64_t T = blockIdx.x; T < n_tiles; T += gridDim.x)
    run_tile<R, RB, false, true>(vec, P, stages, ops, terms, mats, tabs, pass->rest_bit, T, s,
                                 blockDim.x, tm, s_tg, s_tp);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A dependency wait gives up after this many polls (each followed by a
// ~128 ns sleep): seconds, far beyond any tile of a valid batch.
constexpr int kBatchWaitPolls = 1 << 25;

// Persistent batched gate passes: every CTA takes queue items (one tile of
// one job) until the queue is empty.  Jobs are ordered by pass number, so a
// job's dependency has all its tiles earlier in the queue, taken by CTAs that
// are already running: the waits always end.
template <typename R>
__global__ void __launch_bounds__(512)
    batch_kernel(typename CT<R>::C* __restrict__ seg_buf, const BJob* __restrict__ jobs,
                 int n_jobs, long long n_items, int* __restrict__ done,
                 unsigned long long* __restrict__ head, int* __restrict__ err,
                 unsigned long long* __restrict__ stamps) {
  using C = typename CT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  __shared__ long long s_item;
  __shared__ int64_t s_tg[4];
  __shared__ uint32_t s_tp[4];
  __shared__ int s_job, s_ok;
  const uint32_t tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const long long it = (long long)atomicAdd(head, 1ull);
      s_item = it;
      if (it == 0 && stamps) stamps[0] = global_timer();
      if (it < n_items) {
        int lo = 0, hi = n_jobs - 1;  // last job with tile_begin <= it
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (jobs[mid].tile_begin <= it) lo = mid; else hi = mid - 1;
        }
        s_job = lo;
        int ok = 1;
        const int d = jobs[lo].dep;
        if (d >= 0) {
          const int need = (int)jobs[d].n_tiles;
          int polls = 0;
          while (ld_acquire(done + d) < need) {
            if (++polls > kBatchWaitPolls) {
              ok = 0;
              atomicExch(err, 1);
              break;
            }
            __nanosleep(128);
          }
          __threadfence();
        }
        s_ok = ok;
      }
    }
    __syncthreads();
    const long long it = s_item;
    if (it >= n_items) break;
    const int j = s_job;
    if (s_ok) {
      const BJob& J = jobs[j];
      const DPass P = *J.pass;
      C* vec = seg_buf + J.vec_off;
      const int64_t T = it - J.tile_begin;
      const uint32_t na = 1u << (P.k - P.rbits);
      const R* mats = reinterpret_cast<const R*>(J.mats);
      const R* tabs = reinterpret_cast<const R*>(J.tabs);
      switch (P.rbits) {
#define CC_BATCH_TILE(RBV)                                                                       \
  {                                                                                              \
    constexpr int NVB = ilog2<(1 << (RBV)) / CT<R>::PV>();                                       \
    const TileMap<NVB> tm = make_tile_map<CT<R>::PV, NVB>(P, J.pass, na);                       \
    publish_tile_map<NVB>(tm, s_tg, s_tp);                                                       \
    __syncthreads();                                                                             \
    run_tile<R, (RBV), true>(vec, P, J.stages, J.ops, J.terms, mats, tabs, J.pass->rest_bit, T, \
                             s, na, tm, s_tg, s_tp);                                             \
  }
        case 1: CC_BATCH_TILE(1) break;
        case 2: CC_BATCH_TILE(2) break;
        case 3: CC_BATCH_TILE(3) break;
        case 4: CC_BATCH_TILE(4) break;
        default:
          CC_BATCH_TILE(is_f32<R>() ? 5 : 4)
          break;
#undef CC_BATCH_TILE
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(done + j, 1);
  }
}

// CUTSIM_PARAM_PASSES=0 launches every uncut pass with its program in global
// memory (the segment launch always reads global memory).
bool param_launch_enabled() {
  const char* e = std::getenv("CUTSIM_PARAM_PASSES");
  return !(e && e[0] == '0');
}

template <typename R, int RB>
cc_status launch_rb(const DeviceProgram& dp, int pi, void* state, cudaStream_t stream) {
  using C = typename CT<R>::C;
  const DPass& P = dp.passes[pi];
  const int64_t n_tiles = int64_t(1) << (P.nq - P.k);
  const size_t smem = sizeof(C) << P.k;
  const int nt = 1 << (P.k - P.rbits);
  auto kern = stage_kernel<R, RB>;
  static int attr_done[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    // the opt-in limit (227 KB per CTA) covers static and dynamic shared memory
    cudaFuncAttributes fa;
    size_t static_smem = 0;
    if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess) static_smem = fa.sharedSizeBytes;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(227 * 1024 - static_smem));
    cudaGetLastError();
    attr_done[dev] = 1;
  }
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, smem);
  occ = std::max(occ, 1);
  const int64_t grid = std::min(n_tiles, (int64_t)num_sms() * occ);
  const bool param = pi < (int)dp.blob_ok.size() && dp.blob_ok[pi] && param_launch_enabled();
  if (param) {
    auto kp = stage_kernel_p<R, RB>;
    static int attr_p[64] = {0};
    if (dev >= 0 && dev < 64 && !attr_p[dev]) {
      cudaFuncAttributes fa;
      size_t static_smem = 0;
      if (cudaFuncGetAttributes(&fa, kp) == cudaSuccess) static_smem = fa.sharedSizeBytes;
      cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(227 * 1024 - static_smem));
      cudaGetLastError();
      attr_p[dev] = 1;
    }
    int occ_p = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, kp, nt, smem);
    occ_p = std::max(occ_p, 1);
    const int64_t grid_p = std::min(n_tiles, (int64_t)num_sms() * occ_p);
    C* vp = reinterpret_cast<C*>(state);
    int64_t ntl = n_tiles;
    void* args[] = {&vp, const_cast<PassBlob*>(&dp.blobs[pi]), &ntl};
    const cudaError_t le = cudaLaunchKernel(reinterpret_cast<const void*>(kp), dim3((unsigned)grid_p),
                                            dim3(nt), args, smem, stream);
    if (le != cudaSuccess)
      return fail(CC_ECUDA, std::string("gate pass launch: ") + cudaGetErrorString(le));
    return CC_OK;
  }
  const DPass* dpass = reinterpret_cast<const DPass*>(
      reinterpret_cast<const char*>(dp.passes_dev) + sizeof(DPass) * pi);
  kern<<<(unsigned)grid, nt, smem, stream>>>(
      reinterpret_cast<C*>(state), dpass, dp.stages, dp.ops, dp.terms,
      reinterpret_cast<const R*>(dp.mats), reinterpret_cast<const R*>(dp.tabs), n_tiles);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(CC_ECUDA, std::string("gate pass launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

template <typename R>
cc_status launch_pass(const DeviceProgram& dp, int pi, void* state, cudaStream_t stream) {
  switch (dp.passes[pi].rbits) {
    case 1: return launch_rb<R, 1>(dp, pi, state, stream);
    case 2: return launch_rb<R, 2>(dp, pi, state, stream);
    case 3: return launch_rb<R, 3>(dp, pi, state, stream);
    case 4: return launch_rb<R, 4>(dp, pi, state, stream);
    case 5:
      return launch_rb<R, (is_f32<R>() ? 5 : 4)>(dp, pi, state, stream);
    default:
      break;
  }
  return fail(CC_EINVAL, "pass has an unsupported register width");
}

}  // namespace

int reg_bits_max(int precision) {
  const int hi = precision == CC_C128 ? 4 : 5;
  if (const char* e = std::getenv("CUTSIM_REG_BITS")) {  // fewer register bits: more, lighter threads
    const int v = std::atoi(e);
    if (v >= 2 && v <= hi) return v;
  }
  return hi;
}

int gate_arith(int precision) {
  if (precision != CC_C128) return GA_F32;
  if (const char* e = std::getenv("CUTSIM_C128_GATES"))
    if (std::strcmp(e, "fp64") == 0) return GA_F64;
  return GA_DFL;
}

namespace {
const void* batch_kernel_for(int arith) {
  return arith == GA_F64   ? (const void*)batch_kernel<double>
         : arith == GA_DFL ? (const void*)batch_kernel<dfl>
                           : (const void*)batch_kernel<float>;
}
}  // namespace

int batch_segments_occupancy(int arith, int block, size_t smem) {
  static int attr_done[64][3] = {{0}};
  int dev = 0;
  cudaGetDevice(&dev);
  const int pi = arith;
  const void* kern = batch_kernel_for(arith);
  if (dev >= 0 && dev < 64 && !attr_done[dev][pi]) {
    // the opt-in limit (227 KB per CTA) covers static and dynamic shared memory
    cudaFuncAttributes fa;
    size_t static_smem = 0;
    if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess) static_smem = fa.sharedSizeBytes;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(227 * 1024 - static_smem));
    cudaGetLastError();
    attr_done[dev][pi] = 1;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess) {
    cudaGetLastError();
    occ = 0;
  }
  return occ;
}

cc_status launch_batch_segments(void* seg_buf, const BJob* jobs, int n_jobs, int64_t n_items,
                                int* done, unsigned long long* head,
                                unsigned long long* stamps, int arith, int block,
                                size_t smem, int grid, void* stream) {
  if (n_items <= 0) return CC_OK;
  int* err = device_error_flag();
  if (!err) return fail(CC_ENOMEM, "device error flag allocation failed");
  batch_segments_occupancy(arith, block, smem);  // sets the shared-memory attribute once
  cudaStream_t s = (cudaStream_t)stream;
  if (arith == GA_F64)
    batch_kernel<double><<<grid, block, smem, s>>>(static_cast<double2*>(seg_buf), jobs, n_jobs,
                                                   n_items, done, head, err, stamps);
  else if (arith == GA_DFL)
    batch_kernel<dfl><<<grid, block, smem, s>>>(static_cast<cdfl*>(seg_buf), jobs, n_jobs,
                                                n_items, done, head, err, stamps);
  else
    batch_kernel<float><<<grid, block, smem, s>>>(static_cast<float2*>(seg_buf), jobs, n_jobs,
                                                  n_items, done, head, err, stamps);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(CC_ECUDA, std::string("batched gate pass launch: ") + cudaGetErrorString(e));
  return CC_OK;
}

cc_status run_program(const DeviceProgram& dp, int arith, void* state, void* stream) {
  for (int pi = 0; pi < (int)dp.passes.size(); ++pi) {
    const cudaStream_t s = (cudaStream_t)stream;
    const cc_status st = arith == GA_F64   ? launch_pass<double>(dp, pi, state, s)
                         : arith == GA_DFL ? launch_pass<dfl>(dp, pi, state, s)
                                           : launch_pass<float>(dp, pi, state, s);
    if (st != CC_OK) return st;
  }
  return CC_OK;
}

}  // namespace cc
