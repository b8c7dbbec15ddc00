// Double-float arithmetic: a real number as the unevaluated sum h + l of two
// FP32 numbers with |l| <= ulp(h) / 2, about 48 significant bits, computed on
// the FP32 pipes.  GB300's FP64 pipe runs at 1/64 of the FP32 rate, so the
// complex128 gate passes carry their amplitudes in this form.
//
// The error-free transformations are the published ones: the sum of two
// floats as a float plus its exact rounding error (Knuth's TwoSum; Dekker's
// Fast2Sum when |a| >= |b|), and the product as a float plus its exact error
// from one fused multiply-add (Dekker's TwoProduct with an FMA).  Addition and
// multiplication follow Dekker (1971) and the double-double library of
// Hida, Li and Bailey (2001): the result is renormalised so that the pair
// again satisfies |l| <= ulp(h) / 2.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

namespace cc {

struct dfl {
  float h, l;
  dfl() = default;
  __host__ __device__ constexpr dfl(float hh, float ll) : h(hh), l(ll) {}
  __host__ __device__ constexpr dfl(int v) : h((float)v), l(0.0f) {}
};

// a + b = s + e exactly (any magnitudes)
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// a + b = s + e exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

// a b = p + e exactly
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float e;
  const float s = two_sum(a.h, b.h, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  float l;
  const float h = fast_two_sum(s, e, l);
  return dfl(h, l);
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.h, -a.l); }

__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  float e;
  const float p = two_prod(a.h, b.h, e);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  float l;
  const float h = fast_two_sum(p, e, l);
  return dfl(h, l);
}

// a b + c with one rounding step fewer than a * b followed by + c: the
// product's high part enters the TwoSum with c, its error and the cross terms
// join the low part.
__device__ __forceinline__ dfl dfma(dfl a, dfl b, dfl c) {
  float e;
  const float p = two_prod(a.h, b.h, e);
  float e2;
  const float s = two_sum(c.h, p, e2);
  const float lo = __fadd_rn(e2, __fadd_rn(e, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, c.l))));
  float l;
  const float h = fast_two_sum(s, lo, l);
  return dfl(h, l);
}

// FP64 <-> double-float (conversions on the FP64 pipe; the passes use them
// only where a program's vector enters or leaves complex128 storage)
__device__ __forceinline__ dfl dfl_from_double(double d) {
  const float h = __double2float_rn(d);
  const float l = __double2float_rn(d - (double)h);
  return dfl(h, l);
}

__device__ __forceinline__ double dfl_to_double(dfl a) { return (double)a.h + (double)a.l; }

// -a where the sign bit of m (bit 31) is set
__device__ __forceinline__ dfl dfl_flip(dfl a, uint32_t m) {
  const uint32_t s = m & 0x80000000u;
  return dfl(__uint_as_float(__float_as_uint(a.h) ^ s), __uint_as_float(__float_as_uint(a.l) ^ s));
}

struct alignas(16) cdfl {
  dfl x, y;
};

}  // namespace cc
