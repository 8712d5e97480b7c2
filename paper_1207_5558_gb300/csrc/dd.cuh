// Double-float ("dd") arithmetic on the FP32 pipe for the FP64 path.
//
// A value is the unevaluated sum h + l of two floats (about 48 significant
// bits), built from the error-free transformations of Dekker and Knuth:
// TwoProd (the rounding error of a product, exactly, from one fused
// multiply-add) and TwoSum (the rounding error of a sum, exactly, from six
// additions).  GB300 issues FP32 fused multiply-adds at 64 times the FP64
// rate, so a double-float multiply-add (about 12 FP32 operations) still runs
// about four times faster than one FP64 FMA.  Every operation below uses the
// _rn intrinsics, which the compiler neither contracts nor reassociates.
//
// Range: callers scale their operands by powers of two so that the floats
// stay far from FP32 underflow; the scale is applied again when the result is
// assembled as a double (dd_to_double).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// The double x as h + l (FP64 operations: use on tables and coefficients, not
// per sample).
__device__ __forceinline__ void dd_split(double x, float* h, float* l) {
  const float hh = __double2float_rn(x);
  *h = hh;
  *l = __double2float_rn(x - (double)hh);
}

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ float two_sum(float a, float b, float* e) {
  const float s = __fadd_rn(a, b);
  const float v = __fadd_rn(s, -a);
  *e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -v)), __fadd_rn(b, -v));
  return s;
}

// Two floats in one 64-bit register pair for the packed FP32x2 instructions
// of sm_100 and later: one instruction computes both halves, each rounded
// exactly as the scalar instruction would (IEEE round to nearest, never
// contracted), so code on pairs gives the bits of the scalar code at half the
// issue slots.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk2(float a, float b) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(f2p v, float* a, float* b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(*a), "=f"(*b) : "l"(v));
}
__device__ __forceinline__ f2p add2(f2p a, f2p b) {
  f2p r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
  f2p r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
  f2p r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
  f2p r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// two_sum on both halves
__device__ __forceinline__ f2p two_sum2(f2p a, f2p b, f2p* e) {
  const f2p s = add2(a, b);
  const f2p v = sub2(s, a);
  *e = add2(sub2(a, sub2(s, v)), sub2(b, v));
  return s;
}

// Accumulator of a sum of products: (sh, sl) with sh the running float sum
// and sl the collected rounding errors and low-order product terms; the pair
// is renormalised only when read (dd_acc_get).
struct dd_acc {
  float sh, sl;
};
__device__ __forceinline__ dd_acc dd_acc_zero() { return {0.f, 0.f}; }
__device__ __forceinline__ dd_acc dd_acc_of(float h, float l) { return {h, l}; }

// acc += (ah + al) (bh + bl), the al*bl term dropped (below 2^-48 relative).
__device__ __forceinline__ void dd_mac(dd_acc& acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);          // TwoProd: p + e = ah * bh exactly
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float t;
  acc.sh = two_sum(acc.sh, p, &t);
  acc.sl = __fadd_rn(acc.sl, __fadd_rn(t, e));
}

// acc += (bh + bl) (no product).
__device__ __forceinline__ void dd_add(dd_acc& acc, float bh, float bl) {
  float t;
  acc.sh = two_sum(acc.sh, bh, &t);
  acc.sl = __fadd_rn(acc.sl, __fadd_rn(t, bl));
}

// The accumulator as a normalised pair (|l| <= ulp(h) / 2 when |sl| < |sh|).
__device__ __forceinline__ void dd_acc_get(const dd_acc& a, float* h, float* l) {
  const float s = __fadd_rn(a.sh, a.sl);
  *h = s;
  *l = __fadd_rn(a.sl, -__fadd_rn(s, -a.sh));       // sl - (s - sh)
}

// (h + l) * 2^sc as a double, assembled with integer operations (no FP64
// instruction on the common path).  Requires |l| <= ulp(h) (dd_acc_get).
// The 53-bit significand is M = m_h 2^29 + round(l / 2^(e_h - 52)), shifted
// once if l moved it out of [2^52, 2^53).  Zero, FP32-subnormal h, h below
// 2^-74 and results outside the double's normal range take the FP64 route.
// The rare cases of dd_to_double in FP64 arithmetic, kept out of line so
// the compiler does not evaluate them speculatively beside the common path.
static __device__ __noinline__ double dd_to_double_slow(float h, float l, int sc) {
  return ldexp((double)h + (double)l, sc);
}

__device__ __forceinline__ double dd_to_double(float h, float l, int sc) {
  const uint32_t bh = __float_as_uint(h);
  const int eh = (int)((bh >> 23) & 0xffu);          // biased exponent of h
  const int e = eh - 127 + sc;                        // unbiased exponent of the result
  if (eh < 53 || eh == 255 || e < -1000 || e > 1000) {
    // rare: h = 0 (then l = 0), tiny h, or an extreme scale
    return dd_to_double_slow(h, l, sc);
  }
  const int64_t m = (int64_t)((bh & 0x7fffffu) | 0x800000u) << 29;
  // l in units of 2^(eh - 127 - 52): an exact power-of-two scaling (|l| <= 2^(eh - 127 - 23)
  // keeps the product below 2^29), then one rounding to an integer
  const float ls = __fmul_rn(l, __uint_as_float((uint32_t)(306 - eh) << 23));
  const int64_t off = (int64_t)__float2int_rn(ls);
  int64_t M = (bh >> 31) ? off - m : m + off;       // signed significand of h + l
  const uint64_t sgn = M < 0 ? 1ull : 0ull;
  uint64_t mag = (uint64_t)(M < 0 ? -M : M);
  int E = e;
  if (mag >= (1ull << 53)) {                          // carried past 2^53: halve, rounding to nearest even
    const uint64_t half = mag >> 1, lost = mag & 1ull;
    mag = half + (lost & half & 1ull);
    E += 1;
    if (mag >= (1ull << 53)) { mag >>= 1; E += 1; }
  } else if (mag < (1ull << 52)) {                    // borrowed below 2^52 (h a power of two)
    mag <<= 1;
    E -= 1;
  }
  const uint64_t bits = (sgn << 63) | ((uint64_t)(E + 1023) << 52) | (mag & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}
