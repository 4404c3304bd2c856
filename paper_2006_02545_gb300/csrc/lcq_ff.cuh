// Two-float ("double-word") arithmetic on the FP32 pipe, and the Helmholtz kernel value in it.
//
// A value is an unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h) / 2, about 48
// significant bits.  The building blocks are the error-free transformations of Knuth
// (TwoSum), Dekker (Fast2Sum) and the FMA product error, combined as in the double-word
// algorithms analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017): a product carries
// a relative error of a few 2^-48, a sum an absolute error of a few 2^-48 (|a| + |b|).
// On this GPU an FP64 instruction occupies its pipe 64 times longer than an FP32 one, so a
// kernel value in about 300 FP32 and integer instructions and five FP64 ones costs far less
// FP64 pipe time than the 39 FP64 instructions of kernel_eval_fold.
// Every operation uses the _rn intrinsics so that nothing is contracted or reassociated.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lcq {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// requires |a| >= |b| (or a = 0)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.h, b.h);
  return ff_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// Two-float value of an FP64 number by its bits: h holds the sign, the exponent and the
// leading 23 fraction bits (truncated), l the remaining 29 bits rounded to 24 (relative
// error of h + l at most 2^-48).  Exponents outside the FP32 normal range give l = 0 and h
// zero or infinite; no FP64 instruction.
__device__ __forceinline__ ff ff_of(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32);
  const unsigned sgn = hw & 0x80000000u;
  const int fe = (int)((hw >> 20) & 0x7ffu) - 1023 + 127;
  if (fe <= 0) return {__uint_as_float(sgn), 0.0f};
  if (fe >= 255) return {__uint_as_float(sgn | 0x7f800000u), 0.0f};
  const float h = __uint_as_float(sgn | ((unsigned)fe << 23) | ((unsigned)(b >> 29) & 0x7fffffu));
  const unsigned R = (unsigned)b & 0x1fffffffu;  // R 2^(e - 52)
  if (R == 0u) return {h, 0.0f};
  const int lz = __clz(R) - 3;                   // R << lz has its leading one at bit 28
  const int le = fe - 24 - lz;                   // FP32 exponent field of that leading one
  if (le <= 0) return {h, 0.0f};
  const unsigned m = R << lz;
  // exponent, 23 fraction bits and the rounding bit; a carry moves into the exponent
  const unsigned bits = ((unsigned)le << 23) + ((m >> 5) & 0x7fffffu) + ((m >> 4) & 1u);
  return {h, __uint_as_float(sgn | bits)};
}

// FP64 value of an FP32 number by its bits (exact; zero and subnormal inputs give a signed
// zero, infinities and NaN keep their class); no FP64 instruction.
__device__ __forceinline__ double f64_of(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned long long s = (unsigned long long)(b & 0x80000000u) << 32;
  if (e == 0u) return __longlong_as_double((long long)s);
  const unsigned long long de = e == 0xffu ? 0x7ffull : (unsigned long long)(e + (1023u - 127u));
  return __longlong_as_double((long long)(s | (de << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}
// h + l in FP64: exact, since l is below 2^-24 of h (one FP64 addition)
__device__ __forceinline__ double dbl_of(ff a) { return f64_of(a.h) + f64_of(a.l); }

// 1/sqrt(x) for x > 0 in the FP32 normal range: the special function unit's estimate y0,
// e = 1 - x y0^2 formed with the exact square of y0, then y0 (1 + e/2 + 3 e^2/8) (third
// order; e <= 2^-21 leaves 2^-60) kept as y0 plus a correction term.
__device__ __forceinline__ ff ff_rsqrt(ff x) {
  const float y0 = rsqrtf(x.h);
  const ff q = ff_two_prod(y0, y0);
  float e = __fmaf_rn(-x.h, q.h, 1.0f);
  e = __fmaf_rn(-x.h, q.l, e);
  e = __fmaf_rn(-x.l, q.h, e);
  const float c = __fmul_rn(__fmul_rn(y0, e), __fmaf_rn(e, 0.375f, 0.5f));
  return ff_fast_two_sum(y0, c);
}

// sin and cos of th (two-float) by the table method of Gal and Bachelis (ACM TOMS 17,
// 1991), as sincos_tab: th = j (2 pi / 1024) + t, |t| <= pi / 1024, with the step split
// into three FP32 parts (Cody and Waite) and jd C1 formed exactly, so that t carries the
// two-float precision of th; sin t through t^5, cos t = 1 - t^2/2 + t^4/24 with t^2 exact;
// the table holds (cos, sin)(2 pi j / 1024) as two-float pairs.  Returns false (and
// computes nothing) for |th| >= 2^14 or a non-finite th.
__device__ __forceinline__ bool ff_sincos(ff th, const float4* __restrict__ tab, ff* sn, ff* cs) {
  if (!(fabsf(th.h) < 16384.0f)) return false;
  constexpr float kInvStep = 162.97466f;           // 1024 / (2 pi)
  constexpr float kShift = 12582912.0f;            // 1.5 2^23
  constexpr float C1 = 0x1.921fb6p-8f;             // 2 pi / 1024 = C1 + C2 + C3 (+ 4e-26)
  constexpr float C2 = -0x1.777a5cp-33f;
  constexpr float C3 = -0x1.ee59dap-58f;
  const float y = __fmaf_rn(th.h, kInvStep, kShift);
  const int j = __float_as_int(y) & 1023;
  const float jd = __fsub_rn(y, kShift);          // |jd| < 2^22: an exact integer
  const ff p = ff_two_prod(jd, C1);
  const float t0 = __fsub_rn(th.h, p.h);          // exact (Sterbenz)
  float tl = __fsub_rn(th.l, p.l);
  tl = __fmaf_rn(-jd, C2, tl);
  tl = __fmaf_rn(-jd, C3, tl);
  const ff t = ff_two_sum(t0, tl);
  const ff z = ff_two_prod(t.h, t.h);
  // sin t = t - t^3/6 + t^5/120, normalised
  const ff st = ff_fast_two_sum(
      t.h, __fmaf_rn(__fmul_rn(t.h, z.h), __fmaf_rn(z.h, 1.0f / 120.0f, -1.0f / 6.0f), t.l));
  // cos t = 1 - z/2 - (z_l/2 + t_h t_l) + z^2/24
  ff ct = ff_fast_two_sum(1.0f, __fmul_rn(-0.5f, z.h));
  ct.l = __fadd_rn(ct.l, __fmaf_rn(__fmul_rn(z.h, z.h), 1.0f / 24.0f,
                                   __fmaf_rn(-t.h, t.l, __fmul_rn(-0.5f, z.l))));
  const float4 e = __ldg(tab + j);
  const ff C = {e.x, e.y}, S = {e.z, e.w};
  *cs = ff_sub(ff_mul(C, ct), ff_mul(S, st));
  *sn = ff_add(ff_mul(S, ct), ff_mul(C, st));
  return true;
}

// The two-float terms of a dot product a . b with a, b two-float 3-vectors.
__device__ __forceinline__ ff ff_dot3(const ff* a, const ff* b) {
  ff p[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p[c] = ff_two_prod(a[c].h, b[c].h);
    p[c].l = __fmaf_rn(a[c].h, b[c].l, p[c].l);
    p[c].l = __fmaf_rn(a[c].l, b[c].h, p[c].l);
  }
  const ff s1 = ff_two_sum(p[0].h, p[1].h);
  const ff s2 = ff_two_sum(s1.h, p[2].h);
  const float lo = __fadd_rn(__fadd_rn(s1.l, s2.l), __fadd_rn(__fadd_rn(p[0].l, p[1].l), p[2].l));
  return ff_fast_two_sum(s2.h, lo);
}

}  // namespace lcq
