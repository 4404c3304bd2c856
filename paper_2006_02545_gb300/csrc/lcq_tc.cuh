// Building blocks of the split-precision tensor-core contraction and the lean FP64 kernel
// evaluation used by the adaptive near integration (Sec. 4.3).
//
// On GB300 the FP64 pipe retires 2 FMA per clock per SM (measured 1.26 TFLOP/s), the FP32
// pipe 128 and the warp-level f16 tensor-core MMA about 0.47 m16n8k16 per clock per SM
// (measured 602 TFLOP/s).  The dense part of the adaptive integration, the contraction of
// kernel values (targets x leaf nodes) with basis values (leaf nodes x n), is therefore
// done exactly on the tensor cores: each FP64 operand is written as a sum of NS slices of
// 7 bits on a common power-of-two scale (the row's for the kernel values, a fixed per-column
// bound for the basis values; the Ozaki splitting of Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59, 2012), every product of two slices (< 2^14) and every sum of them
// over a chunk of at most 128 nodes and over the at most 8 slice pairs of one diagonal stays
// below 2^24, so the f16 MMA with FP32 accumulators computes each diagonal exactly; the
// diagonals are combined in 64-bit integers and converted to FP64 once per chunk.  With
// NS = 8 (56 bits per operand) and the diagonals i + j <= 8 (43 MMAs per 16-node step; the
// dropped products are below 2^-60 of the operands' scales) the result matches an FP64
// contraction to the FP64 rounding level of the sum of |products|.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lcq_device.cuh"
#include "lcq_ff.cuh"

namespace lcq {

constexpr int kSliceBits = 7;
constexpr int kPoisonExp = 0x40000000;  // row exponent marking a non-finite kernel value

// Shared-memory layout of the tensor-core moment engine for degree D (byte offsets).  The
// f16 slice arrays are [slice][row][CH] with the 16-byte chunks of each row XOR-swizzled by
// the row index (swz), so that ldmatrix reads 8 rows of one chunk without bank conflicts.
template <int D>
struct TcCfg {
  static constexpr int n = (D + 1) * (D + 2) / 2;
  static constexpr int NP = (n + 7) / 8 * 8;       // basis columns padded to MMA n-tiles of 8
  static constexpr int NTILE = NP / 8;
  static constexpr int CH = D <= 6 ? 128 : 64;     // padded nodes per chunk (multiple of 16)
  static constexpr int TT = 8;                     // targets per tile: 16 MMA rows (Re, then Im)
  static constexpr int NSMAX = 8;                  // slices per FP64 operand
  static constexpr int MAXP = CH / 16;             // pieces (segment parts) per chunk at most
  static constexpr int OFF_X = 0;                                  // Xs[3][CH] double
  static constexpr int OFF_N = OFF_X + 3 * CH * 8;                 // Ns[3][CH] double (N w)
  static constexpr int OFF_J = OFF_N + 3 * CH * 8;                 // Js[CH] double (J w)
  static constexpr int OFF_K = OFF_J + CH * 8;                     // Ks[CH] double (folded)
  static constexpr int OFF_BS = OFF_K + CH * 8;                    // Bsl[NSMAX][NP][CH] f16
  static constexpr int OFF_G = OFF_BS + NSMAX * NP * CH * 2;       // Gs + Ef / Asl / row factors
  static constexpr int G_EVAL = TT * CH * 16 + TT * CH * 4;        // Gs[TT][CH] cplx, Ef[TT][CH]
  static constexpr int G_A = NSMAX * 16 * CH * 2;                  // Asl[NSMAX][16][CH] f16
  static constexpr int G_BYTES = G_A > G_EVAL ? G_A : G_EVAL;
  static constexpr int OFF_EF = OFF_G + TT * CH * 16;              // Ef, after Gs
  static constexpr int OFF_JF = OFF_G + G_BYTES;                   // Jf[CH] float
  static constexpr int OFF_NF = OFF_JF + CH * 4;                   // Nf[3][CH] float (mixed)
  static constexpr int OFF_ROWE = OFF_NF + 3 * CH * 4;             // rowE[16] int
  static constexpr int OFF_TX = (OFF_ROWE + 16 * 4 + 15) / 16 * 16;  // tx[3 TT], tn[3 TT] double
  static constexpr int OFF_CI = OFF_TX + 6 * TT * 8;               // colinfo[CH] int
  static constexpr int OFF_PC = OFF_CI + CH * 4;                   // pieces[MAXP][8] int
  static constexpr int BYTES = OFF_PC + MAXP * 8 * 4;
  // element (row, k) of a [rows][CH] f16 array, 16-byte chunks XOR-swizzled by row
  static __device__ __forceinline__ int swz(int row, int k) {
    return row * CH + ((((k >> 3) ^ (row & 7)) << 3) | (k & 7));
  }
};

// |x| 2^(7 NS - E) rounded to the nearest integer, for |x| < 2^E: below 2^(7 NS).  Zero,
// subnormal and non-finite x give 0 (non-finite values are flagged by the caller).
template <int NS>
__device__ __forceinline__ unsigned long long fix_mag(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0 || ex == 0x7ff) return 0ull;
  const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;  // 53 bits
  const int sh = 1075 + E - ex - kSliceBits * NS;
  unsigned long long M;
  if (sh <= 0) {
    M = m << (-sh);
  } else {
    if (sh >= 54) return 0ull;
    M = (m + (1ull << (sh - 1))) >> sh;
  }
  const unsigned long long top = (1ull << (kSliceBits * NS)) - 1ull;
  return M < top ? M : top;
}
template <int NS>
__device__ __forceinline__ unsigned long long fix_mag(float x, int E) {
  const unsigned b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xff);
  if (ex == 0 || ex == 0xff) return 0ull;
  const unsigned long long m = (b & 0x7fffffu) | 0x800000u;  // 24 bits
  const int sh = 150 + E - ex - kSliceBits * NS;
  unsigned long long M;
  if (sh <= 0) {
    M = m << (-sh);
  } else {
    if (sh >= 25) return 0ull;
    M = (m + (1ull << (sh - 1))) >> sh;
  }
  const unsigned long long top = (1ull << (kSliceBits * NS)) - 1ull;
  return M < top ? M : top;
}

// Biased exponent field and the exponent E with |x| < 2^E for a normal number.
__device__ __forceinline__ int exp_field(double x) {
  return (int)((((unsigned long long)__double_as_longlong(x)) >> 52) & 0x7ff);
}
__device__ __forceinline__ int exp_field(float x) { return (int)((__float_as_uint(x) >> 23) & 0xff); }
__device__ __forceinline__ int exp_bound(int field, double) { return field - 1022; }
__device__ __forceinline__ int exp_bound(int field, float) { return field - 126; }
__device__ __forceinline__ bool exp_nonfinite(int field, double) { return field == 0x7ff; }
__device__ __forceinline__ bool exp_nonfinite(int field, float) { return field == 0xff; }

// Slice i (0: most significant) of M, 7 bits.
template <int NS>
__device__ __forceinline__ unsigned slice_of(unsigned long long M, int i) {
  return (unsigned)(M >> (kSliceBits * (NS - 1 - i))) & 0x7fu;
}

// Two f16 values (low half first) holding the integers c0, c1 in [0, 128) with the given
// signs: 1024 + c is the f16 bit pattern 0x6400 | c, and subtracting 1024 is exact.
__device__ __forceinline__ uint32_t half2_ints(unsigned c0, unsigned c1, uint32_t signs) {
  const uint32_t w = (0x6400u | c0) | ((0x6400u | c1) << 16);
  uint32_t r;
  asm("sub.f16x2 %0, %1, %2;" : "=r"(r) : "r"(w), "r"(0x64006400u));
  return r ^ signs;
}
// Slices i and i + 1 of one value as two f16 values (low half: slice i), negative when neg:
// -(1024 + c) is 0xE400 | c, and subtracting -1024 leaves -c.
__device__ __forceinline__ uint32_t half2_pair(unsigned c0, unsigned c1, bool neg) {
  const uint32_t base = neg ? 0xE400E400u : 0x64006400u;
  const uint32_t w = base | c0 | (c1 << 16);
  uint32_t r;
  asm("sub.f16x2 %0, %1, %2;" : "=r"(r) : "r"(w), "r"(base));
  return r;
}

__device__ __forceinline__ uint32_t sign_bits(double a, double b) {
  return ((uint32_t)(__double2hiint(a) < 0) << 15) | ((uint32_t)(__double2hiint(b) < 0) << 31);
}
__device__ __forceinline__ uint32_t sign_bits(float a, float b) {
  return ((__float_as_uint(a) >> 31) << 15) | ((__float_as_uint(b) >> 31) << 31);
}

// D += A B for one m16n8k16 tile: A row-major f16 (4 registers), B column-major f16 (2),
// D FP32 (4).
__device__ __forceinline__ void mma_f16_16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The four 8x8 f16 matrices of an m16n8k16 A operand from shared memory; p is this lane's row
// address (rows (lane & 7) + 8 ((lane >> 3) & 1), columns 8 (lane >> 4) of the 16x16 tile).
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// FP64 value of one accumulator element: the diagonals d = 0..ND-1 (exact integers in FP32)
// weighted 2^(-7 d), combined in 64-bit integers (two halves of at most 53 bits, so that each
// converts exactly), times 2^(E - 14 - 7 (ND - 1)), E = Ea + Eb.
template <int ND>
__device__ __forceinline__ double assemble(const float (*acc)[4], int e, int E) {
  if (E >= kPoisonExp / 2) return __longlong_as_double(0x7ff8000000000000ll);  // NaN
  double v;
  if (ND <= 5) {
    long long s = 0;
#pragma unroll
    for (int d = 0; d < ND; ++d)
      s += (long long)__float2int_rn(acc[d][e]) * (1ll << (kSliceBits * (ND - 1 - d)));
    v = (double)s;
  } else {
    constexpr int H = ND / 2;  // diagonals 0..H-1 in hi, H..ND-1 in lo
    long long hi = 0, lo = 0;
#pragma unroll
    for (int d = 0; d < H; ++d)
      hi += (long long)__float2int_rn(acc[d][e]) * (1ll << (kSliceBits * (H - 1 - d)));
#pragma unroll
    for (int d = H; d < ND; ++d)
      lo += (long long)__float2int_rn(acc[d][e]) * (1ll << (kSliceBits * (ND - 1 - d)));
    v = fma((double)hi, (double)(1ll << (kSliceBits * (ND - H))), (double)lo);
  }
  const int ue = E - 2 * kSliceBits - kSliceBits * (ND - 1);
  if (ue < -1022) return 0.0;
  return v * __longlong_as_double((long long)(ue + 1023) << 52);
}

// FP32 value of an FP64 number by its bits (truncating the mantissa; exponents outside the
// FP32 range flush to zero or saturate): no FP64 instruction, for quantities that only set
// a tolerance floor.
__device__ __forceinline__ float f32_bits(double x) {
  const long long b = __double_as_longlong(x);
  const int hi = (int)(b >> 32);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  if (e <= 0) return 0.0f;
  const unsigned s = (unsigned)hi & 0x80000000u;
  if (e >= 255) return __uint_as_float(s | 0x7f800000u);
  return __uint_as_float(s | ((unsigned)e << 23) | ((unsigned)(b >> 29) & 0x7fffffu));
}

// FP64 value of a positive normal FP32 number by its bits (exact; no FP64 instruction).
__device__ __forceinline__ double f64_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned long long e = (unsigned long long)(((b >> 23) & 0xffu) + (1023u - 127u));
  return __longlong_as_double((long long)((e << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// 1/sqrt(x) for x > 0: the FP32 estimate (special function unit) refined by one third-order
// Newton-Raphson step in FP64, y1 = y0 (1 + e/2 + 3 e^2/8) with e = 1 - x y0^2 (relative
// error O(e^3), e <= 2^-21): five FP64 instructions.  Arguments outside the FP32 range
// take rsqrt().
__device__ __forceinline__ double rsqrt_nr(double x) {
  const int ex = (__double2hiint(x) >> 20) & 0x7ff;
  if (ex < 1023 - 120 || ex > 1023 + 120) return rsqrt(x);
  const double y0 = f64_bits(rsqrtf(f32_bits(x)));
  const double e = fma(-(x * y0), y0, 1.0);
  return fma(y0, e * fma(e, 0.375, 0.5), y0);
}

// sin and cos of th by table lookup and Taylor polynomials (the table method of Gal and
// Bachelis, ACM TOMS 17, 1991): th = j (2 pi / 1024) + t with j = rint(th 1024 / (2 pi))
// (the 1.5 2^52 shifter) and |t| <= pi / 1024; sin t through t^5 and cos t through t^4
// (the next terms are below 2^-59 relative); then the angle-addition formulas with the
// table's (cos, sin)(2 pi j / 1024): 13 FP64 instructions.  Valid for |th| < 2^20 (j times
// the 27-bit leading part of the step stays exact); larger arguments use sincos().
__device__ __forceinline__ void sincos_tab(double th, const double2* __restrict__ tab, double* sn,
                                           double* cs) {
  if (((__double2hiint(th) >> 20) & 0x7ff) >= 1023 + 20) {  // |th| >= 2^20 or not finite
    sincos(th, sn, cs);
    return;
  }
  constexpr double kInvStep = 162.97466172610083;        // 1024 / (2 pi)
  constexpr double kStepHi = 0x1.921fb54p-8;             // 2 pi / 1024 to 27 bits
  constexpr double kStepLo = 3.875365545627111e-12;      // 2 pi / 1024 - kStepHi
  constexpr double kShift = 6755399441055744.0;          // 1.5 2^52
  const double y = fma(th, kInvStep, kShift);
  const int j = __double2loint(y) & (kSinCosTable - 1);
  const double jd = y - kShift;
  double t = fma(-jd, kStepHi, th);
  t = fma(-jd, kStepLo, t);
  const double z = t * t;
  const double s = fma(t * z, fma(z, 1.0 / 120.0, -1.0 / 6.0), t);
  const double c = fma(z, fma(z, 1.0 / 24.0, -0.5), 1.0);
  const double2 e = __ldg(tab + j);
  *cs = fma(e.x, c, -e.y * s);
  *sn = fma(e.y, c, e.x * s);
}

// kernel_eval_tc for real k, kinds S, D and CFIE with a real alpha, with the constants folded
// into the per-node source data: N' = N w alpha / (4 pi) (alpha = 1 for D), Js = beta_r Jw /
// (4 pi) (Jw / (4 pi) for S), Ks = beta_i Jw / (4 pi), fJ = FP32 Jw / (4 pi).  Then
//   S: e^{ikr}/r Js,   D and CFIE: e^{ikr}/r ((1 - ikr) N'.d / r^2 + Js + i Ks),
// about 39 FP64 instructions for the CFIE.  r = 0 gives 0.
__device__ __forceinline__ cplx kernel_eval_fold(int kind, double kr, const KernelParamsF& kf,
                                                 const double2* __restrict__ sct, double x0,
                                                 double x1, double x2, double X0, double X1,
                                                 double X2, double N0, double N1, double N2,
                                                 double Js, double Ks, float fJ, float fR,
                                                 float* env) {
  const double d0 = x0 - X0, d1 = x1 - X1, d2 = x2 - X2;
  const double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
  if ((__double_as_longlong(r2) << 1) == 0) {
    *env = 0.0f;
    return {0.0, 0.0};
  }
  const double rinv = rsqrt_nr(r2);
  const double r = r2 * rinv;
  const double th = kr * r;
  double sn, cs;
  sincos_tab(th, sct, &sn, &cs);
  {
    // |G| Jw (|beta| + |alpha| |1 - ik r| R / r^2) in FP32, k real
    const float fri = f32_bits(rinv), f1 = kf.kr * f32_bits(r);
    const float fa = sqrtf(fmaf(f1, f1, 1.0f));
    *env = fri * fJ * fmaf(kf.ea * fa * fR, fri * fri, kf.eb);
  }
  const double ec = cs * rinv, es = sn * rinv;
  if (kind == 0) return {ec * Js, es * Js};
  const double nd = fma(N0, d0, fma(N1, d1, N2 * d2)) * (rinv * rinv);
  const double mr = kind == 2 ? nd + Js : nd;
  const double mi = kind == 2 ? fma(-th, nd, Ks) : -th * nd;
  return {fma(ec, mr, -es * mi), fma(ec, mi, es * mr)};
}

// kernel_eval_fold in two-float arithmetic (lcq_ff.cuh) on the FP32 pipe: x - X in FP64 (the
// difference stays FP64 near the singularity), then r^2, 1/r, k r, e^{ikr} and the S, D and
// CFIE factors in two-float, the result converted to FP64 exactly; five FP64 instructions.
// Np, Js, Ks: the folded node data (as kernel_eval_fold) as two-float pairs; krf: k.  Each
// value carries a relative error of a few 2^-46 (plus k r 2^-48 in the phase).  Arguments
// outside the two-float range (r^2 outside [1e-30, 1e30], |k r| >= 2^14) take
// kernel_eval_fold.  r = 0 gives 0.
__device__ __forceinline__ cplx kernel_eval_ff(int kind, double kr, ff krf, const KernelParamsF& kf,
                                               const double2* __restrict__ sct,
                                               const float4* __restrict__ sctf, double x0,
                                               double x1, double x2, double X0, double X1,
                                               double X2, const ff* Np, ff Js, ff Ks, float fJ,
                                               float fR, float* env) {
  const double dd0 = x0 - X0, dd1 = x1 - X1, dd2 = x2 - X2;
  if (((__double_as_longlong(dd0) | __double_as_longlong(dd1) | __double_as_longlong(dd2)) << 1) ==
      0) {
    *env = 0.0f;
    return {0.0, 0.0};
  }
  const ff d[3] = {ff_of(dd0), ff_of(dd1), ff_of(dd2)};
  // r^2: exact squares of the leading parts plus 2 d_h d_l (d_l^2 is below 2^-48 of d_h^2)
  ff sq[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    sq[c] = ff_two_prod(d[c].h, d[c].h);
    sq[c].l = __fmaf_rn(2.0f * d[c].h, d[c].l, sq[c].l);
  }
  const ff s1 = ff_two_sum(sq[0].h, sq[1].h), s2 = ff_two_sum(s1.h, sq[2].h);
  const ff r2 = ff_fast_two_sum(
      s2.h, __fadd_rn(__fadd_rn(s1.l, s2.l), __fadd_rn(__fadd_rn(sq[0].l, sq[1].l), sq[2].l)));
  bool ok = r2.h >= 1e-30f && r2.h <= 1e30f;
  ff rinv = {0.0f, 0.0f}, r = rinv, th = rinv, sn = rinv, cs = rinv;
  if (ok) {
    rinv = ff_rsqrt(r2);
    r = ff_mul(r2, rinv);
    th = ff_mul(krf, r);
    ok = ff_sincos(th, sctf, &sn, &cs);
  }
  if (!ok)
    return kernel_eval_fold(kind, kr, kf, sct, x0, x1, x2, X0, X1, X2, dbl_of(Np[0]), dbl_of(Np[1]),
                            dbl_of(Np[2]), dbl_of(Js), dbl_of(Ks), fJ, fR, env);
  {
    // |G| Jw (|beta| + |alpha| |1 - ik r| R / r^2) in FP32, k real
    const float fri = rinv.h, f1 = kf.kr * r.h;
    const float fa = sqrtf(fmaf(f1, f1, 1.0f));
    *env = fri * fJ * fmaf(kf.ea * fa * fR, fri * fri, kf.eb);
  }
  const ff ec = ff_mul(cs, rinv), es = ff_mul(sn, rinv);
  ff re, im;
  if (kind == 0) {
    re = ff_mul(ec, Js);
    im = ff_mul(es, Js);
  } else {
    const ff nd = ff_mul(ff_dot3(Np, d), ff_mul(rinv, rinv));
    const ff tn = ff_mul(th, nd);
    const ff mr = kind == 2 ? ff_add(nd, Js) : nd;
    const ff mi = kind == 2 ? ff_sub(Ks, tn) : ff_neg(tn);
    re = ff_sub(ff_mul(ec, mr), ff_mul(es, mi));
    im = ff_add(ff_mul(ec, mi), ff_mul(es, mr));
  }
  return {dbl_of(re), dbl_of(im)};
}

// kernel_eval (lcq_device.cuh) with the table sincos, the Newton-refined FP32 reciprocal
// square root and the rounding envelope formed in FP32 from the FP64 quantities' bits: the
// same kernel value to a few ulps.  fJw: FP32 copy of Jw; fR: FP32 patch radius; has_ki:
// Im k != 0.  r = 0 gives 0.
__device__ __forceinline__ cplx kernel_eval_tc(const KernelParams& kp, const KernelParamsF& kf,
                                               const double2* __restrict__ sct, double x0,
                                               double x1, double x2, double X0, double X1,
                                               double X2, double N0, double N1, double N2,
                                               double Jw, float fJw, float fR, float* env,
                                               const double* nx, bool has_ki) {
  if (kp.kind == 3) {
    N0 = -nx[0] * Jw;
    N1 = -nx[1] * Jw;
    N2 = -nx[2] * Jw;
  }
  const double d0 = x0 - X0, d1 = x1 - X1, d2 = x2 - X2;
  const double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
  if ((__double_as_longlong(r2) << 1) == 0) {
    *env = 0.0f;
    return {0.0, 0.0};
  }
  const double rinv = rsqrt_nr(r2);
  const double r = r2 * rinv;
  const double th = kp.kr * r;
  double sn, cs;
  sincos_tab(th, sct, &sn, &cs);
  double ex = 0.07957747154594767 * rinv;  // 1/(4 pi r)
  if (has_ki) ex *= exp(-kp.ki * r);
  {
    // |G| Jw (|beta| + |alpha| |1 - ik r| R / r^2) in FP32
    const float fr = f32_bits(r), fri = 1.0f / fr;
    const float f0 = fmaf(kf.ki, fr, 1.0f), f1 = kf.kr * fr;
    const float fa = sqrtf(fmaf(f0, f0, f1 * f1));
    *env = f32_bits(ex) * fJw * fmaf(kf.ea * fa * fR, fri * fri, kf.eb);
  }
  const double ec = ex * cs, es = ex * sn;
  if (kp.kind == 0) return {ec * Jw, es * Jw};
  const double rinv2 = rinv * rinv;
  const double ndx = fma(N0, d0, fma(N1, d1, N2 * d2)) * rinv2;
  // (1 - ikr) ndx with k = kr + i ki: ((1 + ki r) ndx, -kr r ndx)
  double cr = has_ki ? fma(kp.ki, r, 1.0) * ndx : ndx;
  double ci = -th * ndx;
  if (kp.kind == 2) {
    const double tr = fma(kp.ar, cr, fma(-kp.ai, ci, kp.br * Jw));
    const double ti = fma(kp.ar, ci, fma(kp.ai, cr, kp.bi * Jw));
    cr = tr;
    ci = ti;
  }
  return {fma(ec, cr, -es * ci), fma(ec, ci, es * cr)};
}

}  // namespace lcq
