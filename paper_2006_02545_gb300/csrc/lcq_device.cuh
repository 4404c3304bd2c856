// Device building blocks: Koornwinder recurrences (Sec. 2, Eq. for K_nm), chart
// geometry (Sec. 3.1-3.2) and the Helmholtz kernels times the area element
// (Sec. 3, Eq. greenfunhelm, sldef, dldef, urep).  Templated on the patch degree D
// so that the basis loops unroll into registers.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "lcq_internal.h"

namespace lcq {

// c_nm = sqrt(2(2m+1)(n+1)), index n(n+1)/2 + m; filled once per device.
// (static: each translation unit holds and uploads its own copy)
static __constant__ double c_kw[kMaxBasis];

struct cplx {
  double re, im;
};

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// Jacobi P^{(0,b)}_a three-term recurrence coefficients (alpha = 0):
//   P_{a+1} = (c1 y + c0) P_a - c2 P_{a-1}.
// All arguments are compile-time constants after unrolling, so these fold.
__host__ __device__ __forceinline__ void jacobi_coef(int a, int b, double* c1, double* c0,
                                                     double* c2) {
  const double den = 2.0 * (a + 1) * (a + b + 1) * (2 * a + b);
  *c1 = (double)((2 * a + b + 1) * (2 * a + b + 2) * (2 * a + b)) / den;
  *c0 = -(double)((2 * a + b + 1) * b * b) / den;
  *c2 = (double)(2 * a * (a + b) * (2 * a + b + 2)) / den;
}

// Three-term coefficients of P^{(0, 2m+1)}_a, [m][a][c1, c0, c2], for loops that are not
// unrolled; same values as jacobi_coef.  Filled with c_kw by upload_kw_tables.
static __constant__ double c_jac[(kMaxDeg + 1) * (kMaxDeg + 1) * 3];

// Exponents E_nm with |K_nm| < 2^E_nm on T0: |(1-v)^m P_m| <= 1 there and, for Jacobi
// polynomials with max(alpha, beta) >= -1/2, max |P^{(0,b)}_a| on [-1, 1] = binom(a + b, a)
// (Szego, Orthogonal Polynomials, Thm. 7.32.1), so |K_nm| <= c_nm binom(n + m + 1, n - m).
// The split-precision contraction scales basis column nm by 2^-E_nm.
static __constant__ int c_kwexp[kMaxBasis];

// (cos, sin)(2 pi j / 1024), j = 0..1023: the table of sincos_tab (lcq_tc.cuh).
constexpr int kSinCosTable = 1024;
static __device__ double2 g_sct[kSinCosTable];
// the same angles as two-float pairs (cos_h, cos_l, sin_h, sin_l) for the two-float kernel
static __device__ float4 g_sctf[kSinCosTable];

// Fills c_kw, c_jac, c_kwexp, g_sct and g_sctf of the calling translation unit.
static inline cudaError_t upload_kw_tables(cudaStream_t st) {
  double c[kMaxBasis], jc[(kMaxDeg + 1) * (kMaxDeg + 1) * 3] = {};
  int ke[kMaxBasis];
  std::vector<double2> sct(kSinCosTable);
  std::vector<float4> sctf(kSinCosTable);
  for (int nn = 0; nn <= kMaxDeg; ++nn)
    for (int m = 0; m <= nn; ++m) {
      const int idx = nn * (nn + 1) / 2 + m;
      c[idx] = sqrt(2.0 * (2 * m + 1) * (nn + 1));
      double binom = 1.0;  // binom(n + m + 1, n - m)
      for (int i = 1; i <= nn - m; ++i) binom = binom * (2 * m + 1 + i) / i;
      int e2 = 0;
      frexp(c[idx] * binom * (1.0 + 1e-12), &e2);
      ke[idx] = e2;
    }
  for (int m = 0; m <= kMaxDeg; ++m) {
    for (int a = 0; a <= kMaxDeg; ++a) {
      double* q = jc + (m * (kMaxDeg + 1) + a) * 3;
      jacobi_coef(a, 2 * m + 1, q, q + 1, q + 2);
    }
  }
  for (int j = 0; j < kSinCosTable; ++j) {
    const double a = 2.0 * M_PI * j / kSinCosTable;
    sct[j] = make_double2(cos(a), sin(a));
    const float ch = (float)sct[j].x, sh = (float)sct[j].y;
    sctf[j] = make_float4(ch, (float)(sct[j].x - ch), sh, (float)(sct[j].y - sh));
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_kw, c, sizeof(c), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(c_jac, jc, sizeof(jc), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(c_kwexp, ke, sizeof(ke), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(g_sct, sct.data(), sizeof(double2) * kSinCosTable, 0,
                                cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbolAsync(g_sctf, sctf.data(), sizeof(float4) * kSinCosTable, 0,
                                cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the sources live on this stack
  return e;
}

// Koornwinder values K[nm] at (u, v) written with stride `ks`.
template <int D>
__device__ __forceinline__ void kw_values(double u, double v, double* K, int ks) {
  const double s = 2.0 * u + v - 1.0, q2 = (1.0 - v) * (1.0 - v), y = 1.0 - 2.0 * v;
  double Lp = 0.0, L = 1.0;
#pragma unroll
  for (int m = 0; m <= D; ++m) {
    if (m > 0) {
      const double Ln = ((2.0 * m - 1.0) * s * L - (m - 1.0) * q2 * Lp) * (1.0 / m);
      Lp = L;
      L = Ln;
    }
    const int b = 2 * m + 1;
    double Pp = 0.0, P = 1.0;
#pragma unroll
    for (int a = 0; a <= D - m; ++a) {
      const int n = m + a, idx = n * (n + 1) / 2 + m;
      K[idx * ks] = c_kw[idx] * L * P;
      if (a < D - m) {
        double c1, c0, c2;
        jacobi_coef(a, b, &c1, &c0, &c2);
        const double Pn = (c1 * y + c0) * P - c2 * Pp;
        Pp = P;
        P = Pn;
      }
    }
  }
}

// Chart X, X_u, X_v at (u, v) from Koornwinder coefficients cf[nm][3]; optionally
// also K values (stride ks) when K != nullptr.
template <int D>
__device__ __forceinline__ void kw_geometry(double u, double v, const double* __restrict__ cf,
                                            double* X, double* Xu, double* Xv, double* K, int ks) {
  const double s = 2.0 * u + v - 1.0, q = 1.0 - v, q2 = q * q, y = 1.0 - 2.0 * v;
  double Lp = 0.0, L = 1.0, Lup = 0.0, Lu = 0.0, Lvp = 0.0, Lv = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) X[c] = Xu[c] = Xv[c] = 0.0;
#pragma unroll
  for (int m = 0; m <= D; ++m) {
    if (m > 0) {
      const double f1 = 2.0 * m - 1.0, f2 = m - 1.0, im = 1.0 / m;
      const double Ln = (f1 * s * L - f2 * q2 * Lp) * im;
      const double Lun = (f1 * (2.0 * L + s * Lu) - f2 * q2 * Lup) * im;
      const double Lvn = (f1 * (L + s * Lv) - f2 * (-2.0 * q * Lp + q2 * Lvp)) * im;
      Lp = L;
      L = Ln;
      Lup = Lu;
      Lu = Lun;
      Lvp = Lv;
      Lv = Lvn;
    }
    const int b = 2 * m + 1;
    double Pp = 0.0, P = 1.0, dPp = 0.0, dP = 0.0;
#pragma unroll
    for (int a = 0; a <= D - m; ++a) {
      const int n = m + a, idx = n * (n + 1) / 2 + m;
      const double cn = c_kw[idx];
      const double k0 = cn * L * P;
      const double ku = cn * Lu * P;
      const double kv = cn * (Lv * P - 2.0 * L * dP);
      if (K) K[idx * ks] = k0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double x = cf[idx * 3 + c];
        X[c] = fma(x, k0, X[c]);
        Xu[c] = fma(x, ku, Xu[c]);
        Xv[c] = fma(x, kv, Xv[c]);
      }
      if (a < D - m) {
        double c1, c0, c2;
        jacobi_coef(a, b, &c1, &c0, &c2);
        const double t = c1 * y + c0;
        const double Pn = t * P - c2 * Pp;
        const double dPn = c1 * P + t * dP - c2 * dPp;
        Pp = P;
        P = Pn;
        dPp = dP;
        dP = dPn;
      }
    }
  }
}

// Chart X, X_u, X_v at (u, v) from the coefficients cf[nm][3] and the derivative series
// cfd = (X_u coefficients [nd][3], X_v coefficients [nd][3]) in the degree D-1 basis
// (nd its size: the first nd basis functions, those with n < D).  Only the values
// recurrence runs; K (stride 1, written first and read back) receives the basis values.
// Same polynomials as kw_geometry at about half its cost.  WITH_X = false: X is not
// formed (nor written).
template <int D, bool WITH_X = true>
__device__ __forceinline__ void kw_geometry_proj(double u, double v, const double* cf,
                                                 const double* cfd, double* X, double* Xu,
                                                 double* Xv, double* K) {
  constexpr int n = (D + 1) * (D + 2) / 2, nd = D * (D + 1) / 2;
  kw_values<D>(u, v, K, 1);
  double x0 = 0.0, x1 = 0.0, x2 = 0.0, u0 = 0.0, u1 = 0.0, u2 = 0.0, v0 = 0.0, v1 = 0.0,
         v2 = 0.0;
  // rolled loops over the stored values: keeps the coefficient loads next to their use
#pragma unroll 1
  for (int idx = 0; idx < nd; ++idx) {
    const double k = K[idx];
    if (WITH_X) {
      x0 = fma(cf[idx * 3], k, x0);
      x1 = fma(cf[idx * 3 + 1], k, x1);
      x2 = fma(cf[idx * 3 + 2], k, x2);
    }
    u0 = fma(cfd[idx * 3], k, u0);
    u1 = fma(cfd[idx * 3 + 1], k, u1);
    u2 = fma(cfd[idx * 3 + 2], k, u2);
    v0 = fma(cfd[(nd + idx) * 3], k, v0);
    v1 = fma(cfd[(nd + idx) * 3 + 1], k, v1);
    v2 = fma(cfd[(nd + idx) * 3 + 2], k, v2);
  }
  if (WITH_X) {
#pragma unroll 1
    for (int idx = nd; idx < n; ++idx) {
      const double k = K[idx];
      x0 = fma(cf[idx * 3], k, x0);
      x1 = fma(cf[idx * 3 + 1], k, x1);
      x2 = fma(cf[idx * 3 + 2], k, x2);
    }
    X[0] = x0;
    X[1] = x1;
    X[2] = x2;
  }
  Xu[0] = u0;
  Xu[1] = u1;
  Xu[2] = u2;
  Xv[0] = v0;
  Xv[1] = v1;
  Xv[2] = v2;
}

// Row form of kw_geometry_proj for nodes that share v.  K_nm = L_m(u, v) J_nm(v) with
// L_m = (1 - v)^m P_m((2u + v - 1) / (1 - v)) and J_nm = c_nm P^{(0,2m+1)}_{n-m}(1 - 2v), so
// per value of v the J factors and the chart's sums over n at fixed m can be formed once:
// row = [v, (1 - v)^2, Q (D+1), J (n), BX (3 (D+1)), BU (3 D), BV (3 D)], Q[m] = (m-1)/m
// (1 - v)^2 (the v-only coefficient of the L_m recurrence), BX[m][c] = sum_n cf_nm[c] J_nm
// and BU, BV likewise from the derivative series (n < D).
template <int D>
struct KwRow {
  static constexpr int n = (D + 1) * (D + 2) / 2;
  static constexpr int Q = 2, J = Q + D + 1, BX = J + n, BU = BX + 3 * (D + 1),
                       BV = BU + 3 * D;
  static constexpr int size = BV + 3 * D;
};

// The part of the row factors that belongs to one m (the header too when m = 0), so that
// a block spreads a row over D + 1 threads.
template <int D>
__device__ __forceinline__ void kw_row_factors(double v, int m, const double* cf,
                                               const double* cfd, double* row) {
  using RW = KwRow<D>;
  constexpr int nd = D * (D + 1) / 2;
  const double y = 1.0 - 2.0 * v;
  if (m == 0) {
    const double q2 = (1.0 - v) * (1.0 - v);
    row[0] = v;
    row[1] = q2;
#pragma unroll
    for (int mm = 0; mm <= D; ++mm) row[RW::Q + mm] = mm < 2 ? 0.0 : (mm - 1.0) / mm * q2;
  }
  double Pp = 0.0, P = 1.0;
  double x0 = 0.0, x1 = 0.0, x2 = 0.0, u0 = 0.0, u1 = 0.0, u2 = 0.0, v0 = 0.0, v1 = 0.0,
         v2 = 0.0;
  const double* jc = c_jac + m * (kMaxDeg + 1) * 3;
#pragma unroll 1
  for (int a = 0; a <= D - m; ++a) {
    const int nn = m + a, idx = nn * (nn + 1) / 2 + m;
    const double jv = c_kw[idx] * P;
    row[RW::J + idx] = jv;
    x0 = fma(cf[idx * 3], jv, x0);
    x1 = fma(cf[idx * 3 + 1], jv, x1);
    x2 = fma(cf[idx * 3 + 2], jv, x2);
    if (nn < D) {
      u0 = fma(cfd[idx * 3], jv, u0);
      u1 = fma(cfd[idx * 3 + 1], jv, u1);
      u2 = fma(cfd[idx * 3 + 2], jv, u2);
      v0 = fma(cfd[(nd + idx) * 3], jv, v0);
      v1 = fma(cfd[(nd + idx) * 3 + 1], jv, v1);
      v2 = fma(cfd[(nd + idx) * 3 + 2], jv, v2);
    }
    const double Pn = (jc[3 * a] * y + jc[3 * a + 1]) * P - jc[3 * a + 2] * Pp;
    Pp = P;
    P = Pn;
  }
  row[RW::BX + 3 * m] = x0;
  row[RW::BX + 3 * m + 1] = x1;
  row[RW::BX + 3 * m + 2] = x2;
  if (m < D) {
    row[RW::BU + 3 * m] = u0;
    row[RW::BU + 3 * m + 1] = u1;
    row[RW::BU + 3 * m + 2] = u2;
    row[RW::BV + 3 * m] = v0;
    row[RW::BV + 3 * m + 1] = v1;
    row[RW::BV + 3 * m + 2] = v2;
  }
}

// X, X_u, X_v at (u, v) from the row factors of v; each basis value K_nm is handed to
// emit(idx, K_nm) as it is formed (idx = n(n+1)/2 + m).
template <int D, class F>
__device__ __forceinline__ void kw_geometry_row_emit(double u, const double* row, double* X,
                                                     double* Xu, double* Xv, F&& emit) {
  using RW = KwRow<D>;
  const double v = row[0];
  const double s = 2.0 * u + v - 1.0;
  double Lp = 0.0, L = 1.0;
  double x0 = 0.0, x1 = 0.0, x2 = 0.0, u0 = 0.0, u1 = 0.0, u2 = 0.0, v0 = 0.0, v1 = 0.0,
         v2 = 0.0;
#pragma unroll
  for (int m = 0; m <= D; ++m) {
    if (m > 0) {
      // m L_m = (2m - 1) s L_{m-1} - (m - 1) (1 - v)^2 L_{m-2}, the v-only factor per row
      const double Ln = m == 1 ? s : fma((2.0 * m - 1.0) / m * s, L, -row[RW::Q + m] * Lp);
      Lp = L;
      L = Ln;
    }
    x0 = fma(row[RW::BX + 3 * m], L, x0);
    x1 = fma(row[RW::BX + 3 * m + 1], L, x1);
    x2 = fma(row[RW::BX + 3 * m + 2], L, x2);
    if (m < D) {
      u0 = fma(row[RW::BU + 3 * m], L, u0);
      u1 = fma(row[RW::BU + 3 * m + 1], L, u1);
      u2 = fma(row[RW::BU + 3 * m + 2], L, u2);
      v0 = fma(row[RW::BV + 3 * m], L, v0);
      v1 = fma(row[RW::BV + 3 * m + 1], L, v1);
      v2 = fma(row[RW::BV + 3 * m + 2], L, v2);
    }
#pragma unroll
    for (int a = 0; a <= D - m; ++a) {
      const int nn = m + a, idx = nn * (nn + 1) / 2 + m;
      emit(idx, L * row[RW::J + idx]);
    }
  }
  X[0] = x0;
  X[1] = x1;
  X[2] = x2;
  Xu[0] = u0;
  Xu[1] = u1;
  Xu[2] = u2;
  Xv[0] = v0;
  Xv[1] = v1;
  Xv[2] = v2;
}

// X, X_u, X_v and the basis values K (stride 1) at (u, v) from the row factors of v.
template <int D>
__device__ __forceinline__ void kw_geometry_row(double u, const double* row, double* X,
                                                double* Xu, double* Xv, double* K) {
  kw_geometry_row_emit<D>(u, row, X, Xu, Xv, [&](int idx, double k) { K[idx] = k; });
}

// cfd for kw_geometry_proj from cf and the projections duv (Du [n][nd], then Dv), by
// the block's threads.
template <int D>
__device__ __forceinline__ void load_coef_derivs(const double* cf, const double* __restrict__ duv,
                                                 double* cfd) {
  constexpr int n = (D + 1) * (D + 2) / 2, nd = D * (D + 1) / 2;
  for (int e = threadIdx.x; e < 2 * nd * 3; e += blockDim.x) {
    const int which = e / (nd * 3), r = e - which * nd * 3, j = r / 3, c = r - 3 * j;
    const double* Dm = duv + (size_t)which * n * nd;
    double acc = 0.0;
    for (int nm = 0; nm < n; ++nm) acc = fma(cf[nm * 3 + c], Dm[nm * nd + j], acc);
    cfd[e] = acc;
  }
}

// Index helpers for bivariate power series in (du, dv) truncated at degree D: entry
// g(g+1)/2 + j holds the coefficient of du^(g-j) dv^j (the ordering of the basis).
__device__ __forceinline__ void tri_split(int e, int& g, int& j) {
  g = 0;
  while ((g + 1) * (g + 2) / 2 <= e) ++g;
  j = e - g * (g + 1) / 2;
}

// Taylor coefficients of the chord dX(d) = X(P + d) - X(P), d = (du, dv), of the chart
// X = sum_nm cf_nm K_nm of degree D, about the node P = (pu, pv): the Koornwinder
// recurrences of kw_values run on power series in (du, dv) truncated at degree D, which
// is exact for these polynomials, and their coefficients stay those of the derivatives
// at P (no expansion about another point, so no cancellation).  tX[c * n + e] receives
// the coefficient of entry e of component c, tX[c * n] = 0.  Block-wide, with
// __syncthreads; scratch holds (D + 1) n + 2 n^2 doubles.
template <int D>
__device__ void chart_taylor(double pu, double pv, const double* cf, double* scratch,
                             double* tX) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  double* Ls = scratch;          // [D + 1][n]: (1 - v)^m P_m((2u + v - 1) / (1 - v))
  double* Ps = Ls + (D + 1) * n;  // [n][n]: the Jacobi factor of basis index nm
  double* Ks = Ps + n * n;        // [n][n]: K_nm
  const double s0 = 2.0 * pu + pv - 1.0, q0 = 1.0 - pv, y0 = 1.0 - 2.0 * pv;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int e = lane; e < n; e += 32) Ls[e] = e == 0 ? 1.0 : 0.0;
    __syncwarp();
    // s = s0 + 2 du + dv, (1 - v)^2 = q0^2 - 2 q0 dv + dv^2, y = 1 - 2v = y0 - 2 dv
    for (int m = 1; m <= D; ++m) {
      const double* L1 = Ls + (m - 1) * n;
      const double* L2 = Ls + (m >= 2 ? m - 2 : 0) * n;
      for (int e = lane; e < n; e += 32) {
        int g, j;
        tri_split(e, g, j);
        double sL = s0 * L1[e];
        if (g - j >= 1) sL += 2.0 * L1[e - g];
        if (j >= 1) sL += L1[e - g - 1];
        double qL = 0.0;
        if (m >= 2) {
          qL = q0 * q0 * L2[e];
          if (j >= 1) qL -= 2.0 * q0 * L2[e - g - 1];
          if (j >= 2) qL += L2[e - 2 * g - 1];
        }
        Ls[m * n + e] = ((2.0 * m - 1.0) * sL - (m - 1.0) * qL) * (1.0 / m);
      }
      __syncwarp();
    }
#pragma unroll
    for (int m = 0; m <= D; ++m) {
      const int b = 2 * m + 1;
      double* P0 = Ps + (m * (m + 1) / 2 + m) * n;
      for (int e = lane; e < n; e += 32) P0[e] = e == 0 ? 1.0 : 0.0;
      __syncwarp();
#pragma unroll
      for (int a = 0; a < D - m; ++a) {
        double c1, c0, c2;
        jacobi_coef(a, b, &c1, &c0, &c2);
        const double* Pa = Ps + ((m + a) * (m + a + 1) / 2 + m) * n;
        const double* Pb = a > 0 ? Ps + ((m + a - 1) * (m + a) / 2 + m) * n : Pa;
        double* Pn = Ps + ((m + a + 1) * (m + a + 2) / 2 + m) * n;
        for (int e = lane; e < n; e += 32) {
          int g, j;
          tri_split(e, g, j);
          double v = (c1 * y0 + c0) * Pa[e];
          if (j >= 1) v -= 2.0 * c1 * Pa[e - g - 1];
          if (a > 0) v -= c2 * Pb[e];
          Pn[e] = v;
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < n * n; o += blockDim.x) {
    const int idx = o / n, e = o - idx * n;
    int nn, m, g, j;
    tri_split(idx, nn, m);
    tri_split(e, g, j);
    const int i = g - j;
    const double* L = Ls + m * n;
    const double* P = Ps + idx * n;
    double acc = 0.0;
    for (int ja = 0; ja <= j; ++ja)
      for (int ia = 0; ia <= i; ++ia) {
        const int ga = ia + ja, gb = g - ga, jb = j - ja;
        acc = fma(L[ga * (ga + 1) / 2 + ja], P[gb * (gb + 1) / 2 + jb], acc);
      }
    Ks[o] = c_kw[idx] * acc;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 3 * n; o += blockDim.x) {
    const int c = o / n, e = o - c * n;
    double acc = 0.0;
    if (e > 0)
      for (int idx = 0; idx < n; ++idx) acc = fma(cf[idx * 3 + c], Ks[idx * n + e], acc);
    tX[o] = acc;
  }
  __syncthreads();
}

// The chord dX(d) from the coefficients of chart_taylor: Horner in du inside Horner in dv.
template <int D>
__device__ __forceinline__ void chart_chord(const double* tX, double du, double dv, double* dX) {
  constexpr int n = (D + 1) * (D + 2) / 2;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double* t = tX + c * n;
    double acc = 0.0;
#pragma unroll
    for (int j = D; j >= 0; --j) {
      double in = 0.0;
#pragma unroll
      for (int i = D - j; i >= 0; --i) {
        const int g = i + j;
        in = fma(in, du, t[g * (g + 1) / 2 + j]);
      }
      acc = fma(acc, dv, in);
    }
    dX[c] = acc;
  }
}

// f(idx, K_nm, dK_nm/du, dK_nm/dv) for every basis function at (u, v): the recurrences of
// kw_geometry, for callers that need the derivatives one by one (the adjoint).
template <int D, class F>
__device__ __forceinline__ void kw_for_each(double u, double v, F&& f) {
  const double s = 2.0 * u + v - 1.0, q = 1.0 - v, q2 = q * q, y = 1.0 - 2.0 * v;
  double Lp = 0.0, L = 1.0, Lup = 0.0, Lu = 0.0, Lvp = 0.0, Lv = 0.0;
#pragma unroll
  for (int m = 0; m <= D; ++m) {
    if (m > 0) {
      const double f1 = 2.0 * m - 1.0, f2 = m - 1.0, im = 1.0 / m;
      const double Ln = (f1 * s * L - f2 * q2 * Lp) * im;
      const double Lun = (f1 * (2.0 * L + s * Lu) - f2 * q2 * Lup) * im;
      const double Lvn = (f1 * (L + s * Lv) - f2 * (-2.0 * q * Lp + q2 * Lvp)) * im;
      Lp = L;
      L = Ln;
      Lup = Lu;
      Lu = Lun;
      Lvp = Lv;
      Lv = Lvn;
    }
    const int b = 2 * m + 1;
    double Pp = 0.0, P = 1.0, dPp = 0.0, dP = 0.0;
#pragma unroll
    for (int a = 0; a <= D - m; ++a) {
      const int n = m + a, idx = n * (n + 1) / 2 + m;
      const double cn = c_kw[idx];
      f(idx, cn * L * P, cn * Lu * P, cn * (Lv * P - 2.0 * L * dP));
      if (a < D - m) {
        double c1, c0, c2;
        jacobi_coef(a, b, &c1, &c0, &c2);
        const double t = c1 * y + c0;
        const double Pn = t * P - c2 * Pp;
        const double dPn = c1 * P + t * dP - c2 * dPp;
        Pp = P;
        P = Pn;
        dPp = dP;
        dP = dPn;
      }
    }
  }
}

// Kernel times area element and weight, at a source with position X, weighted
// unnormalized normal Nw = (X_u x X_v) w and weighted Jacobian Jw = |X_u x X_v| w:
//   S: G_k(x, X) Jw
//   D: Nw.(x - X) (1 - ik r) e^{ikr} / (4 pi r^3)
//   CFIE: alpha D + beta S.
//   S': the D form with Nw replaced by -n_x Jw (nx: the target's unit normal).
// r = 0 contributes 0.
// With env != nullptr also the rounding envelope from the same r,
//   |G| Jw (|beta| + |alpha| |1 - ik r| R / r^2)   (kp.eb = |beta|, kp.ea = |alpha|),
// the size of the kernel value's rounding noise when positions carry errors of order u R
// (positions are relative to the patch centroid): the adaptive test never asks for less
// than a fixed multiple of its sum.
__device__ __forceinline__ cplx kernel_eval(const KernelParams& kp, double x0, double x1, double x2,
                                            double X0, double X1, double X2, double N0, double N1,
                                            double N2, double Jw, double R = 0.0,
                                            double* env = nullptr, const double* nx = nullptr) {
  if (kp.kind == 3) {  // S': the double-layer form with the source normal replaced by -n_x J
    N0 = -nx[0] * Jw;
    N1 = -nx[1] * Jw;
    N2 = -nx[2] * Jw;
  }
  const double d0 = x0 - X0, d1 = x1 - X1, d2 = x2 - X2;
  const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
  if (r2 == 0.0) {
    if (env) *env = 0.0;
    return {0.0, 0.0};
  }
  const double rinv = rsqrt(r2);
  const double r = r2 * rinv, rinv2 = rinv * rinv;
  const double th = kp.kr * r;
  double sn, cs;
  sincos(th, &sn, &cs);
  double ex = 0.07957747154594767 * rinv;  // 1/(4 pi r)
  if (kp.ki != 0.0) ex *= exp(-kp.ki * r);
  if (env) {
    // |G| Jw (|beta| + |alpha| |1 - ik r| R / r^2); |1 - ik r| only scales a floor, FP32 is ample
    const float f0 = (float)(1.0 + kp.ki * r), f1 = (float)th;
    const double fa = (double)sqrtf(f0 * f0 + f1 * f1);
    *env = ex * Jw * (kp.eb + kp.ea * fa * R * rinv2);
  }
  if (kp.kind == 0) return {ex * cs * Jw, ex * sn * Jw};  // G Jw
  // e^{ikr}/(4 pi r) times c: the double-layer factor (1 - ikr) (N.d)/r^2, with
  // k = kr + i ki so 1 - ikr = (1 + ki r) - i kr r; for the CFIE c = alpha c + beta Jw
  const double ndx = (N0 * d0 + N1 * d1 + N2 * d2) * rinv2;
  cplx c = {(1.0 + kp.ki * r) * ndx, -th * ndx};
  if (kp.kind == 2) {
    c = cmul({kp.ar, kp.ai}, c);
    c.re = fma(kp.br, Jw, c.re);
    c.im = fma(kp.bi, Jw, c.im);
  }
  return {ex * (cs * c.re - sn * c.im), ex * (cs * c.im + sn * c.re)};
}

// Kernel parameters converted to FP32 once per patch (the mixed form's pair evaluations).
struct KernelParamsF {
  float kr, ki, ar, ai, br, bi, eb, ea;
};
__device__ __forceinline__ KernelParamsF to_f32(const KernelParams& kp) {
  return {(float)kp.kr, (float)kp.ki, (float)kp.ar, (float)kp.ai,
          (float)kp.br, (float)kp.bi, (float)kp.eb, (float)kp.ea};
}

// Mixed form: K~ w in FP32 from the FP64 difference d = x - X and r2 = |d|^2; r (refined
// from the FP32 distance by one Newton step) and the phase k r (reduced mod 2 pi) are
// formed in FP64 first; 1/r, sin/cos of the reduced phase, the S and D factors and the
// CFIE combination are FP32.
// N, J: FP32 copies of the weighted normal and area element.  r2 > 0.
__device__ __forceinline__ float2 kernel_eval_f32f(const KernelParams& kp, const KernelParamsF& kf,
                                                   double d0, double d1, double d2, double r2,
                                                   float N0, float N1, float N2, float Jw,
                                                   float R, float* env) {
  const float fr2 = (float)r2;
  const float frinv = rsqrtf(fr2);
  const float fr = fr2 * frinv;
  const double r = (double)fr + (r2 - (double)fr * (double)fr) * (0.5 * (double)frinv);
  double th = kp.kr * r;
  th -= 6.283185307179586 * rint(th * 0.15915494309189535);
  float sn, cs;
  sincosf((float)th, &sn, &cs);
  float ex = 0.0795774715459f * frinv;
  if (kf.ki != 0.0f) ex *= expf(-kf.ki * fr);
  const float Gr = ex * cs, Gi = ex * sn;
  float ore = 0.0f, oim = 0.0f;
  if (kp.kind != 1) {
    const float sr = Gr * Jw, si = Gi * Jw;
    if (kp.kind == 0) {
      ore = sr;
      oim = si;
    } else {
      ore = kf.br * sr - kf.bi * si;
      oim = kf.br * si + kf.bi * sr;
    }
  }
  const float f0 = 1.0f + kf.ki * fr, f1 = -kf.kr * fr;
  if (kp.kind != 0) {
    const float ndx = (N0 * (float)d0 + N1 * (float)d1 + N2 * (float)d2) * frinv * frinv;
    float dr = (Gr * f0 - Gi * f1) * ndx, di = (Gr * f1 + Gi * f0) * ndx;
    if (kp.kind == 2) {
      const float tr = kf.ar * dr - kf.ai * di, ti = kf.ar * di + kf.ai * dr;
      dr = tr;
      di = ti;
    }
    ore += dr;
    oim += di;
  }
  if (env) {
    const float fa = sqrtf(f0 * f0 + f1 * f1);
    *env = ex * Jw * (kf.eb + kf.ea * fa * R * frinv * frinv);
  }
  return make_float2(ore, oim);
}


// Cross product helper.
// Derivatives of kernel_eval's K~(x, X, N) (N the unnormalized normal, no weight) with
// respect to the source position X and to N, for the adjoint.  With d = x - X, r = |d|,
// e = e^{ikr}, G = e/(4 pi r), h = (1 - ikr) e/(4 pi r^3):
//   S~ = G |N|:        dS~/dX = -G (ik - 1/r) |N| d/r,      dS~/dN = G N/|N|
//   D~ = h d.N:        dD~/dX = -h N - (d.N) h'(r) d/r,      dD~/dN = h d,
//                      h'(r) = e (k^2 r^2 + 3ikr - 3)/(4 pi r^4)
//   CFIE alpha D~ + beta S~.  Zero at r = 0 (as kernel_eval).  K~ is homogeneous of degree
// one in N, so with N scaled by a weight w, dX scales by w and dN is unchanged.
__device__ __forceinline__ void kernel_grad(const KernelParams& kp, const double* x,
                                            const double* X, const double* N, cplx* dX,
                                            cplx* dN) {
  const double d[3] = {x[0] - X[0], x[1] - X[1], x[2] - X[2]};
#pragma unroll
  for (int c = 0; c < 3; ++c) dX[c] = dN[c] = {0.0, 0.0};
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (r2 == 0.0) return;
  const double r = sqrt(r2), ir = 1.0 / r;
  double sn, cs;
  sincos(kp.kr * r, &sn, &cs);
  const double dec = exp(-kp.ki * r) * (0.25 / M_PI);
  const cplx e = {dec * cs, dec * sn};  // e^{ikr} / (4 pi)
  cplx cS = {0.0, 0.0}, cD = {0.0, 0.0};
  if (kp.kind == 0) cS = {1.0, 0.0};
  else if (kp.kind == 1) cD = {1.0, 0.0};
  else {
    cS = {kp.br, kp.bi};
    cD = {kp.ar, kp.ai};
  }
  if (cS.re != 0.0 || cS.im != 0.0) {
    const double nN = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    const cplx G = {e.re * ir, e.im * ir};
    const cplx a = cmul(cS, cmul(G, {-kp.ki - ir, kp.kr}));  // beta G (ik - 1/r)
    const double sa = nN * ir;
    const cplx b = cmul(cS, G);
    const double sb = nN > 0.0 ? 1.0 / nN : 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dX[c].re -= a.re * sa * d[c];
      dX[c].im -= a.im * sa * d[c];
      dN[c].re += b.re * sb * N[c];
      dN[c].im += b.im * sb * N[c];
    }
  }
  if (cD.re != 0.0 || cD.im != 0.0) {
    const double ir3 = ir * ir * ir;
    const cplx h0 = cmul({1.0 + kp.ki * r, -kp.kr * r}, e);
    const cplx h = cmul(cD, {h0.re * ir3, h0.im * ir3});
    const cplx poly = {(kp.kr * kp.kr - kp.ki * kp.ki) * r2 - 3.0 * kp.ki * r - 3.0,
                       2.0 * kp.kr * kp.ki * r2 + 3.0 * kp.kr * r};
    const cplx p0 = cmul(poly, e);
    const double ndx = N[0] * d[0] + N[1] * d[1] + N[2] * d[2];
    const double sp = ndx * ir3 * ir * ir;  // (d.N) / r^4 / r
    const cplx hp = cmul(cD, {p0.re * sp, p0.im * sp});
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dX[c].re -= h.re * N[c] + hp.re * d[c];
      dX[c].im -= h.im * N[c] + hp.im * d[c];
      dN[c].re += h.re * d[c];
      dN[c].im += h.im * d[c];
    }
  }
}

__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

}  // namespace lcq
