// Device self-checks of the adaptive kernel's arithmetic building blocks (no counterpart in
// the paper): the table-driven sincos against CUDA's sincos, the split-precision
// tensor-core contraction against a plain FP64 contraction of the same operands, and the
// two-float kernel value and sincos against their FP64 counterparts.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "lcq.h"
#include "lcq_common.cuh"

namespace lcq {
namespace {

// largest |a - b| seen, as the bit pattern of a non-negative double (monotone in its value)
__device__ __forceinline__ void max_into(unsigned long long* slot, double v) {
  atomicMax(slot, (unsigned long long)__double_as_longlong(fabs(v)));
}

// Arguments: a uniform spread over [-lim, lim] plus points just around multiples of
// 2 pi / 1024 (the table's breakpoints).
__global__ void k_check_sincos(int64_t count, double lim, unsigned long long* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    double th;
    if (i & 1) {
      const int64_t j = (i >> 1) % 20000 - 10000;
      th = j * (6.283185307179586 / kSinCosTable) + ((i >> 2) % 7 - 3) * 1e-9;
    } else {
      th = -lim + 2.0 * lim * ((double)(i >> 1) / (double)(count / 2 + 1));
    }
    double s1, c1, s2, c2;
    sincos_tab(th, g_sct, &s1, &c1);
    sincos(th, &s2, &c2);
    max_into(out, s1 - s2);
    max_into(out, c1 - c2);
  }
}

// One block: random complex rows (8 targets, magnitudes over 12 decades, random signs) and
// basis-like columns bounded by 2^E_nm, nq nodes padded to ncp; the tensor-core result of
// each (target, nm) against a double-double sum, relative to sum_q |a_q| |b_q|.
template <int D>
__global__ void __launch_bounds__(256) k_check_tc(int nq, unsigned long long seed,
                                                  unsigned long long* out) {
  using C = TcCfg<D>;
  constexpr int n = C::n;
  extern __shared__ __align__(128) unsigned char smb[];
  uint16_t* Bsl = reinterpret_cast<uint16_t*>(smb + C::OFF_BS);
  cplx* Gs = reinterpret_cast<cplx*>(smb + C::OFF_G);
  uint16_t* Asl = reinterpret_cast<uint16_t*>(smb + C::OFF_G);
  int* rowE = reinterpret_cast<int*>(smb + C::OFF_ROWE);
  __shared__ cplx A0[C::TT][C::CH];
  __shared__ double Bref[C::CH][n];
  __shared__ cplx res[C::TT][n];
  const int ncp = (nq + 15) & ~15;
  auto rnd = [&](unsigned long long k) {  // splitmix64 of (seed, k) -> [0, 1)
    unsigned long long z = seed + 0x9e3779b97f4a7c15ull * (k + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int e = threadIdx.x; e < C::CH * C::NP; e += blockDim.x) {
    const int q = e / C::NP, nm = e - q * C::NP;
    double b = 0.0;
    if (q < nq && nm < n) b = (2.0 * rnd(4 * e) - 1.0) * ldexp(1.0, c_kwexp[nm]) * rnd(4 * e + 1);
    if (nm < n) {
      Bref[q][nm] = b;
      store_basis_slices<D>(Bsl, nm, q, b);
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) Bsl[(size_t)i * C::NP * C::CH + C::swz(nm, q)] = 0;
    }
  }
  for (int e = threadIdx.x; e < C::TT * C::CH; e += blockDim.x) {
    const int t = e / C::CH, q = e - t * C::CH;
    cplx a = {0.0, 0.0};
    if (q < nq) {
      const double mag = pow(10.0, 12.0 * rnd(1000003 + 3 * e) - 6.0);
      const double ang = 6.283185307179586 * rnd(1000003 + 3 * e + 1);
      a = {mag * cos(ang), mag * sin(ang)};
    }
    A0[t][q] = a;
    Gs[t * C::CH + q] = a;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int VPL = C::CH / 32;
  const int q0 = lane * VPL;
  double re[VPL], im[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const cplx g = (q0 + v < ncp) ? Gs[warp * C::CH + q0 + v] : cplx{0.0, 0.0};
    re[v] = g.re;
    im[v] = g.im;
  }
  __syncthreads();
  split_row_pair<D, 8, VPL>(re, im, true, Asl, warp, q0, rowE);
  __syncthreads();
  for (int ct = warp; ct < C::NTILE; ct += blockDim.x >> 5)
    tc_tile<D, 8, 9>(Bsl, Asl, rowE, ct, 0, ncp, C::TT, 0, 0, true,
                     [&](int t) { return &res[t][0]; });
  __syncthreads();
  for (int e = threadIdx.x; e < C::TT * n; e += blockDim.x) {
    const int t = e / n, nm = e - t * n;
    // reference sums in double-double (Dekker's product by FMA, Knuth's two-sum), so that
    // the measured difference is the tensor-core path's own error
    double sr = 0.0, lr = 0.0, si = 0.0, li = 0.0, sa = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double b = Bref[q][nm];
      const double pr = A0[t][q].re * b, er = fma(A0[t][q].re, b, -pr);
      const double pi = A0[t][q].im * b, ei = fma(A0[t][q].im, b, -pi);
      double s2 = sr + pr, z = s2 - sr;
      lr += (sr - (s2 - z)) + (pr - z) + er;
      sr = s2;
      s2 = si + pi;
      z = s2 - si;
      li += (si - (s2 - z)) + (pi - z) + ei;
      si = s2;
      sa = fma(hypot(A0[t][q].re, A0[t][q].im), fabs(b), sa);
    }
    if (sa > 0.0) {
      max_into(out, ((res[t][nm].re - sr) - lr) / sa);
      max_into(out, ((res[t][nm].im - si) - li) / sa);
    }
  }
}

// Two-float kernel values (kernel_eval_ff) against the FP64 ones (kernel_eval_fold) at the
// same inputs: sources |X| <= 0.3, targets at 10^-4 .. 1 of that in random directions (half
// in the source's tangent plane), random weighted normals and folded constants, k in
// {1.3, 2 pi, 20} and kinds S, D and CFIE; the difference relative to the sum of the
// magnitudes of the terms (|e^{ikr}/r| (|N'| (1 + k r) / r + |Js| + |Ks|)), out[0]; and
// the two-float sincos against sincos over |th| < 3000, relative to 1 + |th|, out[1].
__global__ void k_check_ff(int64_t count, unsigned long long* out) {
  auto rnd = [](unsigned long long k) {  // splitmix64 of k -> [0, 1)
    unsigned long long z = 0x9e3779b97f4a7c15ull * (k + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = 64ull * (unsigned long long)i;
    double X[3], N[3], u[3];
    for (int c = 0; c < 3; ++c) {
      X[c] = 0.3 * (2.0 * rnd(b + c) - 1.0);
      N[c] = 2.0 * rnd(b + 3 + c) - 1.0;
      u[c] = 2.0 * rnd(b + 6 + c) - 1.0;
    }
    const double nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    if (i & 1) {  // tangent plane of the source
      const double t = (u[0] * N[0] + u[1] * N[1] + u[2] * N[2]) / (nn * nn);
      for (int c = 0; c < 3; ++c) u[c] -= t * N[c];
    }
    const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double dist = 0.3 * pow(10.0, -4.0 * rnd(b + 9));
    double x[3];
    for (int c = 0; c < 3; ++c) x[c] = X[c] + dist * u[c] / un;
    const double ks[3] = {1.3, 6.283185307179586, 20.0};
    const double kr = ks[(i >> 1) % 3];
    const int kind = (int)((i >> 3) % 3);
    const double w = 0.01 + rnd(b + 10);
    const double Js = kind == 0 ? w * 0.0795 : (kind == 2 ? 0.7 * w * 0.0795 : 0.0);
    const double Ks = kind == 2 ? -kr * w * 0.0795 : 0.0;
    const double Np[3] = {N[0] * w * 0.0795, N[1] * w * 0.0795, N[2] * w * 0.0795};
    const KernelParamsF kf = {(float)kr, 0.0f, 1.0f, 0.0f, 0.7f, 0.0f, 1.0f, 1.0f};
    const ff Nf[3] = {ff_of(Np[0]), ff_of(Np[1]), ff_of(Np[2])};
    float e1 = 0.0f, e2 = 0.0f;
    const cplx g64 = kernel_eval_fold(kind, kr, kf, g_sct, x[0], x[1], x[2], X[0], X[1], X[2],
                                      Np[0], Np[1], Np[2], Js, Ks, 1.0f, 0.3f, &e1);
    const cplx gff = kernel_eval_ff(kind, kr, ff_of(kr), kf, g_sct, g_sctf, x[0], x[1], x[2], X[0],
                                    X[1], X[2], Nf, ff_of(Js), ff_of(Ks), 1.0f, 0.3f, &e2);
    const double r = sqrt((x[0] - X[0]) * (x[0] - X[0]) + (x[1] - X[1]) * (x[1] - X[1]) +
                          (x[2] - X[2]) * (x[2] - X[2]));
    const double nq = sqrt(Np[0] * Np[0] + Np[1] * Np[1] + Np[2] * Np[2]);
    const double mag = (kind == 0 ? 0.0 : nq * (1.0 + kr * r) / r) + fabs(Js) + fabs(Ks);
    const double scale = mag / r;
    max_into(out, fmax(fabs(gff.re - g64.re), fabs(gff.im - g64.im)) / scale);
    // sincos over |th| < 3000
    const double th = 3000.0 * (2.0 * rnd(b + 11) - 1.0);
    ff sn, cs;
    if (ff_sincos(ff_of(th), g_sctf, &sn, &cs)) {
      double s2, c2;
      sincos(th, &s2, &c2);
      const double e = fmax(fabs(dbl_of(sn) - s2), fabs(dbl_of(cs) - c2)) / (1.0 + fabs(th));
      max_into(out + 1, e);
    } else {
      max_into(out + 1, 1.0);  // |th| < 2^14 must be in range
    }
  }
}

}  // namespace
}  // namespace lcq

using namespace lcq;

extern "C" lcq_status lcq_selftest(int device, double* out, int n_out) {
  if (!out || n_out < 1) return LCQ_ERR_ARG;
  for (int i = 0; i < n_out; ++i) out[i] = -1.0;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return LCQ_ERR_CUDA;
  }
  lcq_status status = LCQ_OK;
  unsigned long long* d = nullptr;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&d, 8 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemsetAsync(d, 0, 8 * sizeof(unsigned long long), st) != cudaSuccess ||
      upload_kw_tables(st) != cudaSuccess)
    status = LCQ_ERR_CUDA;
  if (status == LCQ_OK) {
    k_check_sincos<<<256, 256, 0, st>>>(int64_t(1) << 22, 3000.0, d);
    using C6 = TcCfg<6>;
    const int sm6 = C6::BYTES;
    cudaFuncSetAttribute(k_check_tc<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm6);
    k_check_tc<6><<<1, 256, sm6, st>>>(100, 12345ull, d + 1);
    k_check_tc<6><<<1, 256, sm6, st>>>(128, 777ull, d + 1);
    using C10 = TcCfg<10>;
    const int sm10 = C10::BYTES;
    cudaFuncSetAttribute(k_check_tc<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm10);
    k_check_tc<10><<<1, 256, sm10, st>>>(49, 4242ull, d + 2);
    k_check_ff<<<256, 256, 0, st>>>(int64_t(1) << 21, d + 3);
    unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      status = LCQ_ERR_CUDA;
    } else {
      // [0] max |sincos_tab - sincos| over sin and cos; [1] D = 6 and [2] D = 10: max
      // |tensor-core - FP64| / sum |a| |b| over every output; [3] two-float kernel values
      // against FP64 ones relative to the magnitude of their terms; [4] two-float sincos
      // against sincos relative to 1 + |th|
      for (int i = 0; i < 5 && i < n_out; ++i) memcpy(&out[i], &h[i], sizeof(double));
    }
  }
  if (d) cudaFree(d);
  if (st) cudaStreamDestroy(st);
  cudaGetLastError();
  cudaSetDevice(prev);
  return status;
}
