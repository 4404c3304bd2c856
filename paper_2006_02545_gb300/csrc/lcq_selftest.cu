// Device self-checks of the adaptive kernel's arithmetic building blocks (no counterpart in
// the paper): the table-driven sincos against CUDA's sincos, and the split-precision
// tensor-core contraction against a plain FP64 contraction of the same operands.
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
      cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), st) != cudaSuccess ||
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
    unsigned long long h[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      status = LCQ_ERR_CUDA;
    } else {
      // [0] max |sincos_tab - sincos| over sin and cos; [1] D = 6 and [2] D = 10: max
      // |tensor-core - FP64| / sum |a| |b| over every output
      for (int i = 0; i < 3 && i < n_out; ++i) memcpy(&out[i], &h[i], sizeof(double));
    }
  }
  if (d) cudaFree(d);
  if (st) cudaStreamDestroy(st);
  cudaGetLastError();
  cudaSetDevice(prev);
  return status;
}
