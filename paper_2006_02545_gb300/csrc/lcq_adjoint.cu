// Adjoint of the corrected layer potential (an extension; the paper has no gradients).
//
// u = A(y) sigma at the targets (Sec. 5.3: far sum over the smooth rules q_j plus the
// CSR corrections).  For a real functional L with upstream gradient g = dL/d(conj u):
//   density:      A^H g = far transposed sum + conj(CSR)^T g            (k_far_sum_T,
//                 k_adj_patch)
//   coordinates:  dL/dy with every discrete choice frozen (near lists, q_j, annulus
//                 orders, refinement trees).  For an off-surface target each pair (t, j)
//                 contributes through exactly one rule: q_j (far pair), the annulus rule,
//                 or the accepted leaves of its tree (adaptive pair; the stored a - s plus
//                 the far term's s leaves a).  The trees are not stored: the union-tree
//                 kernel runs again in its gradient mode and differentiates at every
//                 accepted node (k_adaptive<D, true>).  Only X and N = X_u x X_v depend on
//                 y, through the chart coefficients x = V y; the moments dL/dx_nm collect
//                 in M and k_grad_v2c maps them to the nodes, dL/dy_l = sum_nm V_nm,l M_nm.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lcq_common.cuh"
#include "lcq_degree.h"

namespace lcq {

// Far sources' share of the coordinate gradient, thread per source q of patch j: over the
// targets t of q's surface that are neither on patch j nor near it (the same FP64 test as
// the near lists),
//   TX_q = sum_t conj(g_t) dK~/dX (x_t, X_q, N_q w_q),  TN_q = sum_t conj(g_t) dK~/dN (...).
// Output tg[12][n_over]: Re/Im of TX (3) then of TN (3).
__global__ void __launch_bounds__(kThreads) k_far_grad_sum(
    Dev dv, int64_t P, const double* __restrict__ src, int64_t n_over,
    const int64_t* __restrict__ src_off, const KernelParams kp, const int32_t* __restrict__ tgroup,
    const cplx* __restrict__ g, double* __restrict__ tg) {
  __shared__ double sx[3][kThreads];
  __shared__ cplx sgw[kThreads];
  __shared__ int stp[kThreads], sgr[kThreads];
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool on = q < n_over;
  int j = 0, grp = 0;
  double X[3] = {0, 0, 0}, Nw[3] = {0, 0, 0}, c[3] = {0, 0, 0}, rr = 0.0;
  KernelParams kq = kp;
  if (on) {
    j = patch_of_source(src_off, P, q);
    for (int k = 0; k < 3; ++k) {
      X[k] = src[k * n_over + q];
      Nw[k] = src[(3 + k) * n_over + q];
      c[k] = dv.cen[3 * j + k];
    }
    const double r = dv.eta[j] * dv.rad[j];
    rr = r * r;
    if (dv.pgroup) {
      grp = dv.pgroup[j];
      kq = dv.grp[grp].kp;
    }
  }
  cplx TX[3] = {{0, 0}, {0, 0}, {0, 0}}, TN[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int64_t t0 = 0; t0 < dv.NT; t0 += kThreads) {
    __syncthreads();
    const int64_t t = t0 + threadIdx.x;
    if (t < dv.NT) {
      for (int k = 0; k < 3; ++k) sx[k][threadIdx.x] = dv.tgt[k * dv.NT + t];
      const cplx gv = g[t];
      sgw[threadIdx.x] = {gv.re, -gv.im};
      stp[threadIdx.x] = dv.tpatch[t];
      sgr[threadIdx.x] = tgroup ? tgroup[t] : 0;
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kThreads, dv.NT - t0);
    if (on)
      for (int i = 0; i < cnt; ++i) {
        if (stp[i] == j || sgr[i] != grp) continue;
        const double x[3] = {sx[0][i], sx[1][i], sx[2][i]};
        const double e0 = x[0] - c[0], e1 = x[1] - c[1], e2 = x[2] - c[2];
        if (e0 * e0 + e1 * e1 + e2 * e2 <= rr) continue;  // near pair: its own rule
        cplx dX[3], dN[3];
        kernel_grad(kq, x, X, Nw, dX, dN);
        const cplx w = sgw[i];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const cplx a = cmul(w, dX[k]), b = cmul(w, dN[k]);
          TX[k].re += a.re;
          TX[k].im += a.im;
          TN[k].re += b.re;
          TN[k].im += b.im;
        }
      }
  }
  if (on)
    for (int k = 0; k < 3; ++k) {
      tg[(2 * k) * n_over + q] = TX[k].re;
      tg[(2 * k + 1) * n_over + q] = TX[k].im;
      tg[(6 + 2 * k) * n_over + q] = TN[k].re;
      tg[(6 + 2 * k + 1) * n_over + q] = TN[k].im;
    }
}

// A^H, far part: z_q = sum_t conj(K~w(x_t, X_q)) g_t over the targets of q's surface not on
// q's patch (the far sum of apply includes near pairs; their smooth-rule term is part of A).
__global__ void __launch_bounds__(kThreads) k_far_sum_T(
    Dev dv, int64_t P, const double* __restrict__ src, int64_t n_over,
    const int64_t* __restrict__ src_off, const KernelParams kp, const int32_t* __restrict__ tgroup,
    const cplx* __restrict__ g, cplx* __restrict__ z) {
  __shared__ double sx[3][kThreads];
  __shared__ cplx sg[kThreads];
  __shared__ int stp[kThreads], sgr[kThreads];
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool on = q < n_over;
  int j = 0, grp = 0;
  double s[7] = {0, 0, 0, 0, 0, 0, 0};
  KernelParams kq = kp;
  if (on) {
    j = patch_of_source(src_off, P, q);
    for (int k = 0; k < 7; ++k) s[k] = src[k * n_over + q];
    if (dv.pgroup) {
      grp = dv.pgroup[j];
      kq = dv.grp[grp].kp;
    }
  }
  double re = 0.0, im = 0.0;
  for (int64_t t0 = 0; t0 < dv.NT; t0 += kThreads) {
    __syncthreads();
    const int64_t t = t0 + threadIdx.x;
    if (t < dv.NT) {
      for (int k = 0; k < 3; ++k) sx[k][threadIdx.x] = dv.tgt[k * dv.NT + t];
      sg[threadIdx.x] = g[t];
      stp[threadIdx.x] = dv.tpatch[t];
      sgr[threadIdx.x] = tgroup ? tgroup[t] : 0;
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kThreads, dv.NT - t0);
    if (on)
      for (int i = 0; i < cnt; ++i) {
        if (stp[i] == j || sgr[i] != grp) continue;
        const int64_t tt = t0 + i;
        const double nx[3] = {dv.tnrm ? dv.tnrm[tt] : 0.0, dv.tnrm ? dv.tnrm[dv.NT + tt] : 0.0,
                              dv.tnrm ? dv.tnrm[2 * dv.NT + tt] : 0.0};
        const cplx k = kernel_eval(kq, sx[0][i], sx[1][i], sx[2][i], s[0], s[1], s[2], s[3], s[4],
                                   s[5], s[6], 0.0, nullptr, nx);
        // conj(k) * g
        re += k.re * sg[i].re + k.im * sg[i].im;
        im += k.re * sg[i].im - k.im * sg[i].re;
      }
  }
  if (on) z[q] = {re, im};
}

namespace {
template <template <int> class F, class... Args>
bool dispatch(int d, Args&&... args) {
  switch (d) {
#define LCQ_CASE(D) \
  case D: F<D>::run(args...); return true;
    LCQ_CASE(1) LCQ_CASE(2) LCQ_CASE(3) LCQ_CASE(4) LCQ_CASE(5)
    LCQ_CASE(6) LCQ_CASE(7) LCQ_CASE(8) LCQ_CASE(9) LCQ_CASE(10)
#undef LCQ_CASE
    default: return false;
  }
}
}  // namespace

cudaError_t upload_constants_adjoint(cudaStream_t st) {
  const cudaError_t e = upload_kw_tables(st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

bool launch_shat(int d, const LaunchCommon& lc, const int* plist, int count,
                 const int64_t* node_off, const double* Vt, const void* sigma, void* shat) {
  return dispatch<ShatL>(d, lc, plist, count, node_off, Vt, sigma, shat);
}

void launch_far_grad_sum(const LaunchCommon& lc, const Dev& dv, int64_t P, const double* src,
                         int64_t n_over, const int64_t* src_off, const KernelParams& kp,
                         const int32_t* tgroup, const void* g, double* tg) {
  const int64_t b = (n_over + kThreads - 1) / kThreads;
  if (b <= 0) return;
  ++*lc.launches;
  k_far_grad_sum<<<(unsigned)b, kThreads, 0, lc.stream>>>(dv, P, src, n_over, src_off, kp, tgroup,
                                                          (const cplx*)g, tg);
}

bool launch_grad_rules(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                       const KernelParams& kp, const int32_t* qn, const int64_t* src_off,
                       int64_t n_over, const double* tg, const void* g, const void* shat,
                       double* M) {
  return dispatch<GradRulesL>(d, lc, plist, count, dv, kp, qn, src_off, n_over, tg, g, shat, M);
}

bool launch_adaptive_grad(int d, const LaunchCommon& lc, const int* plist, int count,
                          const Dev& dv, const KernelParams& kp, double eps, double normV,
                          int leaf_order, int max_depth, const void* I_smooth, void* I_near,
                          int32_t* leaves, void* work, int64_t stride, int A_max, int levels,
                          int grid, int* status, int* sched, int form, const GradArgs& ga) {
  return dispatch<AdaptiveGradL>(d, lc, plist, count, dv, kp, eps, normV, leaf_order, max_depth,
                                 I_smooth, I_near, leaves, work, stride, A_max, levels, grid,
                                 status, sched, form, ga);
}

bool launch_grad_v2c(int d, const LaunchCommon& lc, const int* plist, int count,
                     const int64_t* node_off, const double* Vt, const double* M, int64_t N,
                     double* out) {
  return dispatch<GradV2cL>(d, lc, plist, count, node_off, Vt, M, N, out);
}

void launch_far_sum_T(const LaunchCommon& lc, const Dev& dv, int64_t P, const double* src,
                      int64_t n_over, const int64_t* src_off, const KernelParams& kp,
                      const int32_t* tgroup, const void* g, void* z) {
  const int64_t b = (n_over + kThreads - 1) / kThreads;
  if (b <= 0) return;
  ++*lc.launches;
  k_far_sum_T<<<(unsigned)b, kThreads, 0, lc.stream>>>(dv, P, src, n_over, src_off, kp, tgroup,
                                                       (const cplx*)g, (cplx*)z);
}

bool launch_adj_patch(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                      const double* Vt, const int64_t* src_off, const void* z, const double* val,
                      const void* g, double jump, void* out) {
  return dispatch<AdjPatchL>(d, lc, plist, count, dv, Vt, src_off, z, val, g, jump, out);
}

}  // namespace lcq

