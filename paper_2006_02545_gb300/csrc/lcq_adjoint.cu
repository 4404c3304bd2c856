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

namespace lcq {
namespace {

__device__ __forceinline__ int patch_of_source(const int64_t* src_off, int64_t P, int64_t q) {
  int64_t lo = 0, hi = P;  // largest j with src_off[j] <= q
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    if (src_off[mid] <= q) lo = mid; else hi = mid;
  }
  return (int)lo;
}

// Koornwinder coefficients of the density in each patch's node slots: shat_j = V sigma_j.
template <int D>
__global__ void k_shat(const int* __restrict__ plist, int count, const int64_t* __restrict__ node_off,
                       const double* __restrict__ Vt, const cplx* __restrict__ sigma,
                       cplx* __restrict__ shat) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const int64_t off = node_off[plist[b]];
    for (int nm = threadIdx.x; nm < n; nm += blockDim.x) {
      double re = 0.0, im = 0.0;
      for (int l = 0; l < n; ++l) {
        re = fma(Vt[nm * n + l], sigma[off + l].re, re);
        im = fma(Vt[nm * n + l], sigma[off + l].im, im);
      }
      shat[off + nm] = {re, im};
    }
  }
}

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

// Block per patch: M_j = far-rule part (from tg) + annulus pairs (rule q_near), written.
template <int D>
__global__ void __launch_bounds__(kThreads) k_grad_rules(
    const int* __restrict__ plist, int count, Dev dv, const KernelParams kp,
    const int32_t* __restrict__ qn, const int64_t* __restrict__ src_off, int64_t n_over,
    const double* __restrict__ tg, const cplx* __restrict__ g, const cplx* __restrict__ shat_g,
    double* __restrict__ M) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  __shared__ double cf[3 * n];
  __shared__ cplx shat[n];
  __shared__ SegMap segs[1];
  __shared__ KernelParams kps;
  __shared__ double red[(kThreads / 32) * 3 * n];
  double Mg[3 * n];
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const int j = plist[b];
    const int64_t off = dv.node_off[j];
    __syncthreads();
    load_coef<D>(dv.coef, off, cf);
    for (int e = threadIdx.x; e < n; e += blockDim.x) shat[e] = shat_g[off + e];
    if (threadIdx.x == 0) {
      segs[0] = seg_T0();
      kps = patch_kp(dv, j, kp);
    }
    for (int e = threadIdx.x; e < 3 * n; e += blockDim.x) M[off * 3 + e] = 0.0;
#pragma unroll
    for (int e = 0; e < 3 * n; ++e) Mg[e] = 0.0;
    __syncthreads();
    // far rule q_j: node q of the rule is source src_off[j] + q
    const int m = dv.q[j], Q = m * m;
    const double* ru = dv.ru + dv.roff[m];
    const double* rv = dv.rv + dv.roff[m];
    const double* rw = dv.rw + dv.roff[m];
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
      const double u = ru[q], v = rv[q], w = rw[q];
      double X[3], Xu[3], Xv[3];
      kw_geometry<D>(u, v, cf, X, Xu, Xv, nullptr, 1);
      cplx sg = {0.0, 0.0};
      kw_for_each<D>(u, v, [&](int idx, double k0, double, double) {
        sg.re = fma(shat[idx].re, k0, sg.re);
        sg.im = fma(shat[idx].im, k0, sg.im);
      });
      const int64_t o = src_off[j] + q;
      double aX[3], aN[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double xr = tg[(2 * k) * n_over + o], xi = tg[(2 * k + 1) * n_over + o];
        const double nr = tg[(6 + 2 * k) * n_over + o], ni = tg[(6 + 2 * k + 1) * n_over + o];
        aX[k] = sg.re * xr - sg.im * xi;
        aN[k] = w * (sg.re * nr - sg.im * ni);
      }
      double bu[3], bv[3];
      cross3(Xv, aN, bu);
      cross3(aN, Xu, bv);
      kw_for_each<D>(u, v, [&](int idx, double k0, double ku, double kv) {
#pragma unroll
        for (int k = 0; k < 3; ++k) Mg[idx * 3 + k] += k0 * aX[k] + ku * bu[k] + kv * bv[k];
      });
    }
    // annulus pairs: one rule q_near on T0
    const int64_t a0 = dv.an_ptr[j], na = dv.an_ptr[j + 1] - a0;
    const int mn = qn[j];
    if (na > 0 && mn > 0) {
      const int32_t* pl = dv.an_pair + a0;
      TgtPairIdx ta{dv.tgt, dv.NT, dv.pair_tgt, pl, dv.tnrm};
      block_grad<D>(cf, dv.ru + dv.roff[mn], dv.rv + dv.roff[mn], dv.rw + dv.roff[mn], mn * mn,
                    segs, 1, ta, (int)na,
                    [&](int i) -> cplx {
                      const cplx c = g[dv.pair_tgt[pl[i]]];
                      return {c.re, -c.im};
                    },
                    kps, shat, dv.cen + 3 * j, Mg);
    }
    block_reduce_M<D>(Mg, red, M + off * 3);
  }
}

// dL/dy_l = sum_nm V_nm,l M_nm per patch, into out SoA [3][N].
template <int D>
__global__ void k_grad_v2c(const int* __restrict__ plist, int count, const int64_t* __restrict__ node_off,
                           const double* __restrict__ Vt, const double* __restrict__ M, int64_t N,
                           double* __restrict__ out) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const int64_t off = node_off[plist[b]];
    for (int e = threadIdx.x; e < 3 * n; e += blockDim.x) {
      const int l = e / 3, c = e - 3 * l;
      double acc = 0.0;
      for (int nm = 0; nm < n; ++nm) acc = fma(Vt[nm * n + l], M[(off + nm) * 3 + c], acc);
      out[c * N + off + l] = acc;
    }
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

// A^H per patch: out_l = (V^T K z)_l over the rule q_j, plus conj(c) g over the patch's
// near pairs and self pairs in patch-major order (deterministic, no atomics), plus
// jump * g_t at the node of each on-surface target t.
template <int D>
__global__ void k_adj_patch(const int* __restrict__ plist, int count, Dev dv,
                            const double* __restrict__ Vt, const int64_t* __restrict__ src_off,
                            const cplx* __restrict__ z, const double* __restrict__ val,
                            const cplx* __restrict__ g, double jump, cplx* __restrict__ out) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  __shared__ cplx kz[n];
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const int j = plist[b];
    const int64_t off = dv.node_off[j];
    const int m = dv.q[j], Q = m * m;
    const double* ru = dv.ru + dv.roff[m];
    const double* rv = dv.rv + dv.roff[m];
    __syncthreads();
    // (K z)_nm: thread per basis function, nodes in order
    for (int nm = threadIdx.x; nm < n; nm += blockDim.x) {
      double re = 0.0, im = 0.0;
      for (int q = 0; q < Q; ++q) {
        double K[n];
        kw_values<D>(ru[q], rv[q], K, 1);
        const cplx zq = z[src_off[j] + q];
        re = fma(K[nm], zq.re, re);
        im = fma(K[nm], zq.im, im);
      }
      kz[nm] = {re, im};
    }
    __syncthreads();
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      double re = 0.0, im = 0.0;
      for (int nm = 0; nm < n; ++nm) {
        re = fma(Vt[nm * n + l], kz[nm].re, re);
        im = fma(Vt[nm * n + l], kz[nm].im, im);
      }
      for (int64_t p = dv.pair_ptr[j]; p < dv.pair_ptr[j + 1]; ++p) {
        const int64_t e = dv.pair_csr[p] + l;
        const cplx gt = g[dv.pair_tgt[p]];
        const double vr = val[2 * e], vi = val[2 * e + 1];
        re += vr * gt.re + vi * gt.im;
        im += vr * gt.im - vi * gt.re;
      }
      for (int64_t p = dv.self_ptr[j]; p < dv.self_ptr[j + 1]; ++p) {
        const int64_t e = dv.self_csr[p] + l;
        const int t = dv.self_tgt[p];
        const cplx gt = g[t];
        const double vr = val[2 * e], vi = val[2 * e + 1];
        re += vr * gt.re + vi * gt.im;
        im += vr * gt.im - vi * gt.re;
        if (dv.tlnode[t] == l) {  // the jump term jump * sigma(x_t) of apply
          re += jump * gt.re;
          im += jump * gt.im;
        }
      }
      out[off + l] = {re, im};
    }
  }
}

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

int grid_of(const LaunchCommon& lc, int count) {
  return count < 2 * lc.num_sms ? (count > 0 ? count : 1) : 2 * lc.num_sms;
}

template <int D>
struct ShatL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                  const double* Vt, const void* sigma, void* shat) {
    ++*lc.launches;
    k_shat<D><<<grid_of(lc, count), 64, 0, lc.stream>>>(plist, count, node_off, Vt,
                                                        (const cplx*)sigma, (cplx*)shat);
  }
};

template <int D>
struct GradRulesL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, const int32_t* qn, const int64_t* src_off, int64_t n_over,
                  const double* tg, const void* g, const void* shat, double* M) {
    ++*lc.launches;
    k_grad_rules<D><<<grid_of(lc, count), kThreads, 0, lc.stream>>>(
        plist, count, dv, kp, qn, src_off, n_over, tg, (const cplx*)g, (const cplx*)shat, M);
  }
};

template <int D>
struct AdaptiveGradL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, double eps, double normV, int leaf_order, int max_depth,
                  const void* I_smooth, void* I_near, int32_t* leaves, void* work, int64_t stride,
                  int A_max, int levels, int grid, int* status, int* sched, double mix,
                  const GradArgs& ga) {
    const size_t sm = adaptive_smem_bytes<D>();
    cudaFuncSetAttribute(k_adaptive<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    AdaptiveWS w{stride, A_max, levels};
    cudaMemsetAsync(sched, 0, sizeof(int), lc.stream);
    ++*lc.launches;
    k_adaptive<D, true><<<grid, kThreads, sm, lc.stream>>>(
        plist, count, dv, kp, eps, normV, leaf_order, max_depth, (const cplx*)I_smooth,
        (cplx*)I_near, leaves, (unsigned char*)work, w, status, sched, mix, ga, nullptr, 0);
  }
};

template <int D>
struct GradV2cL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                  const double* Vt, const double* M, int64_t N, double* out) {
    ++*lc.launches;
    k_grad_v2c<D><<<grid_of(lc, count), 128, 0, lc.stream>>>(plist, count, node_off, Vt, M, N,
                                                             out);
  }
};

template <int D>
struct AdjPatchL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const double* Vt, const int64_t* src_off, const void* z, const double* val,
                  const void* g, double jump, void* out) {
    ++*lc.launches;
    k_adj_patch<D><<<grid_of(lc, count), 64, 0, lc.stream>>>(plist, count, dv, Vt, src_off,
                                                             (const cplx*)z, val, (const cplx*)g,
                                                             jump, (cplx*)out);
  }
};

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
                          int grid, int* status, int* sched, double mix, const GradArgs& ga) {
  return dispatch<AdaptiveGradL>(d, lc, plist, count, dv, kp, eps, normV, leaf_order, max_depth,
                                 I_smooth, I_near, leaves, work, stride, A_max, levels, grid,
                                 status, sched, mix, ga);
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
