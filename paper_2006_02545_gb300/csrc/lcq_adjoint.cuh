// Degree-templated kernels and launchers of the adjoint (lcq_adjoint.cu has the overview),
// instantiated one patch degree per translation unit in lcq_deg.cu.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lcq_kernels.cuh"

namespace lcq {


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


// Block per patch: M_j = far-rule part (from tg) + annulus pairs (rule q_near), written.
// Each warp sums its nodes' contributions into its own row of `red` (warp sums in a fixed
// order, no per-thread gradient row); the rows are added in warp order at the end.
template <int D>
__global__ void __launch_bounds__(kThreads) k_grad_rules(
    const int* __restrict__ plist, int count, Dev dv, const KernelParams kp,
    const int32_t* __restrict__ qn, const int64_t* __restrict__ src_off, int64_t n_over,
    const double* __restrict__ tg, const cplx* __restrict__ g, const cplx* __restrict__ shat_g,
    double* __restrict__ M) {
  constexpr int n = (D + 1) * (D + 2) / 2, n3 = 3 * n, nwarps = kThreads / 32;
  __shared__ double cf[3 * n];
  __shared__ cplx shat[n];
  __shared__ SegMap segs[1];
  __shared__ KernelParams kps;
  __shared__ double red[nwarps * n3];
  double* Mw = red + (threadIdx.x >> 5) * n3;
  const bool lead = (threadIdx.x & 31) == 0;
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
    for (int e = threadIdx.x; e < nwarps * n3; e += blockDim.x) red[e] = 0.0;
    __syncthreads();
    // far rule q_j: node q of the rule is source src_off[j] + q; every lane runs the same
    // number of passes (zeros where q >= Q) so that the warp sums see all 32 lanes
    const int m = dv.q[j], Q = m * m;
    const double* ru = dv.ru + dv.roff[m];
    const double* rv = dv.rv + dv.roff[m];
    const double* rw = dv.rw + dv.roff[m];
    for (int q0 = 0; q0 < Q; q0 += blockDim.x) {
      const int q = q0 + threadIdx.x;
      double u = 0.0, v = 0.0;
      double X[3] = {0, 0, 0}, Xu[3] = {0, 0, 0}, Xv[3] = {0, 0, 0};
      double aX[3] = {0, 0, 0}, aN[3] = {0, 0, 0};
      if (q < Q) {
        u = ru[q];
        v = rv[q];
        const double w = rw[q];
        kw_geometry<D>(u, v, cf, X, Xu, Xv, nullptr, 1);
        cplx sg = {0.0, 0.0};
        kw_for_each<D>(u, v, [&](int idx, double k0, double, double) {
          sg.re = fma(shat[idx].re, k0, sg.re);
          sg.im = fma(shat[idx].im, k0, sg.im);
        });
        const int64_t o = src_off[j] + q;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double xr = tg[(2 * k) * n_over + o], xi = tg[(2 * k + 1) * n_over + o];
          const double nr = tg[(6 + 2 * k) * n_over + o], ni = tg[(6 + 2 * k + 1) * n_over + o];
          aX[k] = sg.re * xr - sg.im * xi;
          aN[k] = w * (sg.re * nr - sg.im * ni);
        }
      }
      double bu[3], bv[3];
      cross3(Xv, aN, bu);
      cross3(aN, Xu, bv);
      kw_for_each<D>(u, v, [&](int idx, double k0, double ku, double kv) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double s = warp_sum(k0 * aX[k] + ku * bu[k] + kv * bv[k]);
          if (lead) Mw[idx * 3 + k] += s;
        }
      });
    }
    // annulus pairs: one rule q_near on T0
    const int64_t a0 = dv.an_ptr[j], na = dv.an_ptr[j + 1] - a0;
    const int mn = qn[j];
    if (na > 0 && mn > 0) {
      const int32_t* pl = dv.an_pair + a0;
      TgtPairIdx ta{dv.tgt, dv.NT, dv.pair_tgt, pl, dv.tnrm};
      block_grad<D, true>(cf, dv.ru + dv.roff[mn], dv.rv + dv.roff[mn], dv.rw + dv.roff[mn],
                          mn * mn, segs, 1, ta, (int)na,
                          [&](int i) -> cplx {
                            const cplx c = g[dv.pair_tgt[pl[i]]];
                            return {c.re, -c.im};
                          },
                          kps, shat, dv.cen + 3 * j, Mw);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n3; e += blockDim.x) {
      double acc = 0.0;
      for (int wp = 0; wp < nwarps; ++wp) acc += red[wp * n3 + e];
      M[off * 3 + e] = acc;
    }
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

inline int grid_of(const LaunchCommon& lc, int count) {
  return count < 2 * lc.num_sms ? (count > 0 ? count : 1) : 2 * lc.num_sms;
}

template <int D>
void ShatL<D>::run(const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                  const double* Vt, const void* sigma, void* shat) {
    ++*lc.launches;
    k_shat<D><<<grid_of(lc, count), 64, 0, lc.stream>>>(plist, count, node_off, Vt,
                                                        (const cplx*)sigma, (cplx*)shat);
  }

template <int D>
void GradRulesL<D>::run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, const int32_t* qn, const int64_t* src_off, int64_t n_over,
                  const double* tg, const void* g, const void* shat, double* M) {
    ++*lc.launches;
    k_grad_rules<D><<<grid_of(lc, count), kThreads, 0, lc.stream>>>(
        plist, count, dv, kp, qn, src_off, n_over, tg, (const cplx*)g, (const cplx*)shat, M);
  }

template <int D>
void AdaptiveGradL<D>::run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, double eps, double normV, int leaf_order, int max_depth,
                  const void* I_smooth, void* I_near, int32_t* leaves, void* work, int64_t stride,
                  int A_max, int levels, int grid, int* status, int* sched, int form,
                  const GradArgs& ga) {
    const size_t sm = adaptive_smem_bytes<D>();
    cudaFuncSetAttribute(k_adaptive<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    AdaptiveWS w{stride, A_max, levels};
    cudaMemsetAsync(sched, 0, sizeof(int), lc.stream);
    ++*lc.launches;
    k_adaptive<D, true><<<grid, kThreads, sm, lc.stream>>>(
        plist, count, dv, kp, eps, normV, leaf_order, max_depth, (const cplx*)I_smooth,
        (cplx*)I_near, leaves, (unsigned char*)work, w, status, sched, form, ga, nullptr, 0);
  }

template <int D>
void GradV2cL<D>::run(const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                  const double* Vt, const double* M, int64_t N, double* out) {
    ++*lc.launches;
    k_grad_v2c<D><<<grid_of(lc, count), 128, 0, lc.stream>>>(plist, count, node_off, Vt, M, N,
                                                             out);
  }

template <int D>
void AdjPatchL<D>::run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const double* Vt, const int64_t* src_off, const void* z, const double* val,
                  const void* g, double jump, void* out) {
    ++*lc.launches;
    k_adj_patch<D><<<grid_of(lc, count), 64, 0, lc.stream>>>(plist, count, dv, Vt, src_off,
                                                             (const cplx*)z, val, (const cplx*)g,
                                                             jump, (cplx*)out);
  }

}  // namespace lcq
