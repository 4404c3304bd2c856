// Degree-templated CUDA kernels of the correction path (sm_103a) and their launchers,
// instantiated one patch degree per translation unit (lcq_deg.cu built with -DLCQ_DEG=d) so
// that the degrees compile in parallel; lcq_kernels.cu dispatches to them by degree.
//
//   k_geom         chart coefficients, centroid, radius, d_j        (Sec. 3.2, Sec. 4)
//   k_farorder     far order q_j and annulus order                  (Sec. 4.2, Eq. qj)
//   k_rule_moments smooth-rule / annulus moments for many targets    (Sec. 4.2, Remark on eta_1)
//   k_adaptive     adaptive subdivision over a per-patch union tree  (Sec. 4.3; lcq_common.cuh)
//   k_self         singular self rules                              (Sec. 4, Eq. errestself)
//   k_v2c          a - s = V^T (I_near - I_smooth) into the CSR       (Sec. 4.3, 5.3)
//   k_far_src      oversampled far sources of the corrected potential (Sec. 5.3)
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lcq_common.cuh"
#include "lcq_degree.h"

namespace lcq {

// ============================================================================ geometry
// One block per patch: x_nm = V y, J at the nodes, c_j, R_j, d_j (Sec. 3.2, 4).
template <int D>
__global__ void k_geom(const int* __restrict__ plist, int count, const int64_t* __restrict__ node_off,
                       const double* __restrict__ xyz, int64_t N, const double* __restrict__ Vt,
                       const double* __restrict__ nodes, double eta_p, double eta1_p,
                       double* __restrict__ coef, double* __restrict__ cen, double* __restrict__ rad,
                       double* __restrict__ dj, double* __restrict__ eta, double* __restrict__ eta1,
                       int* __restrict__ status) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  __shared__ double y[3][n];
  __shared__ double cf[n * 3];
  __shared__ double J[n];
  __shared__ double c[3];
  __shared__ double red[kThreads / 32];
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const int j = plist[b];
    const int64_t off = node_off[j];
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * n; e += blockDim.x) {
      const int cc = e / n, l = e % n;
      const double val = xyz[cc * N + off + l];
      if (!isfinite(val)) atomicOr(status, kStNonFinite);
      y[cc][l] = val;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * n; e += blockDim.x) {
      const int nm = e / 3, cc = e % 3;
      double acc = 0.0;
      for (int l = 0; l < n; ++l) acc = fma(Vt[nm * n + l], y[cc][l], acc);
      cf[nm * 3 + cc] = acc;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      double X[3], Xu[3], Xv[3], Nn[3];
      kw_geometry<D>(nodes[l], nodes[n + l], cf, X, Xu, Xv, nullptr, 1);
      cross3(Xu, Xv, Nn);
      const double jj = sqrt(Nn[0] * Nn[0] + Nn[1] * Nn[1] + Nn[2] * Nn[2]);
      if (!(jj > 0.0)) atomicOr(status, kStDegenerate);
      J[l] = jj;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sw = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0, dmin = 1e300;
      for (int l = 0; l < n; ++l) {
        const double wj = nodes[2 * n + l] * J[l];
        sw += wj;
        s0 += wj * y[0][l];
        s1 += wj * y[1][l];
        s2 += wj * y[2][l];
        dmin = fmin(dmin, sqrt(wj));
      }
      c[0] = s0 / sw;
      c[1] = s1 / sw;
      c[2] = s2 / sw;
      dj[j] = dmin;
      const double e1 = eta_p > 0.0 ? eta_p : eta_default(D);
      eta[j] = e1;
      eta1[j] = fmin(eta1_p, e1);
    }
    __syncthreads();
    // radius: 153 vertices of the level-4 subdivision of T0 plus the nodes
    double rmax = 0.0;
    for (int s = threadIdx.x; s < 153 + n; s += blockDim.x) {
      double p0, p1, p2;
      if (s < 153) {
        int a = 0, r = s;
        while (r >= 17 - a) {
          r -= 17 - a;
          ++a;
        }
        double X[3], Xu[3], Xv[3];
        kw_geometry<D>(a / 16.0, r / 16.0, cf, X, Xu, Xv, nullptr, 1);
        p0 = X[0];
        p1 = X[1];
        p2 = X[2];
      } else {
        p0 = y[0][s - 153];
        p1 = y[1][s - 153];
        p2 = y[2][s - 153];
      }
      const double d0 = p0 - c[0], d1 = p1 - c[1], d2 = p2 - c[2];
      rmax = fmax(rmax, sqrt(d0 * d0 + d1 * d1 + d2 * d2));
    }
    rmax = warp_max(rmax);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
      rad[j] = r;
      cen[3 * j] = c[0];
      cen[3 * j + 1] = c[1];
      cen[3 * j + 2] = c[2];
    }
    // coefficients of X - c_j (K_00 = sqrt(2) is constant): every local quadrature works
    // with positions relative to the centroid
    for (int e = threadIdx.x; e < 3 * n; e += blockDim.x)
      coef[off * 3 + e] = e < 3 ? cf[e] - c[e] * 0.70710678118654752 : cf[e];
  }
}

// Smooth rule q_j moments for every near pair of the patch (Sec. 4.2): I_smooth (modes
// bit 0, rule qv, out_smooth); and annulus-rule moments for the annulus pairs (Remark on
// eta_1; modes bit 1, rule qn, out_ann).  One block per patch and launch, both passes in it.
template <int D>
__global__ void __launch_bounds__(kThreads, 2) k_rule_moments(
    const int* __restrict__ plist, int count, Dev dv, int modes, const int32_t* __restrict__ qv,
    const int32_t* __restrict__ qn, const KernelParams kp, cplx* __restrict__ out_smooth,
    cplx* __restrict__ out_ann, int form) {
  using C = Cfg<D>;
  extern __shared__ double smem[];
  double* cf = smem;
  SegMap* segs = reinterpret_cast<SegMap*>(cf + C::n * 3);
  // tensor-core moment workspace, 128-byte aligned
  unsigned char* smb = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(segs + 4) + 127) & ~static_cast<uintptr_t>(127));
  __shared__ KernelParams kps;
  __shared__ double cfd[2 * 3 * (D * (D + 1) / 2)];  // derivative series of the chart
  const double* cfdp = cfd;
  const int64_t ld = dv.ldI;
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const int j = plist[b];
    const int formj = pair_form(dv, j, form);  // FP64, FP32 or two-float pair evaluation
    __syncthreads();
    load_coef<D>(dv.coef, dv.node_off[j], cf);
    if (threadIdx.x == 0) {
      segs[0] = seg_T0();
      kps = patch_kp(dv, j, kp);
    }
    __syncthreads();
    load_coef_derivs<D>(cf, dv.duv[D], cfd);
    long long evals = 0;
    for (int mode = 0; mode < 2; ++mode) {
      if (!(modes & (1 << mode))) continue;
      const int m = mode == 0 ? qv[j] : qn[j];
      if (m <= 0) continue;
      const double* ru = dv.ru + dv.roff[m];
      const double* rv = dv.rv + dv.roff[m];
      const double* rw = dv.rw + dv.roff[m];
      if (mode == 0) {
        const int64_t p0 = dv.pair_ptr[j], np = dv.pair_ptr[j + 1] - p0;
        TgtIdx ta{dv.tgt, dv.NT, dv.pair_tgt + p0, dv.tnrm};
        cplx* base = out_smooth + p0 * ld;
        block_moments_any<D>(cf, cfdp, ru, rv, rw, m * m, segs, 1, ta, (int)np,
                             [=] __device__(int i) { return base + (int64_t)i * ld; }, kps, smb,
                             dv.cen + 3 * j, 0.0, nullptr, formj);
        evals += np * m * m;
      } else {
        const int64_t a0 = dv.an_ptr[j], na = dv.an_ptr[j + 1] - a0;
        const int32_t* pl = dv.an_pair + a0;
        TgtPairIdx ta{dv.tgt, dv.NT, dv.pair_tgt, pl, dv.tnrm};
        block_moments_any<D>(cf, cfdp, ru, rv, rw, m * m, segs, 1, ta, (int)na,
                             [=] __device__(int i) { return out_ann + (int64_t)pl[i] * ld; }, kps,
                             smb, dv.cen + 3 * j, 0.0, nullptr, formj);
        evals += na * m * m;
      }
    }
    if (threadIdx.x == 0 && evals > 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(dv.counters + 3), (unsigned long long)evals);
  }
}

// ============================================================================ far order
// q_j (Eq. qj) and the annulus order: smallest m with
//   max_x ||I_m(x) - I_{m+1}(x)||_2 <= eps d_j / ||V||  over the test points.
template <int D>
__global__ void __launch_bounds__(kThreads, 2) k_farorder(const int* __restrict__ plist, int count,
                                                       Dev dv, const KernelParams kp, double eps,
                                                       int m_max, double normV,
                                                       const double* __restrict__ dirs, int ndirs,
                                                       cplx* __restrict__ scratch,
                                                       int32_t* __restrict__ q_out,
                                                       int32_t* __restrict__ qn_out,
                                                       int* __restrict__ sched) {
  using C = Cfg<D>;
  extern __shared__ double smem[];
  double* cf = smem;
  SegMap* segs = reinterpret_cast<SegMap*>(cf + C::n * 3);
  double* pts = reinterpret_cast<double*>(segs + 4);        // [kMaxTestPts][3]
  double* red = pts + 3 * kMaxTestPts;                      // [kThreads/32]
  int* sel = reinterpret_cast<int*>(red + kThreads / 32);   // [2]
  double* ws = reinterpret_cast<double*>(sel + 4);
  __shared__ KernelParams kps;
  __shared__ double cfd[2 * 3 * (D * (D + 1) / 2)];  // derivative series of the chart
  const double* cfdp = cfd;
  cplx* bufA = scratch + (int64_t)blockIdx.x * 2 * kMaxTestPts * C::n;
  cplx* bufB = bufA + kMaxTestPts * C::n;
  const int m_min = (D + 2) / 2;
  __shared__ int next_b;
  // patches are taken from the counter *sched (zeroed before the launch), so blocks that
  // drew cheap patches take more of them
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) next_b = atomicAdd(sched, 1);
    __syncthreads();
    const int b = next_b;
    if (b >= count) break;
    const int j = plist[b];
    load_coef<D>(dv.coef, dv.node_off[j], cf);
    if (threadIdx.x == 0) {
      segs[0] = seg_T0();
      kps = patch_kp(dv, j, kp);
    }
    __syncthreads();
    load_coef_derivs<D>(cf, dv.duv[D], cfd);
    const int64_t p0 = dv.pair_ptr[j], np = dv.pair_ptr[j + 1] - p0;
    const double R = dv.rad[j], c0 = dv.cen[3 * j], c1 = dv.cen[3 * j + 1], c2 = dv.cen[3 * j + 2];
    const double tol = (dv.pgroup ? dv.grp[dv.pgroup[j]].eps : eps) * dv.dj[j] / normV;
    for (int pass = 0; pass < 2; ++pass) {
      // test points (Sec. 4.2): pass 0 = far order, pass 1 = annulus order
      __syncthreads();
      if (threadIdx.x == 0) {
        int F = 0;
        if (pass == 0) {
          const int cnt = np >= 20 ? 10 : (int)(np / 2);
          // repeated selection: largest d2, ties by smaller target id.  d2 >= 0, whose bit
          // patterns order like the values: the compares run on the integer pipe.
          long long lastd = 0x7fffffffffffffffll;
          int lastt = -1;
          for (int k = 0; k < cnt; ++k) {
            long long bd = -1;
            int bt = 0x7fffffff;
            for (int64_t p = 0; p < np; ++p) {
              const long long d = __double_as_longlong(dv.pair_d2[p0 + p]);
              const int t = dv.pair_tgt[p0 + p];
              const bool after = (d < lastd) || (d == lastd && t > lastt);
              if (!after) continue;
              if (d > bd || (d == bd && t < bt)) {
                bd = d;
                bt = t;
              }
            }
            lastd = bd;
            lastt = bt;
            pts[3 * F] = dv.tgt[bt];
            pts[3 * F + 1] = dv.tgt[dv.NT + bt];
            pts[3 * F + 2] = dv.tgt[2 * dv.NT + bt];
            ++F;
          }
          if (np < 20)
            for (int k = 0; k < ndirs && F < kMaxTestPts; ++k) {
              const double rr = dv.eta[j] * R;
              pts[3 * F] = c0 + rr * dirs[3 * k];
              pts[3 * F + 1] = c1 + rr * dirs[3 * k + 1];
              pts[3 * F + 2] = c2 + rr * dirs[3 * k + 2];
              ++F;
            }
        } else {
          const int64_t a0 = dv.an_ptr[j], na = dv.an_ptr[j + 1] - a0;
          if (na > 0) {
            for (int k = 0; k < ndirs && F < kMaxTestPts; ++k) {
              const double rr = dv.eta1[j] * R;
              pts[3 * F] = c0 + rr * dirs[3 * k];
              pts[3 * F + 1] = c1 + rr * dirs[3 * k + 1];
              pts[3 * F + 2] = c2 + rr * dirs[3 * k + 2];
              ++F;
            }
            const int cnt = na < 10 ? (int)na : 10;
            long long lastd = -1;
            int lastt = -1;
            for (int k = 0; k < cnt && F < kMaxTestPts; ++k) {
              long long bd = 0x7fffffffffffffffll;
              int bt = 0x7fffffff;
              for (int64_t a = 0; a < na; ++a) {
                const int64_t p = dv.an_pair[a0 + a];
                const long long d = __double_as_longlong(dv.pair_d2[p]);
                const int t = dv.pair_tgt[p];
                const bool after = (d > lastd) || (d == lastd && t > lastt);
                if (!after) continue;
                if (d < bd || (d == bd && t < bt)) {
                  bd = d;
                  bt = t;
                }
              }
              lastd = bd;
              lastt = bt;
              pts[3 * F] = dv.tgt[bt];
              pts[3 * F + 1] = dv.tgt[dv.NT + bt];
              pts[3 * F + 2] = dv.tgt[2 * dv.NT + bt];
              ++F;
            }
          }
        }
        sel[0] = F;
      }
      __syncthreads();
      const int F = sel[0];
      if (pass == 1 && F == 0) {
        if (threadIdx.x == 0) qn_out[j] = 0;
        continue;
      }
      TgtPts ta{pts};
      int m = m_min, chosen = m_max;
      {
        const double* ru = dv.ru + dv.roff[m];
        block_moments<D>(cf, cfdp, ru, dv.rv + dv.roff[m], dv.rw + dv.roff[m], m * m, segs, 1, ta, F,
                         [=] __device__(int i) { return bufA + (int64_t)i * C::n; }, C::n, kps, ws,
                         dv.cen + 3 * j);
      }
      cplx* A = bufA;
      cplx* Bf = bufB;
      for (; m < m_max; ++m) {
        const int m1 = m + 1;
        block_moments<D>(cf, cfdp, dv.ru + dv.roff[m1], dv.rv + dv.roff[m1], dv.rw + dv.roff[m1], m1 * m1,
                         segs, 1, ta, F, [=] __device__(int i) { return Bf + (int64_t)i * C::n; },
                         C::n, kps, ws, dv.cen + 3 * j);
        __syncthreads();
        // max over points of the 2-norm of the difference
        double e = 0.0;
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = w; i < F; i += blockDim.x >> 5) {
          double s = 0.0;
          for (int nm = lane; nm < C::n; nm += 32) {
            const cplx a = A[i * C::n + nm], bb = Bf[i * C::n + nm];
            const double dr = a.re - bb.re, di = a.im - bb.im;
            s += dr * dr + di * di;
          }
          s = warp_sum(s);
          e = fmax(e, sqrt(s));
        }
        if (lane == 0) red[w] = e;
        __syncthreads();
        if (threadIdx.x == 0) {
          double mx = 0.0;
          for (int k = 0; k < (int)(blockDim.x >> 5); ++k) mx = fmax(mx, red[k]);
          sel[1] = mx <= tol ? 1 : 0;
        }
        __syncthreads();
        if (sel[1]) {
          chosen = m;
          break;
        }
        cplx* tmp = A;
        A = Bf;
        Bf = tmp;
      }
      if (threadIdx.x == 0) {
        if (pass == 0) q_out[j] = chosen; else qn_out[j] = chosen;
      }
    }
  }
}

// ============================================================================ self
// Self rule for the target at node i (Sec. 4, Eq. errestself; stand-in for
// generalized Gaussian rules): affine map M = G^{-1/2} (G the first fundamental
// form at the node) making the chart conformal there, split at the node into three
// Duffy triangles; s: n_s-point Gauss-Legendre; t: split at the foot of the
// perpendicular, sinh substitution t - t0 = mu sinh(xi), [0, xi_max] cut into
// ceil(xi_max / 1.5) panels of n_t-point Gauss-Legendre.
struct SelfSeg {
  double E0x, E0y, Dx, Dy, t0, mu, area2, xi_max, side;
  int npan, off;
};

// Block per self target: the self rule above applied to the chart, contracted with the
// basis into the target's self weights (Sec. 4).
template <int D>
__global__ void __launch_bounds__(128) k_self(Dev dv, const int32_t* __restrict__ deg_of_patch,
                                              const KernelParams kp, int order,
                                              cplx* __restrict__ out_self) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  __shared__ double cf[3 * n];
  __shared__ SelfSeg sg[6];
  __shared__ double Mm[5];  // M00 M01 M10 M11 detM
  __shared__ double P[2];
  __shared__ int nseg, total;
  __shared__ cplx red[4][n];
  __shared__ KernelParams kps;
  __shared__ int ord;
  __shared__ double nP[3];  // unit chart normal at the target node (S')
  __shared__ double cfd[2 * 3 * (D * (D + 1) / 2)];  // derivative series of the chart
  __shared__ cplx gbuf[128];                          // kernel values of a chunk's nodes
  __shared__ double tX[3 * n];                        // Taylor coefficients of the chord at P
  extern __shared__ double krows[];                   // [128][n + 1] basis rows of a chunk
  long long my_nodes = 0;
  for (int64_t s = blockIdx.x; s < dv.n_self; s += gridDim.x) {
    const int t = dv.self_tgt[s];
    const int j = dv.tpatch[t];
    if (deg_of_patch[j] != D) continue;
    const int i = dv.tlnode[t];
    __syncthreads();
    load_coef<D>(dv.coef, dv.node_off[j], cf);
    if (threadIdx.x == 0) {
      kps = patch_kp(dv, j, kp);
      ord = dv.pgroup ? dv.grp[dv.pgroup[j]].self_order : order;
    }
    __syncthreads();
    load_coef_derivs<D>(cf, dv.duv[D], cfd);
    const int ns = ord, nt = ord;
    const double* glx_s = dv.gl_x + dv.gl_off[ns];
    const double* glw_s = dv.gl_w + dv.gl_off[ns];
    const double* glx_t = dv.gl_x + dv.gl_off[nt];
    const double* glw_t = dv.gl_w + dv.gl_off[nt];
    if (threadIdx.x == 0) {
      const double pu = dv.nodes_uv[D][i], pv = dv.nodes_uv[D][n + i];
      P[0] = pu;
      P[1] = pv;
      double X[3], Xu[3], Xv[3];
      kw_geometry<D>(pu, pv, cf, X, Xu, Xv, nullptr, 1);
      {
        double Np[3];
        cross3(Xu, Xv, Np);
        const double ln = sqrt(Np[0] * Np[0] + Np[1] * Np[1] + Np[2] * Np[2]);
        nP[0] = Np[0] / ln;
        nP[1] = Np[1] / ln;
        nP[2] = Np[2] / ln;
      }
      const double a = Xu[0] * Xu[0] + Xu[1] * Xu[1] + Xu[2] * Xu[2];
      const double bb = Xu[0] * Xv[0] + Xu[1] * Xv[1] + Xu[2] * Xv[2];
      const double c = Xv[0] * Xv[0] + Xv[1] * Xv[1] + Xv[2] * Xv[2];
      const double sq = sqrt(a * c - bb * bb);
      const double tt = sqrt(a + c + 2.0 * sq);
      // R = sqrt(G) = (G + sq I)/tt ; M = R^{-1}
      const double R00 = (a + sq) / tt, R01 = bb / tt, R11 = (c + sq) / tt;
      const double detR = R00 * R11 - R01 * R01;
      Mm[0] = R11 / detR;
      Mm[1] = -R01 / detR;
      Mm[2] = -R01 / detR;
      Mm[3] = R00 / detR;
      Mm[4] = 1.0 / detR;
      double Z[3][2];
      const double VX[3] = {0.0, 1.0, 0.0}, VY[3] = {0.0, 0.0, 1.0};
      for (int k = 0; k < 3; ++k) {
        const double dx = VX[k] - pu, dy = VY[k] - pv;
        Z[k][0] = R00 * dx + R01 * dy;
        Z[k][1] = R01 * dx + R11 * dy;
      }
      int cntg = 0, off = 0;
      for (int e = 0; e < 3; ++e) {
        const double E0x = Z[e][0], E0y = Z[e][1];
        const double Dx = Z[(e + 1) % 3][0] - E0x, Dy = Z[(e + 1) % 3][1] - E0y;
        const double L2 = Dx * Dx + Dy * Dy;
        double t0 = -(E0x * Dx + E0y * Dy) / L2;
        t0 = fmin(fmax(t0, 0.0), 1.0);
        const double area2 = fabs(E0x * Dy - E0y * Dx);
        const double mu = area2 / L2;
        for (int sd = 0; sd < 2; ++sd) {
          const double side = sd == 0 ? 1.0 : -1.0;
          const double len = sd == 0 ? 1.0 - t0 : t0;
          if (len <= 0.0) continue;
          const double xm = asinh(len / mu);
          int npan = 1;
          if (isfinite(xm) && xm > 0.0) npan = (int)fmin(ceil(xm / 1.5), 64.0);
          else atomicOr(dv.status, kStNonFinite);
          SelfSeg g{E0x, E0y, Dx, Dy, t0, mu, area2, xm, side, npan, off};
          sg[cntg++] = g;
          off += npan * nt * ns;
        }
      }
      nseg = cntg;
      total = off;
    }
    __syncthreads();
    const KernelParamsF kfs = to_f32(kps);
    chart_taylor<D>(P[0], P[1], cf, krows, tX);  // krows is free until the first chunk
    // the target is the chart's value at the node: x - X(P + delta) = -(dX)
    // chunks of 128 nodes: each thread forms one node's kernel value and basis row in
    // shared memory, then the block contracts them, thread (nm, quarter of the chunk)
    const int tot = total;
    constexpr int NR = (n + 31) / 32;  // basis indices per thread in the contraction
    const int lane = threadIdx.x & 31, part = threadIdx.x >> 5;
    double are[NR], aim[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) are[r] = aim[r] = 0.0;
    for (int c0 = 0; c0 < tot; c0 += 128) {
      const int idx = c0 + threadIdx.x;
      cplx gk = {0.0, 0.0};
      double* Kq = krows + threadIdx.x * (n + 1);
      if (idx < tot) {
        int k = 0;
        while (k + 1 < nseg && idx >= sg[k + 1].off) ++k;
        const SelfSeg& g = sg[k];
        const int loc = idx - g.off;
        const int p = loc / (nt * ns);
        const int rem = loc - p * nt * ns;
        const int ti = rem / ns, si = rem - ti * ns;
        const double lo = g.xi_max * p / g.npan, hi = g.xi_max * (p + 1) / g.npan;
        const double xi = lo + (hi - lo) * glx_t[ti];
        // sinh and cosh from one exponential (xi >= 0: the difference loses at most a few
        // 1e-16 absolute near xi = 0, which moves the node by mu times that)
        const double ex = exp(xi), exi = 1.0 / ex;
        const double tpar = g.t0 + g.side * g.mu * (0.5 * (ex - exi));
        const double wt = glw_t[ti] * (hi - lo) * g.mu * (0.5 * (ex + exi));
        const double sv = glx_s[si];
        const double w = glw_s[si] * wt * sv * g.area2 * Mm[4];
        const double zx = sv * (g.E0x + tpar * g.Dx), zy = sv * (g.E0y + tpar * g.Dy);
        const double du = Mm[0] * zx + Mm[1] * zy;
        const double dvv = Mm[2] * zx + Mm[3] * zy;
        double dX[3], Xu[3], Xv[3], Nn[3];
        kw_geometry_proj<D, false>(P[0] + du, P[1] + dvv, cf, cfd, nullptr, Xu, Xv, Kq);
        chart_chord<D>(tX, du, dvv, dX);
        cross3(Xu, Xv, Nn);
        const double J = sqrt(Nn[0] * Nn[0] + Nn[1] * Nn[1] + Nn[2] * Nn[2]);
        float unused;
        gk = kernel_eval_tc(kps, kfs, g_sct, 0.0, 0.0, 0.0, dX[0], dX[1], dX[2], Nn[0] * w,
                            Nn[1] * w, Nn[2] * w, J * w, 0.0f, 0.0f, &unused, nP, kps.ki != 0.0);
      } else {
        for (int e = 0; e < n; ++e) Kq[e] = 0.0;
      }
      gbuf[threadIdx.x] = gk;
      __syncthreads();
      const int qa = part * 32, qb = min(qa + 32, tot - c0);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int nm = lane + 32 * r;
        if (nm < n)
          for (int q = qa; q < qb; ++q) {
            const cplx gq = gbuf[q];
            const double kv = krows[q * (n + 1) + nm];
            are[r] = fma(gq.re, kv, are[r]);
            aim[r] = fma(gq.im, kv, aim[r]);
          }
      }
      __syncthreads();
    }
    my_nodes += tot;
    // the four quarters, in a fixed order
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int nm = lane + 32 * r;
      if (nm < n) red[part][nm] = {are[r], aim[r]};
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      cplx sum = red[0][k];
      for (int q = 1; q < 4; ++q) {
        sum.re += red[q][k].re;
        sum.im += red[q][k].im;
      }
      out_self[s * dv.ldI + k] = sum;
    }
  }
  if (threadIdx.x == 0)
    atomicAdd(reinterpret_cast<unsigned long long*>(dv.counters + 2), (unsigned long long)my_nodes);
}

// ============================================================================ target normals
// Unit normals for S': the chart normal X_u x X_v / |.| at the node of an on-surface target
// on a degree-D patch; with do_off, the normalized user normal of an off-surface target.
template <int D>
__global__ void k_tgt_normals(Dev dv, const int32_t* __restrict__ deg, const double* __restrict__ user,
                              bool do_off, double* __restrict__ out) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dv.NT;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int tp = dv.tpatch[t];
    double v[3];
    if (tp >= 0) {
      if (deg[tp] != D) continue;
      double cf[3 * n], X[3], Xu[3], Xv[3];
      const int64_t off = dv.node_off[tp];
      for (int e = 0; e < 3 * n; ++e) cf[e] = dv.coef[off * 3 + e];
      const int i = dv.tlnode[t];
      kw_geometry<D>(dv.nodes_uv[D][i], dv.nodes_uv[D][n + i], cf, X, Xu, Xv, nullptr, 1);
      cross3(Xu, Xv, v);
    } else {
      if (!do_off) continue;
      v[0] = user[t];
      v[1] = user[dv.NT + t];
      v[2] = user[2 * dv.NT + t];
    }
    const double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(l > 0.0) || !isfinite(l)) atomicOr(dv.status, kStNonFinite);
    for (int c = 0; c < 3; ++c) out[c * dv.NT + t] = v[c] / l;
  }
}

// ============================================================================ V contraction
// c_l = sum_nm V[nm][l] (I_near[nm] - I_smooth[nm]) written to the CSR (Sec. 4.3, 5.3).
template <int D>
__global__ void k_v2c(const int* __restrict__ plist, int count, Dev dv,
                      const double* __restrict__ Vt, const cplx* __restrict__ In,
                      const cplx* __restrict__ Is, const cplx* __restrict__ InS,
                      double* __restrict__ val) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  __shared__ double V[n * n];
  __shared__ cplx diff[kThreads / 32][n];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = Vt[e];
  __syncthreads();
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const int j = plist[b];
    const int64_t p0 = dv.pair_ptr[j], np = dv.pair_ptr[j + 1] - p0;
    const int64_t s0 = dv.self_ptr[j], nsf = dv.self_ptr[j + 1] - s0;
    for (int64_t k = w; k < np + nsf; k += nw) {
      const bool self = k >= np;
      const int64_t id = self ? (s0 + k - np) : (p0 + k);
      // self pairs store the self weights themselves: the own patch is masked out of the
      // far sum (no spurious smooth-rule contribution to subtract)
      const cplx* a = self ? InS + id * dv.ldI : In + id * dv.ldI;
      const cplx* s = Is + id * dv.ldI;
      for (int nm = lane; nm < n; nm += 32)
        diff[w][nm] = self ? a[nm] : cplx{a[nm].re - s[nm].re, a[nm].im - s[nm].im};
      __syncwarp();
      const int64_t dst = self ? dv.self_csr[id] : dv.pair_csr[id];
      for (int l = lane; l < n; l += 32) {
        double re = 0.0, im = 0.0;
        for (int nm = 0; nm < n; ++nm) {
          const double vv = V[nm * n + l];
          re = fma(vv, diff[w][nm].re, re);
          im = fma(vv, diff[w][nm].im, im);
        }
        val[2 * (dst + l)] = re;
        val[2 * (dst + l) + 1] = im;
      }
      __syncwarp();
    }
  }
}

// ============================================================================ apply
// Oversampled sources of rule q_j: X, (X_u x X_v) w, |.| w and w-weighted density
// sigma~_q = sum_nm K_nm(u_q) s_nm, s = V sigma (Sec. 4.2 Remark, Sec. 5.3).  With fold
// (real k, kinds S, D and CFIE with a real alpha) the patch's kernel constants are folded
// into the source data as kernel_eval_fold takes them: rows 3-5 N w alpha / (4 pi), row 6
// beta_r J w / (4 pi), row 9 beta_i J w / (4 pi).
template <int D>
__global__ void k_far_src(const int* __restrict__ plist, int count, Dev dv,
                          const double* __restrict__ Vt, const int32_t* __restrict__ qv,
                          const int64_t* __restrict__ src_off, const cplx* __restrict__ sigma,
                          double* __restrict__ src /*[9 or 10][N_over]*/, int64_t n_over,
                          const KernelParams kp, bool fold) {
  constexpr int n = (D + 1) * (D + 2) / 2;
  __shared__ double cf[3 * n];
  __shared__ double cfd[2 * 3 * (D * (D + 1) / 2)];  // derivative series of the chart
  __shared__ cplx sc[n];
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const int j = plist[b];
    const int64_t off = dv.node_off[j];
    const KernelParams kj = patch_kp(dv, j, kp);
    constexpr double kInv4Pi = 0.07957747154594767;
    const double fa_n = fold ? (kj.kind == 1 ? 1.0 : kj.ar) * kInv4Pi : 1.0;
    const double fj_r = fold ? (kj.kind == 0 ? 1.0 : kj.br) * kInv4Pi : 1.0;
    const double fj_i = kj.bi * kInv4Pi;
    __syncthreads();
    load_coef<D>(dv.coef, off, cf);
    __syncthreads();
    load_coef_derivs<D>(cf, dv.duv[D], cfd);
    for (int nm = threadIdx.x; nm < n; nm += blockDim.x) {
      double re = 0.0, im = 0.0;
      if (sigma)  // null: geometry only (the adjoint's sources)
        for (int l = 0; l < n; ++l) {
          re = fma(Vt[nm * n + l], sigma[off + l].re, re);
          im = fma(Vt[nm * n + l], sigma[off + l].im, im);
        }
      sc[nm] = {re, im};
    }
    __syncthreads();
    const int m = qv[j], Q = m * m;
    const double* ru = dv.ru + dv.roff[m];
    const double* rv = dv.rv + dv.roff[m];
    const double* rw = dv.rw + dv.roff[m];
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
      // chart and tangents by the projected derivative series (rolled sums over the stored
      // basis values keep the register count low), then the interpolated density
      double X[3], Xu[3], Xv[3], Nn[3], K[n];
      kw_geometry_proj<D>(ru[q], rv[q], cf, cfd, X, Xu, Xv, K);
      double re = 0.0, im = 0.0;
#pragma unroll 1
      for (int k = 0; k < n; ++k) {
        re = fma(K[k], sc[k].re, re);
        im = fma(K[k], sc[k].im, im);
      }
      cross3(Xu, Xv, Nn);
      const double w = rw[q];
      const double J = sqrt(Nn[0] * Nn[0] + Nn[1] * Nn[1] + Nn[2] * Nn[2]);
      const int64_t o = src_off[j] + q;
      src[0 * n_over + o] = X[0] + dv.cen[3 * j];
      src[1 * n_over + o] = X[1] + dv.cen[3 * j + 1];
      src[2 * n_over + o] = X[2] + dv.cen[3 * j + 2];
      const double wn = w * fa_n;
      src[3 * n_over + o] = Nn[0] * wn;
      src[4 * n_over + o] = Nn[1] * wn;
      src[5 * n_over + o] = Nn[2] * wn;
      src[6 * n_over + o] = J * w * fj_r;
      src[7 * n_over + o] = re;
      src[8 * n_over + o] = im;
      if (fold) src[9 * n_over + o] = J * w * fj_i;
    }
  }
}

// ============================================================================ launchers
template <class K>
void set_smem(K kern, size_t bytes) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int D>
void GeomL<D>::run(const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                  const double* xyz, int64_t N, const double* Vt, const double* nodes, double eta_p,
                  double eta1_p, double* coef, double* cen, double* rad, double* dj, double* eta,
                  double* eta1, int* status) {
    const int grid = count < lc.num_sms * 8 ? count : lc.num_sms * 8;
    ++*lc.launches;
    k_geom<D><<<grid, 128, 0, lc.stream>>>(plist, count, node_off, xyz, N, Vt, nodes, eta_p, eta1_p,
                                           coef, cen, rad, dj, eta, eta1, status);
  }


template <int D>
size_t moments_smem_bytes(int extra_doubles) {
  using C = Cfg<D>;
  return sizeof(double) * (C::n * 3 + extra_doubles + C::WS) + sizeof(SegMap) * 4 + 1024;
}

template <int D>
void RuleMomL<D>::run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv, int modes,
                  const int32_t* qv, const int32_t* qn, const KernelParams& kp, void* out_smooth,
                  void* out_ann, int form) {
    const size_t sm = sizeof(double) * 3 * Cfg<D>::n + sizeof(SegMap) * 4 + 128 + moment_ws_bytes<D>();
    set_smem(k_rule_moments<D>, sm);
    ++*lc.launches;
    // one block per patch: the hardware hands the next patch to whichever block slot frees
    k_rule_moments<D><<<count, kThreads, sm, lc.stream>>>(plist, count, dv, modes, qv, qn, kp,
                                                          (cplx*)out_smooth, (cplx*)out_ann, form);
  }

template <int D>
void FarOrderL<D>::run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, double eps, int m_max, double normV, const double* dirs,
                  int ndirs, void* scratch, int grid, int32_t* q, int32_t* qn, int* sched) {
    const size_t sm = moments_smem_bytes<D>(3 * kMaxTestPts + kThreads / 32 + 4);
    set_smem(k_farorder<D>, sm);
    ++*lc.launches;
    cudaMemsetAsync(sched, 0, sizeof(int), lc.stream);
    k_farorder<D><<<grid, kThreads, sm, lc.stream>>>(plist, count, dv, kp, eps, m_max, normV, dirs,
                                                     ndirs, (cplx*)scratch, q, qn, sched);
  }

template <int D>
int AdaptiveL<D>::blocks_per_sm() {
    int nb = 1;
    const size_t sm = adaptive_smem_bytes<D>();
    set_smem(k_adaptive<D>, sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adaptive<D>, kThreads, sm);
    cudaGetLastError();
    return nb < 1 ? 1 : nb;
  }

template <int D>
void AdaptiveL<D>::run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, double eps, double normV, int leaf_order, int max_depth,
                  const void* I_smooth, void* I_near, int32_t* leaves, void* work,
                  int64_t stride, int A_max, int levels, int grid, int* status, int* sched,
                  int form, const int64_t* gofs, int gsz) {
    const size_t sm = adaptive_smem_bytes<D>();
    set_smem(k_adaptive<D>, sm);
    AdaptiveWS w{stride, A_max, levels};
    ++*lc.launches;
    cudaMemsetAsync(sched, 0, sizeof(int), lc.stream);
    k_adaptive<D><<<grid, kThreads, sm, lc.stream>>>(plist, count, dv, kp, eps, normV, leaf_order,
                                                     max_depth, (const cplx*)I_smooth, (cplx*)I_near,
                                                     leaves, (unsigned char*)work, w, status, sched,
                                                     form, GradArgs{}, gofs, gsz);
  }

template <int D>
void SelfL<D>::run(const LaunchCommon& lc, const Dev& dv, const int32_t* deg, const KernelParams& kp,
                  int order, void* out) {
    // one block per self target: short-lived blocks, so that kernels on higher-priority
    // streams take the SMs they free first
    const int64_t g = dv.n_self < (int64_t)0x7fffffff ? dv.n_self : (int64_t)0x7fffffff;
    if (g <= 0) return;
    ++*lc.launches;
    constexpr size_t n = (D + 1) * (D + 2) / 2;
    constexpr size_t rows = 128 * (n + 1), taylor = (D + 1) * n + 2 * n * n;
    const size_t sm = (rows > taylor ? rows : taylor) * sizeof(double);
    set_smem(k_self<D>, sm);
    k_self<D><<<(int)g, 128, sm, lc.stream>>>(dv, deg, kp, order, (cplx*)out);
  }

template <int D>
void TgtNormalsL<D>::run(const LaunchCommon& lc, const Dev& dv, const int32_t* deg, const double* user,
                  bool do_off, double* out) {
    const int64_t b = (dv.NT + 127) / 128;
    const int g = (int)(b < lc.num_sms * 8 ? (b > 0 ? b : 1) : lc.num_sms * 8);
    ++*lc.launches;
    k_tgt_normals<D><<<g, 128, 0, lc.stream>>>(dv, deg, user, do_off, out);
  }

template <int D>
void V2cL<D>::run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const double* Vt, const void* In, const void* Is, const void* InS,
                  double* val) {
    const int grid = count < lc.num_sms * 4 ? count : lc.num_sms * 4;
    ++*lc.launches;
    k_v2c<D><<<grid, kThreads, 0, lc.stream>>>(plist, count, dv, Vt, (const cplx*)In,
                                               (const cplx*)Is, (const cplx*)InS, val);
  }

template <int D>
void FarSrcL<D>::run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const double* Vt, const int32_t* qv, const int64_t* src_off, const void* sigma,
                  double* src, int64_t n_over, const KernelParams& kp, bool fold) {
    const int grid = count < lc.num_sms * 4 ? count : lc.num_sms * 4;
    ++*lc.launches;
    k_far_src<D><<<grid, 128, 0, lc.stream>>>(plist, count, dv, Vt, qv, src_off,
                                              (const cplx*)sigma, src, n_over, kp, fold);
  }

template <int D>
cudaError_t upload_deg_constants(cudaStream_t st) {
  return upload_kw_tables(st);
}

}  // namespace lcq
