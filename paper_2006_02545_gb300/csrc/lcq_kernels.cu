// CUDA kernels of the correction path (sm_103a).  FP64 throughout.
//
//   k_geom         chart coefficients, centroid, radius, d_j        (Sec. 3.2, Sec. 4)
//   (near lists: lcq_nearlist.cu)
//   k_farorder     far order q_j and annulus order                  (Sec. 4.2, Eq. qj)
//   k_rule_moments smooth-rule / annulus moments for many targets    (Sec. 4.2, Remark on eta_1)
//   k_adaptive     adaptive subdivision over a per-patch union tree  (Sec. 4.3)
//   k_self         singular self rules                              (Sec. 4, Eq. errestself)
//   k_v2c          a - s = V^T (I_near - I_smooth) into the CSR       (Sec. 4.3, 5.3)
//   k_far_src / k_far_sum / k_csr_apply   corrected potential      (Sec. 5.3)
//   (the degree-templated kernels are in lcq_kernels.cuh, one object per degree: lcq_deg.cu)
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lcq_common.cuh"
#include "lcq_degree.h"

namespace lcq {

// ============================================================================ near lists
__global__ void k_tgt_patch(const double* __restrict__ tgt, const int64_t* __restrict__ tnode,
                            int64_t NT, const int64_t* __restrict__ node_off, int64_t P, int64_t N,
                            int32_t* __restrict__ tpatch, int32_t* __restrict__ tlnode,
                            int* __restrict__ status) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < NT;
       t += (int64_t)gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c)
      if (!isfinite(tgt[c * NT + t])) atomicOr(status, kStNonFinite);
    const int64_t nd = tnode[t];
    if (nd < 0 || nd >= N) {
      tpatch[t] = -1;
      tlnode[t] = -1;
      continue;
    }
    int64_t lo = 0, hi = P;  // largest j with node_off[j] <= nd
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (node_off[mid] <= nd) lo = mid; else hi = mid;
    }
    tpatch[t] = (int32_t)lo;
    tlnode[t] = (int32_t)(nd - node_off[lo]);
  }
}

// ============================================================================ scans
// Exclusive scan of int64 in blocks of 1024 (two passes + recursion on block sums).
__global__ void k_scan_block(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             int64_t* __restrict__ bsum) {
  __shared__ int64_t s[1024];
  const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
  const int64_t x = i < n ? in[i] : 0;
  s[threadIdx.x] = x;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int64_t add = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - x;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = s[1023];
}
// Second pass: adds the scanned block sums to each block's entries.
__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ boff) {
  const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}

// Direct far sum over all oversampled sources, one thread per target (tiles of sources
// staged through shared memory); kernel values by kernel_eval_tc (table sincos and the
// Newton-refined reciprocal square root: FP64 throughout, about 48 FP64 instructions per
// pair for the CFIE), or with fold by kernel_eval_fold on sources that carry the kernel
// constants (about 41).
// The sources of an on-surface target's own patch are skipped (their contribution is
// carried entirely by the self correction).  In a batch of independent surfaces a target
// sums only its own surface's sources [gsrc[g], gsrc[g+1]) with that surface's kernel.
__global__ void __launch_bounds__(kThreads) k_far_sum(const double* __restrict__ tgt, int64_t NT,
                                                      const double* __restrict__ src, int64_t n_over,
                                                      const KernelParams kp,
                                                      const int32_t* __restrict__ tpatch,
                                                      const int64_t* __restrict__ src_off,
                                                      const int32_t* __restrict__ tgroup,
                                                      const GroupParams* __restrict__ grp,
                                                      const int64_t* __restrict__ gsrc,
                                                      const double* __restrict__ tnrm,
                                                      cplx* __restrict__ out, bool fold) {
  __shared__ double s[10][kThreads];
  __shared__ unsigned long long blo, bhi;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double x0 = 0, x1 = 0, x2 = 0;
  int64_t skip0 = -1, skip1 = -1, lo = 0, hi = 0;
  double nx[3] = {0.0, 0.0, 0.0};
  KernelParams kt = kp;
  if (threadIdx.x == 0) {
    blo = ~0ull;
    bhi = 0ull;
  }
  __syncthreads();
  if (t < NT) {
    x0 = tgt[t];
    x1 = tgt[NT + t];
    x2 = tgt[2 * NT + t];
    if (tnrm) {
      nx[0] = tnrm[t];
      nx[1] = tnrm[NT + t];
      nx[2] = tnrm[2 * NT + t];
    }
    const int tp = tpatch[t];
    if (tp >= 0) {
      skip0 = src_off[tp];
      skip1 = src_off[tp + 1];
    }
    hi = n_over;
    if (tgroup) {
      const int g = tgroup[t];
      kt = grp[g].kp;
      lo = gsrc[g];
      hi = gsrc[g + 1];
    }
    atomicMin(&blo, (unsigned long long)lo);
    atomicMax(&bhi, (unsigned long long)hi);
  }
  __syncthreads();
  const int64_t b0 = (int64_t)blo, b1 = (int64_t)bhi;
  const KernelParamsF kf = to_f32(kt);
  const bool has_ki = kt.ki != 0.0;
  float env;  // not used: the far sum needs no rounding envelope
  double re = 0.0, im = 0.0;
  const int rows = fold ? 10 : 9;
  for (int64_t s0 = b0; s0 < b1; s0 += kThreads) {
    __syncthreads();
    const int64_t q = s0 + threadIdx.x;
    for (int c = 0; c < rows; ++c) s[c][threadIdx.x] = q < b1 ? src[c * n_over + q] : 0.0;
    __syncthreads();
    const int cnt = (int)min((int64_t)kThreads, b1 - s0);
    if (t < NT)
      for (int k = 0; k < cnt; ++k) {
        const int64_t qq = s0 + k;
        if (qq < lo || qq >= hi || (qq >= skip0 && qq < skip1)) continue;
        const cplx g =
            fold ? kernel_eval_fold(kt.kind, kt.kr, kf, g_sct, x0, x1, x2, s[0][k], s[1][k],
                                    s[2][k], s[3][k], s[4][k], s[5][k], s[6][k], s[9][k], 0.0f,
                                    0.0f, &env)
                 : kernel_eval_tc(kt, kf, g_sct, x0, x1, x2, s[0][k], s[1][k], s[2][k], s[3][k],
                                  s[4][k], s[5][k], s[6][k], 0.0f, 0.0f, &env, nx, has_ki);
        re = fma(g.re, s[7][k], re);
        re = fma(-g.im, s[8][k], re);
        im = fma(g.re, s[8][k], im);
        im = fma(g.im, s[7][k], im);
      }
  }
  if (t < NT) out[t] = {re, im};
}

// The correction part of the corrected potential (Sec. 5.3): warp per target row,
// out_t += sum_row c sigma, plus jump * sigma at an on-surface target's own node.
__global__ void k_csr_apply(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const cplx* __restrict__ sigma,
                            const int64_t* __restrict__ tnode, int64_t NT, double jump,
                            cplx* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < NT; t += warps) {
    double re = 0.0, im = 0.0;
    for (int64_t e = row_ptr[t] + lane; e < row_ptr[t + 1]; e += 32) {
      const double vr = val[2 * e], vi = val[2 * e + 1];
      const cplx sg = sigma[col[e]];
      re += vr * sg.re - vi * sg.im;
      im += vr * sg.im + vi * sg.re;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) {
      cplx o = out[t];
      o.re += re;
      o.im += im;
      if (jump != 0.0 && tnode[t] >= 0) {
        o.re += jump * sigma[tnode[t]].re;
        o.im += jump * sigma[tnode[t]].im;
      }
      out[t] = o;
    }
  }
}

// complex64 density -> complex128 (apply of a density stored in single precision)
__global__ void k_widen_c64(const float2* __restrict__ in, int64_t n, cplx* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    out[i] = {(double)v.x, (double)v.y};
  }
}

// ============================================================================ launchers
namespace {
template <template <int> class F, class... Args>
bool dispatch(int d, Args&&... args) {
  switch (d) {
    case 1: F<1>::run(args...); return true;
    case 2: F<2>::run(args...); return true;
    case 3: F<3>::run(args...); return true;
    case 4: F<4>::run(args...); return true;
    case 5: F<5>::run(args...); return true;
    case 6: F<6>::run(args...); return true;
    case 7: F<7>::run(args...); return true;
    case 8: F<8>::run(args...); return true;
    case 9: F<9>::run(args...); return true;
    case 10: F<10>::run(args...); return true;
    default: return false;
  }
}

template <int D>
struct UploadL {
  static void run(cudaStream_t st, cudaError_t* e) {
    if (*e == cudaSuccess) *e = upload_deg_constants<D>(st);
  }
};
template <int D>
struct BlocksL {
  static void run(int* nb) { *nb = AdaptiveL<D>::blocks_per_sm(); }
};
}  // namespace

cudaError_t upload_constants(cudaStream_t st) {
  cudaError_t e = upload_kw_tables(st);
  for (int d = 1; d <= kMaxDeg && e == cudaSuccess; ++d) dispatch<UploadL>(d, st, &e);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

bool launch_geom(int d, const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                 const double* xyz, int64_t N, const double* Vt, const double* nodes, double eta_p,
                 double eta1_p, double* coef, double* cen, double* rad, double* dj, double* eta,
                 double* eta1, int* status) {
  return dispatch<GeomL>(d, lc, plist, count, node_off, xyz, N, Vt, nodes, eta_p, eta1_p, coef, cen,
                         rad, dj, eta, eta1, status);
}

void launch_tgt_patch(const LaunchCommon& lc, const double* tgt, const int64_t* tnode, int64_t NT,
                      const int64_t* node_off, int64_t P, int64_t N, int32_t* tpatch,
                      int32_t* tlnode, int* status) {
  const int64_t blocks = (NT + 255) / 256;
  const int g = (int)(blocks < lc.num_sms * 16 ? (blocks > 0 ? blocks : 1) : lc.num_sms * 16);
  ++*lc.launches;
  k_tgt_patch<<<g, 256, 0, lc.stream>>>(tgt, tnode, NT, node_off, P, N, tpatch, tlnode, status);
}

// On-surface targets follow their nodes (a captured regeneration after the nodes moved):
// tgt[:, t] = xyz[:, tnode[t]] where 0 <= tnode[t] < N; off-surface targets are kept.
__global__ void k_tgt_from_nodes(double* __restrict__ tgt, const int64_t* __restrict__ tnode,
                                 int64_t NT, const double* __restrict__ xyz, int64_t N) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < NT;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nd = tnode[t];
    if (nd < 0 || nd >= N) continue;
    for (int c = 0; c < 3; ++c) tgt[c * NT + t] = xyz[c * N + nd];
  }
}
void launch_tgt_from_nodes(const LaunchCommon& lc, double* tgt, const int64_t* tnode, int64_t NT,
                           const double* xyz, int64_t N) {
  if (NT <= 0) return;
  const int64_t blocks = (NT + 255) / 256;
  const int g = (int)(blocks < lc.num_sms * 16 ? blocks : lc.num_sms * 16);
  ++*lc.launches;
  k_tgt_from_nodes<<<g, 256, 0, lc.stream>>>(tgt, tnode, NT, xyz, N);
}

// out[i] = sum_{k<i} in[i]; needs scratch of >= 2 * ceil(n/1024) + 2048 int64 elements.
void launch_scan(const LaunchCommon& lc, const int64_t* in, int64_t* out, int64_t n,
                 int64_t* scratch) {
  if (n <= 0) return;
  const int64_t nb = (n + 1023) / 1024;
  ++*lc.launches;
  k_scan_block<<<(unsigned)nb, 1024, 0, lc.stream>>>(in, out, n, scratch);
  if (nb > 1) {
    launch_scan(lc, scratch, scratch + nb, nb, scratch + 2 * nb);
    ++*lc.launches;
    k_scan_add<<<(unsigned)nb, 1024, 0, lc.stream>>>(out, n, scratch + nb);
  }
}

bool launch_rule_moments(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                         int modes, const int32_t* qv, const int32_t* qn, const KernelParams& kp,
                         void* out_smooth, void* out_ann, int form) {
  return dispatch<RuleMomL>(d, lc, plist, count, dv, modes, qv, qn, kp, out_smooth, out_ann,
                            form);
}
bool launch_farorder(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                     const KernelParams& kp, double eps, int m_max, double normV, const double* dirs,
                     int ndirs, void* scratch, int grid, int32_t* q, int32_t* qn, int* sched) {
  return dispatch<FarOrderL>(d, lc, plist, count, dv, kp, eps, m_max, normV, dirs, ndirs, scratch,
                             grid, q, qn, sched);
}
bool launch_adaptive(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                     const KernelParams& kp, double eps, double normV, int leaf_order, int max_depth,
                     const void* I_smooth, void* I_near, int32_t* leaves, void* work, int64_t stride,
                     int A_max, int levels, int grid, int* status, int* sched, int form,
                     const int64_t* gofs, int gsz) {
  return dispatch<AdaptiveL>(d, lc, plist, count, dv, kp, eps, normV, leaf_order, max_depth,
                             I_smooth, I_near, leaves, work, stride, A_max, levels, grid, status,
                             sched, form, gofs, gsz);
}

// Groups of at most gsz adaptive targets per listed patch: ng[b] = ceil(A_b / gsz) for
// b < count and ng[count] = 0, so that the exclusive scan of the count + 1 entries (gofs)
// ends with the number of groups.
__global__ void k_group_counts(const int* __restrict__ plist, int count,
                               const int64_t* __restrict__ ad_ptr, int gsz, int64_t* __restrict__ ng) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= count; b += gridDim.x * blockDim.x) {
    int64_t g = 0;
    if (b < count) {
      const int j = plist[b];
      g = (ad_ptr[j + 1] - ad_ptr[j] + gsz - 1) / gsz;
    }
    ng[b] = g;
  }
}

void launch_group_offsets(const LaunchCommon& lc, const int* plist, int count, const int64_t* ad_ptr,
                          int gsz, int64_t* ng, int64_t* gofs, int64_t* scratch) {
  const int blocks = (count + 1 + 255) / 256;
  ++*lc.launches;
  k_group_counts<<<blocks < lc.num_sms * 4 ? blocks : lc.num_sms * 4, 256, 0, lc.stream>>>(
      plist, count, ad_ptr, gsz, ng);
  launch_scan(lc, ng, gofs, count + 1, scratch);
}
bool launch_self(int d, const LaunchCommon& lc, const Dev& dv, const int32_t* deg,
                 const KernelParams& kp, int order, void* out) {
  return dispatch<SelfL>(d, lc, dv, deg, kp, order, out);
}
bool launch_tgt_normals(int d, const LaunchCommon& lc, const Dev& dv, const int32_t* deg,
                        const double* user, bool do_off, double* out) {
  return dispatch<TgtNormalsL>(d, lc, dv, deg, user, do_off, out);
}
bool launch_v2c(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                const double* Vt, const void* In, const void* Is, const void* InS,
                double* val) {
  return dispatch<V2cL>(d, lc, plist, count, dv, Vt, In, Is, InS, val);
}
bool launch_far_src(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                    const double* Vt, const int32_t* qv, const int64_t* src_off, const void* sigma,
                    double* src, int64_t n_over, const KernelParams& kp, bool fold) {
  return dispatch<FarSrcL>(d, lc, plist, count, dv, Vt, qv, src_off, sigma, src, n_over, kp, fold);
}
void launch_far_sum(const LaunchCommon& lc, const double* tgt, int64_t NT, const double* src,
                    int64_t n_over, const KernelParams& kp, const int32_t* tpatch,
                    const int64_t* src_off, const int32_t* tgroup, const GroupParams* grp,
                    const int64_t* gsrc, const double* tnrm, void* out, bool fold) {
  const int64_t g = (NT + kThreads - 1) / kThreads;
  if (g <= 0) return;
  ++*lc.launches;
  k_far_sum<<<(unsigned)g, kThreads, 0, lc.stream>>>(tgt, NT, src, n_over, kp, tpatch, src_off,
                                                     tgroup, grp, gsrc, tnrm, (cplx*)out, fold);
}
void launch_widen_c64(const LaunchCommon& lc, const void* in, int64_t n, void* out) {
  if (n <= 0) return;
  const int64_t b = (n + 255) / 256;
  ++*lc.launches;
  k_widen_c64<<<(unsigned)(b < lc.num_sms * 8 ? b : lc.num_sms * 8), 256, 0, lc.stream>>>(
      (const float2*)in, n, (cplx*)out);
}
void launch_csr_apply(const LaunchCommon& lc, const int64_t* row_ptr, const int32_t* col,
                      const double* val, const void* sigma, const int64_t* tnode, int64_t NT,
                      double jump, void* out) {
  const int g = lc.num_sms * 8;
  ++*lc.launches;
  k_csr_apply<<<g, 256, 0, lc.stream>>>(row_ptr, col, val, (const cplx*)sigma, tnode, NT, jump,
                                        (cplx*)out);
}

// Resident blocks per SM of k_adaptive<d> (the persistent grid is this times the SM count).
int adaptive_blocks_per_sm(int d) {
  int nb = 1;
  dispatch<BlocksL>(d, &nb);
  return nb;
}

}  // namespace lcq
