// Kernel launchers of liblcq (defined in lcq_kernels.cu, called by lcq_api.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lcq_internal.h"

namespace lcq {

struct LaunchCommon {
  cudaStream_t stream;
  int num_sms;
  long long* launches;  // incremented once per kernel launch
};

// Read-only device view of a near-list object plus tables, passed by value to kernels.
struct Dev {
  const double* coef;
  const int64_t* node_off;
  const double* cen;
  const double* rad;
  const double* dj;
  const double* eta;
  const double* eta1;
  const double* tgt;
  int64_t NT;
  const int32_t* tpatch;
  const int32_t* tlnode;
  const int64_t* pair_ptr;
  const int32_t* pair_tgt;
  const double* pair_d2;
  const int64_t* pair_csr;
  const int64_t* ad_ptr;
  const int32_t* ad_pair;
  const int64_t* an_ptr;
  const int32_t* an_pair;
  const int64_t* self_ptr;
  const int32_t* self_tgt;
  const int64_t* self_csr;
  int64_t n_self;
  const int32_t* q;
  // batches of independent surfaces: surface of each patch and its physics (null: one
  // surface whose physics come from the launch arguments)
  const int32_t* pgroup;
  const GroupParams* grp;
  // unit target normals, SoA [3][NT] (S' only, else null)
  const double* tnrm;
  // tables
  const int* roff;
  const double* ru;
  const double* rv;
  const double* rw;
  const int* gl_off;
  const double* gl_x;
  const double* gl_w;
  const double* nodes_uv[kMaxDeg + 1];
  const double* duv[kMaxDeg + 1];  // derivative projections per degree: Du [n][n_{d-1}], then Dv
  long long* counters;
  int* status;
  int ldI;  // row stride (complex entries) of the pair/self moment buffers
};

// Adjoint inputs and accumulator of the adaptive kernel's gradient mode: g (complex
// [NT], interleaved) the upstream gradient of the targets, shat (complex [N]) the
// Koornwinder coefficients V sigma_j of the density in each patch's node slots, M
// (double [N][3]) dL/dx_nm in the same slots (added to).
struct GradArgs {
  const double* g;
  const double* shat;
  double* M;
};

struct NearArgs {
  const double* tgt;
  int64_t NT;
  const double* cen;
  const double* rad;
  const double* eta;
  const double* eta1;
  const int32_t* pgroup;  // null: one surface
  const int32_t* tgroup;
};

cudaError_t upload_constants(cudaStream_t st);

bool launch_geom(int d, const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                 const double* xyz, int64_t N, const double* Vt, const double* nodes, double eta_p,
                 double eta1_p, double* coef, double* cen, double* rad, double* dj, double* eta,
                 double* eta1, int* status);
void launch_tgt_from_nodes(const LaunchCommon& lc, double* tgt, const int64_t* tnode, int64_t NT,
                           const double* xyz, int64_t N);
void launch_tgt_patch(const LaunchCommon& lc, const double* tgt, const int64_t* tnode, int64_t NT,
                      const int64_t* node_off, int64_t P, int64_t N, int32_t* tpatch,
                      int32_t* tlnode, int* status);
// Uniform grid over patch centroids: cell (i, j, k) holds centroids c with
// floor((c - lo) * inv_h) = (i, j, k); 1 / inv_h >= max eta_j R_j.
struct GridSpec {
  double lo[3];
  double inv_h;
  int nx, ny, nz;
};
// Surface of each patch (from the patch ranges) and of each target (kStBadGroup on a
// caller's value outside [0, G)).
void launch_groups(const LaunchCommon& lc, int64_t NT, const int32_t* tpatch,
                   const int64_t* gpatch_off, int G, const int32_t* user, int32_t* pgroup,
                   int32_t* tgroup, int* status);
void launch_grid_bounds(const LaunchCommon& lc, const NearArgs& a, int64_t P, double* out7);
void launch_cell_bins(const LaunchCommon& lc, const NearArgs& a, int64_t P, const GridSpec& g,
                      unsigned long long* cnt, int64_t* cell_ptr, unsigned long long* cursor,
                      int32_t* cell_patch, int64_t* scan_scratch);
void launch_row_count(const LaunchCommon& lc, const NearArgs& a, const GridSpec& g,
                      const int64_t* cell_ptr, const int32_t* cell_patch, const int32_t* tpatch,
                      const int32_t* deg, int64_t* row_np, int64_t* row_nnz);
void launch_row_fill(const LaunchCommon& lc, const NearArgs& a, const GridSpec& g,
                     const int64_t* cell_ptr, const int32_t* cell_patch, const int32_t* tpatch,
                     const int32_t* deg, const int64_t* node_off, const int64_t* rowp_ptr,
                     const int64_t* row_ptr, int32_t* tmp, int32_t* rowp_patch, int64_t* rowp_off,
                     int32_t* col, unsigned long long* npair, unsigned long long* nad,
                     unsigned long long* nself);
void launch_patch_fill(const LaunchCommon& lc, const NearArgs& a, const int32_t* tpatch, int64_t P,
                       const int64_t* pair_ptr, const int64_t* ad_ptr, const int64_t* an_ptr,
                       const int64_t* self_ptr, const int64_t* rowp_ptr, const int32_t* rowp_patch,
                       const int64_t* rowp_off, const int64_t* row_ptr, unsigned long long* pcur,
                       unsigned long long* scur, int32_t* ptmp, int32_t* stmp, int32_t* pair_tgt,
                       uint8_t* pair_ad, double* pair_d2, int64_t* pair_csr, int32_t* ad_pair,
                       int32_t* an_pair, int32_t* self_tgt, int64_t* self_csr);
void launch_scan(const LaunchCommon& lc, const int64_t* in, int64_t* out, int64_t n,
                 int64_t* scratch);
// modes: bit 0 the smooth rule qv into out_smooth, bit 1 the annulus rule qn into out_ann
bool launch_rule_moments(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                         int modes, const int32_t* qv, const int32_t* qn, const KernelParams& kp,
                         void* out_smooth, void* out_ann, int form = 0);
// sched: a device counter the launch zeroes and the blocks draw patches from
bool launch_farorder(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                     const KernelParams& kp, double eps, int m_max, double normV, const double* dirs,
                     int ndirs, void* scratch, int grid, int32_t* q, int32_t* qn, int* sched);
bool launch_adaptive(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                     const KernelParams& kp, double eps, double normV, int leaf_order, int max_depth,
                     const void* I_smooth, void* I_near, int32_t* leaves, void* work, int64_t stride,
                     int A_max, int levels, int grid, int* status, int* sched, int form = 0,
                     const int64_t* gofs = nullptr, int gsz = 0);
// gofs[count + 1]: exclusive scan of ceil(A_b / gsz) over the listed patches (work groups of
// at most gsz adaptive targets for launch_adaptive); ng[count + 1] and scratch as launch_scan.
void launch_group_offsets(const LaunchCommon& lc, const int* plist, int count, const int64_t* ad_ptr,
                          int gsz, int64_t* ng, int64_t* gofs, int64_t* scratch);
bool launch_self(int d, const LaunchCommon& lc, const Dev& dv, const int32_t* deg,
                 const KernelParams& kp, int order, void* out);
bool launch_v2c(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                const double* Vt, const void* In, const void* Is, const void* InS,
                double* val);
// fold: the sources carry the kernel constants (k_far_src), the far sum evaluates by
// kernel_eval_fold; only for real k and kinds S, D, CFIE with a real alpha (every surface's)
bool launch_far_src(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                    const double* Vt, const int32_t* qv, const int64_t* src_off, const void* sigma,
                    double* src, int64_t n_over, const KernelParams& kp = KernelParams{},
                    bool fold = false);
void launch_far_sum(const LaunchCommon& lc, const double* tgt, int64_t NT, const double* src,
                    int64_t n_over, const KernelParams& kp, const int32_t* tpatch,
                    const int64_t* src_off, const int32_t* tgroup, const GroupParams* grp,
                    const int64_t* gsrc, const double* tnrm, void* out, bool fold = false);
void launch_widen_c64(const LaunchCommon& lc, const void* in, int64_t n, void* out);
void launch_csr_apply(const LaunchCommon& lc, const int64_t* row_ptr, const int32_t* col,
                      const double* val, const void* sigma, const int64_t* tnode, int64_t NT,
                      double jump, void* out);
int adaptive_blocks_per_sm(int d);

// Unit target normals for S' (SoA [3][NT]): the chart normal at the node of an on-surface
// target of degree d; with do_off also the normalized user[t] of off-surface targets.
bool launch_tgt_normals(int d, const LaunchCommon& lc, const Dev& dv, const int32_t* deg,
                        const double* user, bool do_off, double* out);

// Adjoint (lcq_adjoint.cu).
cudaError_t upload_constants_adjoint(cudaStream_t st);
bool launch_shat(int d, const LaunchCommon& lc, const int* plist, int count,
                 const int64_t* node_off, const double* Vt, const void* sigma, void* shat);
void launch_far_grad_sum(const LaunchCommon& lc, const Dev& dv, int64_t P, const double* src,
                         int64_t n_over, const int64_t* src_off, const KernelParams& kp,
                         const int32_t* tgroup, const void* g, double* tg);
bool launch_grad_rules(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                       const KernelParams& kp, const int32_t* qn, const int64_t* src_off,
                       int64_t n_over, const double* tg, const void* g, const void* shat,
                       double* M);
bool launch_adaptive_grad(int d, const LaunchCommon& lc, const int* plist, int count,
                          const Dev& dv, const KernelParams& kp, double eps, double normV,
                          int leaf_order, int max_depth, const void* I_smooth, void* I_near,
                          int32_t* leaves, void* work, int64_t stride, int A_max, int levels,
                          int grid, int* status, int* sched, int form, const GradArgs& ga);
bool launch_grad_v2c(int d, const LaunchCommon& lc, const int* plist, int count,
                     const int64_t* node_off, const double* Vt, const double* M, int64_t N,
                     double* out);
void launch_far_sum_T(const LaunchCommon& lc, const Dev& dv, int64_t P, const double* src,
                      int64_t n_over, const int64_t* src_off, const KernelParams& kp,
                      const int32_t* tgroup, const void* g, void* z);
bool launch_adj_patch(int d, const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                      const double* Vt, const int64_t* src_off, const void* z, const double* val,
                      const void* g, double jump, void* out);

}  // namespace lcq
