// Launchers of the degree-templated kernels, declared for every degree; their definitions
// (lcq_kernels.cuh, lcq_adjoint.cuh) are instantiated one degree per translation unit in
// lcq_deg.cu, and lcq_kernels.cu / lcq_adjoint.cu dispatch to them by degree.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lcq_internal.h"
#include "lcq_launch.h"

namespace lcq {

template <int D>
struct GeomL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                  const double* xyz, int64_t N, const double* Vt, const double* nodes, double eta_p,
                  double eta1_p, double* coef, double* cen, double* rad, double* dj, double* eta,
                  double* eta1, int* status);
};

template <int D>
struct RuleMomL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv, int modes,
                  const int32_t* qv, const int32_t* qn, const KernelParams& kp, void* out_smooth,
                  void* out_ann, int form);
};

template <int D>
struct FarOrderL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, double eps, int m_max, double normV, const double* dirs,
                  int ndirs, void* scratch, int grid, int32_t* q, int32_t* qn, int* sched);
};

template <int D>
struct AdaptiveL {
  static int blocks_per_sm();
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, double eps, double normV, int leaf_order, int max_depth,
                  const void* I_smooth, void* I_near, int32_t* leaves, void* work,
                  int64_t stride, int A_max, int levels, int grid, int* status, int* sched,
                  int form, const int64_t* gofs, int gsz);
};

template <int D>
struct SelfL {
  static void run(const LaunchCommon& lc, const Dev& dv, const int32_t* deg, const KernelParams& kp,
                  int order, void* out);
};

template <int D>
struct TgtNormalsL {
  static void run(const LaunchCommon& lc, const Dev& dv, const int32_t* deg, const double* user,
                  bool do_off, double* out);
};

template <int D>
struct V2cL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const double* Vt, const void* In, const void* Is, const void* InS,
                  double* val);
};

template <int D>
struct FarSrcL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const double* Vt, const int32_t* qv, const int64_t* src_off, const void* sigma,
                  double* src, int64_t n_over, const KernelParams& kp, bool fold);
};

template <int D>
struct ShatL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                  const double* Vt, const void* sigma, void* shat);
};

template <int D>
struct GradRulesL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, const int32_t* qn, const int64_t* src_off, int64_t n_over,
                  const double* tg, const void* g, const void* shat, double* M);
};

template <int D>
struct AdaptiveGradL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const KernelParams& kp, double eps, double normV, int leaf_order, int max_depth,
                  const void* I_smooth, void* I_near, int32_t* leaves, void* work, int64_t stride,
                  int A_max, int levels, int grid, int* status, int* sched, int form,
                  const GradArgs& ga);
};

template <int D>
struct GradV2cL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const int64_t* node_off,
                  const double* Vt, const double* M, int64_t N, double* out);
};

template <int D>
struct AdjPatchL {
  static void run(const LaunchCommon& lc, const int* plist, int count, const Dev& dv,
                  const double* Vt, const int64_t* src_off, const void* z, const double* val,
                  const void* g, double jump, void* out);
};

// Uploads the per-translation-unit constants (Koornwinder normalizations, Jacobi
// coefficients, basis bounds, sincos table) of degree D's translation unit.
template <int D>
cudaError_t upload_deg_constants(cudaStream_t st);

}  // namespace lcq
