// One patch degree's instantiations of the degree-templated kernels and launchers
// (lcq_kernels.cuh, lcq_adjoint.cuh), built once per degree with -DLCQ_DEG=d so that the
// degrees compile in parallel; lcq_kernels.cu and lcq_adjoint.cu dispatch to them.
#include "lcq_adjoint.cuh"
#include "lcq_kernels.cuh"

#ifndef LCQ_DEG
#error "LCQ_DEG must be defined (1..10)"
#endif

namespace lcq {
template struct GeomL<LCQ_DEG>;
template struct RuleMomL<LCQ_DEG>;
template struct FarOrderL<LCQ_DEG>;
template struct AdaptiveL<LCQ_DEG>;
template struct SelfL<LCQ_DEG>;
template struct TgtNormalsL<LCQ_DEG>;
template struct V2cL<LCQ_DEG>;
template struct FarSrcL<LCQ_DEG>;
template cudaError_t upload_deg_constants<LCQ_DEG>(cudaStream_t);
template struct ShatL<LCQ_DEG>;
template struct GradRulesL<LCQ_DEG>;
template struct AdaptiveGradL<LCQ_DEG>;
template struct GradV2cL<LCQ_DEG>;
template struct AdjPatchL<LCQ_DEG>;
}  // namespace lcq
