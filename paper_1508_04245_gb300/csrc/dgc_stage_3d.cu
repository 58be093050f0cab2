// Stage-kernel instantiations for tetrahedra, k = 1..5, FP64 and FP32 contractions.
#include "dgc_kernels.h"
#include "dgc_stage.cuh"

namespace dgc {

cudaError_t launch_stage_3d(int K, bool fp32, const StageArgs* a, cudaStream_t s) {
  switch (K) {
#define DGC_CASE(k) \
  case k: return fp32 ? launch_stage_t<3, k, float>(a, s) : launch_stage_t<3, k, double>(a, s);
    DGC_CASE(1) DGC_CASE(2) DGC_CASE(3) DGC_CASE(4) DGC_CASE(5)
#undef DGC_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgc
