// Stage-kernel instantiations for triangles, k = 1..6, FP64 and FP32 contractions.
#include "dgc_kernels.h"
#include "dgc_stage.cuh"

namespace dgc {

cudaError_t launch_stage_2d(int K, bool fp32, const StageArgs* a, cudaStream_t s) {
  switch (K) {
#define DGC_CASE(k) \
  case k: return fp32 ? launch_stage_t<2, k, float>(a, s) : launch_stage_t<2, k, double>(a, s);
    DGC_CASE(1) DGC_CASE(2) DGC_CASE(3) DGC_CASE(4) DGC_CASE(5) DGC_CASE(6)
#undef DGC_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgc
