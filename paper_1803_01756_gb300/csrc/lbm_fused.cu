// Fused lattice update: one launch per step (not yet available).
#include "lbm_internal.h"

namespace lbm {

bool fused_supported(const DevParams &) { return false; }

cudaError_t launch_fused(const DevParams &, const float *, float *, const float *, float *,
                         unsigned *, StepScalars, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace lbm
