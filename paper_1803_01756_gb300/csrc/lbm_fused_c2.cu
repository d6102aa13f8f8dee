// The fused single-lattice kernel with two lattice columns per thread (CPT = 2):
// instantiation and launch (the tiling is chosen in lbm_fused.cu).
#include "lbm_fused_step.cuh"

#ifndef LBM_FUSED_C2_THREADS
#define LBM_FUSED_C2_THREADS 128
#endif

namespace lbm {

namespace {
constexpr int C2T = LBM_FUSED_C2_THREADS;
constexpr int C2B = 256 / LBM_FUSED_C2_THREADS;  // resident CTAs per SM the registers allow
}  // namespace

int fused_c2_threads() { return C2T; }

cudaError_t fused_c2_prepare(const DevParams &p, int storage, int *occ) {
  return prepare_any<C2T, 2, C2B, C2B>(p, storage, occ);
}

cudaError_t fused_c2_launch(const DevParams &p, int storage, const void *gs, void *gout,
                            const float *Tin, float *Tout, unsigned *status, const StepScalars *sc,
                            dim3 grid, cudaStream_t s) {
  return launch_any<C2T, 2, C2B, C2B>(p, storage, gs, gout, Tin, Tout, status, sc, grid, false,
                                      s);
}

}  // namespace lbm
