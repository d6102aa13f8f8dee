// Kernel launchers shared by the host runtime (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include "lbm_common.cuh"

namespace lbm {

// population storage codes (values of lbm_params_t.storage)
enum : int { STORAGE_F32 = 0, STORAGE_BF16 = 1, STORAGE_F16 = 2 };
inline int storage_bytes(int storage) { return storage == STORAGE_F32 ? 4 : 2; }

// split path: three launches per update; population pointers point at `storage` elements
cudaError_t launch_density_psi(const DevParams &p, int storage, const void *gs, const float *Tdev,
                               float *rho, float *psi, unsigned *status, StepScalars sc,
                               cudaStream_t s);
cudaError_t launch_collide(const DevParams &p, int storage, const void *gs, void *gout,
                           const float *Tdev, const float *psi, float *ux, float *uy,
                           unsigned *status, StepScalars sc, bool write_populations,
                           cudaStream_t s);
cudaError_t launch_energy(const DevParams &p, const float *Tin, float *Tout, const float *rho,
                          const float *ux, const float *uy, unsigned *status, StepScalars sc,
                          cudaStream_t s);

// one lattice of a batched fused launch (device-resident table entry)
struct BatchChannel {
  DevParams p;
  const void *gs;  // populations read this step
  void *gout;      // populations written this step
  const float *Tin;
  float *Tout;
  unsigned *status;
  int W, H, strips;  // tiling of this lattice
  int tile_begin;    // index of its first tile in the work-list
};

// fused path: one launch per update; sc points to the update's scalars in device memory
struct FusedTiling {
  int W;    // output columns per CTA (at most fused_max_width(cpt))
  int H;    // output rows per CTA
  int cpt;  // lattice columns per thread: 1 or 2
  int pdl;  // launch each update as a programmatic dependent of the previous one
};
cudaError_t launch_fused(const DevParams &p, int storage, const void *gs, void *gout,
                         const float *Tin, float *Tout, unsigned *status, const StepScalars *sc,
                         FusedTiling tiling, cudaStream_t s);
bool fused_supported(const DevParams &p);
// tiling for one wave of resident CTAs on this device with cpt columns per thread
// ({0, 0, cpt} on failure); also sets the kernel's shared-memory attribute
FusedTiling fused_tiling(const DevParams &p, int storage, int device, int cpt);
// output columns of one CTA of the fused kernel with cpt columns per thread
int fused_max_width(int cpt);
// the CPT = 2 kernel (lbm_fused_c2.cu): threads per CTA, occupancy, launch on a grid of
// (strips, row chunks)
int fused_c2_threads();
cudaError_t fused_c2_prepare(const DevParams &p, int storage, int *occ);
cudaError_t fused_c2_launch(const DevParams &p, int storage, const void *gs, void *gout,
                            const float *Tin, float *Tout, unsigned *status, const StepScalars *sc,
                            dim3 grid, cudaStream_t s);

// batched fused path: a persistent grid of `grid` CTAs walks the tiles of nch
// lattices (all with the modes of `mode` and storage `storage`) with cpt lattice columns
// per thread (2: even tile widths); counter: two ints, zero before the first launch, left
// at zero by every launch
cudaError_t launch_fused_batch(const DevParams &mode, int storage, int cpt, const BatchChannel *ch,
                               int nch, const StepScalars *sc, int ntiles, int *counter, int grid,
                               cudaStream_t s);
// resident CTAs of the batched kernel with cpt columns per thread on this device (0 on
// failure, and for cpt = 2 in modes without the energy equation or the pseudopotential)
int fused_batch_grid(const DevParams &mode, int storage, int cpt, int device);
// output columns of one CTA of the batched kernel with cpt columns per thread
int fused_batch_width(int cpt);

// two-pass path (lbm_twopass.cu): pass A streams and collides (and, with the energy
// equation on, writes rho and u of every node), pass B advances T with the RK4 stages;
// Ha and Hb are the row-chunk heights of the two launches
struct TwoPassTiling {
  int Ha, Hb;
};
// chunk heights for this device ({0, 0} on failure); also sets pass B's shared-memory
// attribute
TwoPassTiling twopass_tiling(const DevParams &p, int storage, int device);
int twopass_width_a();  // output columns of a pass-A CTA
int twopass_width_b();  // output columns of a pass-B CTA
cudaError_t launch_stream_collide(const DevParams &p, int storage, const void *gs, void *gout,
                                  const float *Tin, float *rho, float *ux, float *uy,
                                  unsigned *status, const StepScalars *sc, int Ha,
                                  cudaStream_t s);
cudaError_t launch_energy_rk4(const DevParams &p, const float *Tin, float *Tout, const float *rho,
                              const float *ux, const float *uy, unsigned *status,
                              const StepScalars *sc, int Hb, cudaStream_t s);

// set-up and reductions
cudaError_t launch_init(const DevParams &p, int storage, const double *rho0, void *gout,
                        cudaStream_t s);
cudaError_t launch_mass_heat(const DevParams &p, const float *rho, const float *Tdev,
                             double T_ref, double Cv, double *partials, int nblocks,
                             double *out, cudaStream_t s);
int mass_heat_blocks(const DevParams &p);
// field conversion between the pitched FP32 planes and the caller's [ny][nx] FP64 layout:
// dst[y][x] = src[y * pitch + x] + add, and (T may be NULL for a zero deviation)
// dst[y * pitch + x] = T[y][x] - T_ref with zero padding columns
cudaError_t launch_unpitch(const float *src, int nx, int ny, int pitch, double add, double *dst,
                           cudaStream_t s);
cudaError_t launch_pitch_T(const double *T, int nx, int ny, int pitch, double T_ref, float *dst,
                           cudaStream_t s);

}  // namespace lbm
