// Fused lattice update, one launch per step: the single-lattice kernel and its
// launch, templated on the threads per CTA (NT) and the lattice columns per thread
// (CPT).  lbm_fused.cu instantiates CPT = 1 and holds the tiling, lbm_fused_c2.cu
// instantiates CPT = 2; the per-tile sweep is in lbm_fused_tile.cuh.
#pragma once
#include "lbm_fused_tile.cuh"

namespace lbm {

namespace {

template <bool YW, bool XO, bool TH, bool MP, class ST, int NT, int CPT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_fused_step(DevParams p, const typename ST::T *__restrict__ gs,
                 typename ST::T *__restrict__ gout, const float *__restrict__ Tin,
                 float *__restrict__ Tout, unsigned *status,
                 const StepScalars *__restrict__ sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmemT<NT * CPT> &S = *reinterpret_cast<FusedSmemT<NT * CPT> *>(smem_raw);
  // strips and row chunks of nearly equal size (they differ by at most one row, and by
  // at most one column, or two with CPT = 2, whose strips start at even columns)
  int X0, X1;
  if constexpr (CPT == 1) {
    X0 = (int)(((long long)blockIdx.x * p.nx) / gridDim.x);
    X1 = (int)(((long long)(blockIdx.x + 1) * p.nx) / gridDim.x);
  } else {
    const long long m = (p.nx + 1) / 2;
    X0 = 2 * (int)(((long long)blockIdx.x * m) / gridDim.x);
    X1 = min(p.nx, 2 * (int)(((long long)(blockIdx.x + 1) * m) / gridDim.x));
  }
  const int Y0 = (int)(((long long)blockIdx.y * p.ny) / gridDim.y);
  const int ye = (int)(((long long)(blockIdx.y + 1) * p.ny) / gridDim.y);
  // the update's boundary scalars, read where used
  __shared__ StepScalars ssc;
  // Launched as a programmatic dependent of the previous update (see launch_t), the CTAs
  // of this update start while the previous grid drains: they allow the next update's
  // launch at once and read their boundary scalars (staged before the chunk), then wait
  // for the previous grid to complete and its writes to be visible before touching the
  // populations and temperatures it wrote or read.  Launched otherwise, both are no-ops.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (threadIdx.x == 0) ssc = *sc;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  fused_tile<YW, XO, TH, MP, ST, (CPT == 1 ? 2 : 1), NT, CPT>(p, p, gs, gout, Tin, Tout, status,
                                                             ssc, X0, X1 - X0, Y0, ye, S);
}

template <class ST>
using FusedFn = void (*)(DevParams, const typename ST::T *, typename ST::T *, const float *,
                         float *, unsigned *, const StepScalars *);

// MFULL: resident CTAs per SM the registers are sized for in the variants with the energy
// equation and the pseudopotential forces (TH and MP); MREST: in the others
template <class ST, int NT, int CPT, int MFULL, int MREST>
FusedFn<ST> fused_variant(const DevParams &p) {
#define KF(a, b, c, d) k_fused_step<a, b, c, d, ST, NT, CPT, ((c) && (d) ? MFULL : MREST)>
  static const FusedFn<ST> table[16] = {
      KF(false, false, false, false), KF(false, false, false, true), KF(false, false, true, false),
      KF(false, false, true, true),   KF(false, true, false, false), KF(false, true, false, true),
      KF(false, true, true, false),   KF(false, true, true, true),   KF(true, false, false, false),
      KF(true, false, false, true),   KF(true, false, true, false),  KF(true, false, true, true),
      KF(true, true, false, false),   KF(true, true, false, true),   KF(true, true, true, false),
      KF(true, true, true, true)};
#undef KF
  const int k = (p.y_walls ? 8 : 0) | (p.x_open ? 4 : 0) | (p.thermal ? 2 : 0) |
                (p.multiphase ? 1 : 0);
  return table[k];
}

// Sets the kernel's shared-memory attribute and returns its resident CTAs per SM.
template <class ST, int NT, int CPT, int MFULL, int MREST>
cudaError_t prepare_t(const DevParams &p, int *occ) {
  const FusedFn<ST> fn = fused_variant<ST, NT, CPT, MFULL, MREST>(p);
  const int smem = (int)sizeof(FusedSmemT<NT * CPT>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, NT, smem);
}

// M32: resident CTAs per SM the registers are sized for in the FP32 variants with the
// energy equation and the pseudopotential forces; M16: in every other variant
template <int NT, int CPT, int M32, int M16>
cudaError_t prepare_any(const DevParams &p, int storage, int *occ) {
  return storage == STORAGE_BF16  ? prepare_t<StoreBF16, NT, CPT, M16, M16>(p, occ)
         : storage == STORAGE_F16 ? prepare_t<StoreF16, NT, CPT, M16, M16>(p, occ)
                                  : prepare_t<StoreF32, NT, CPT, M32, M16>(p, occ);
}

// pdl: the launch may begin before the previous kernel on the stream completes (programmatic
// stream serialization; the kernel waits for it before touching the lattice state)
template <class ST, int NT, int CPT, int MFULL, int MREST>
cudaError_t launch_t(const DevParams &p, const void *gs, void *gout, const float *Tin, float *Tout,
                     unsigned *status, const StepScalars *sc, dim3 grid, bool pdl,
                     cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sizeof(FusedSmemT<NT * CPT>);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fused_variant<ST, NT, CPT, MFULL, MREST>(p), p,
                            static_cast<const typename ST::T *>(gs),
                            static_cast<typename ST::T *>(gout), Tin, Tout, status, sc);
}

template <int NT, int CPT, int M32, int M16>
cudaError_t launch_any(const DevParams &p, int storage, const void *gs, void *gout,
                       const float *Tin, float *Tout, unsigned *status, const StepScalars *sc,
                       dim3 grid, bool pdl, cudaStream_t s) {
  switch (storage) {
    case STORAGE_BF16:
      return launch_t<StoreBF16, NT, CPT, M16, M16>(p, gs, gout, Tin, Tout, status, sc, grid, pdl,
                                                     s);
    case STORAGE_F16:
      return launch_t<StoreF16, NT, CPT, M16, M16>(p, gs, gout, Tin, Tout, status, sc, grid, pdl,
                                                    s);
    default:
      return launch_t<StoreF32, NT, CPT, M32, M16>(p, gs, gout, Tin, Tout, status, sc, grid, pdl,
                                                    s);
  }
}

}  // namespace

}  // namespace lbm
