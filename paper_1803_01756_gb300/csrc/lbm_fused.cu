// Fused lattice update, one launch per step: the single-lattice kernel, its
// tiling and its launch.  The per-tile sweep is in lbm_fused_tile.cuh.
#include "lbm_fused_tile.cuh"

namespace lbm {

namespace {

template <bool YW, bool XO, bool TH, bool MP, class ST>
__global__ void __launch_bounds__(FNT, LBM_FUSED_MIN_CTAS)
    k_fused_step(DevParams p, const typename ST::T *__restrict__ gs,
                 typename ST::T *__restrict__ gout, const float *__restrict__ Tin,
                 float *__restrict__ Tout, unsigned *status,
                 const StepScalars *__restrict__ sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmem &S = *reinterpret_cast<FusedSmem *>(smem_raw);
  // strips and row chunks of nearly equal size (they differ by at most one column or row)
  const int X0 = (int)(((long long)blockIdx.x * p.nx) / gridDim.x);
  const int X1 = (int)(((long long)(blockIdx.x + 1) * p.nx) / gridDim.x);
  const int Y0 = (int)(((long long)blockIdx.y * p.ny) / gridDim.y);
  const int ye = (int)(((long long)(blockIdx.y + 1) * p.ny) / gridDim.y);
  // the update's boundary scalars, read where used (registers are at the launch bound)
  __shared__ StepScalars ssc;
  if (threadIdx.x == 0) ssc = *sc;
  __syncthreads();
  fused_tile<YW, XO, TH, MP, ST, 2>(p, p, gs, gout, Tin, Tout, status, ssc, X0, X1 - X0, Y0, ye,
                                    S);
}

}  // namespace

// 32-bit element offsets cover all nine population planes
bool fused_supported(const DevParams &p) {
  return p.nx >= 1 && p.ny >= 1 && 9LL * p.plane + p.pitch < 2147483647LL;
}

namespace {

template <class ST>
using FusedFn = void (*)(DevParams, const typename ST::T *, typename ST::T *, const float *,
                         float *, unsigned *, const StepScalars *);

template <class ST>
FusedFn<ST> fused_variant(const DevParams &p) {
  static const FusedFn<ST> table[16] = {
      k_fused_step<false, false, false, false, ST>, k_fused_step<false, false, false, true, ST>,
      k_fused_step<false, false, true, false, ST>,  k_fused_step<false, false, true, true, ST>,
      k_fused_step<false, true, false, false, ST>,  k_fused_step<false, true, false, true, ST>,
      k_fused_step<false, true, true, false, ST>,   k_fused_step<false, true, true, true, ST>,
      k_fused_step<true, false, false, false, ST>,  k_fused_step<true, false, false, true, ST>,
      k_fused_step<true, false, true, false, ST>,   k_fused_step<true, false, true, true, ST>,
      k_fused_step<true, true, false, false, ST>,   k_fused_step<true, true, false, true, ST>,
      k_fused_step<true, true, true, false, ST>,    k_fused_step<true, true, true, true, ST>};
  const int k = (p.y_walls ? 8 : 0) | (p.x_open ? 4 : 0) | (p.thermal ? 2 : 0) |
                (p.multiphase ? 1 : 0);
  return table[k];
}

template <class ST>
cudaError_t prepare(const DevParams &p, int *occ) {
  const FusedFn<ST> fn = fused_variant<ST>(p);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(FusedSmem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, FNT, sizeof(FusedSmem));
}

template <class ST>
cudaError_t launch_t(const DevParams &p, const void *gs, void *gout, const float *Tin, float *Tout,
                     unsigned *status, const StepScalars *sc, FusedTiling tl, cudaStream_t s) {
  // ceil(nx / W) strips of at most W columns and ceil(ny / H) chunks of at most H rows
  dim3 grid((p.nx + tl.W - 1) / tl.W, (p.ny + tl.H - 1) / tl.H);
  fused_variant<ST>(p)<<<grid, FNT, sizeof(FusedSmem), s>>>(
      p, static_cast<const typename ST::T *>(gs), static_cast<typename ST::T *>(gout), Tin, Tout,
      status, sc);
  return cudaGetLastError();
}

}  // namespace

int fused_max_width() { return FW; }

FusedTiling fused_tiling(const DevParams &p, int storage, int device) {
  FusedTiling best{0, 0};
  int sms = 0, occ = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return best;
  cudaError_t e = storage == STORAGE_BF16  ? prepare<StoreBF16>(p, &occ)
                  : storage == STORAGE_F16 ? prepare<StoreF16>(p, &occ)
                                           : prepare<StoreF32>(p, &occ);
  if (e != cudaSuccess || occ < 1) return best;
  // Widest strips (fewest halo columns), then the row-chunk height H with the shortest
  // estimated launch time over one wave of resident CTAs.  Every CTA sweeps H + 15 row
  // steps, and a row step takes longer the more CTAs share the SM: one CTA alone is bound
  // by the latency of the row step, four share the SM's issue slots.  kStep is the
  // measured time of one row step with k CTAs per SM, relative (200 x 50, 1024 x 128 and
  // 4096 x 512 channels, FP32); equal-work tilings with narrower strips or two waves were
  // 2-35 % slower on 4096 x 512.  A small lattice thus gets short chunks spread over
  // idle SMs (1 row on 200 x 50, 2x the rate of 16-row chunks), a large one one wave
  // of tall chunks.
  static const double kStep[5] = {0.0, 0.85, 0.97, 1.42, 1.64};
  const long long slots = (long long)sms * occ;
  const int strips = (p.nx + FW - 1) / FW;
  long long max_chunks = slots / strips;
  if (max_chunks < 1) max_chunks = 1;
  if (max_chunks > p.ny) max_chunks = p.ny;
  int H = p.ny;
  double best_cost = -1.0;
  for (long long c = 1; c <= max_chunks; c++) {
    const int h = (int)((p.ny + c - 1) / c);
    const long long tiles = (long long)strips * ((p.ny + h - 1) / h);
    const long long k = (tiles + sms - 1) / sms;  // CTAs per SM
    const double step = k <= 4 ? kStep[k] : kStep[4] * (double)k / 4.0;
    const double cost = (h + 15) * step;
    if (best_cost < 0.0 || cost < best_cost) {  // ties keep the taller chunk
      best_cost = cost;
      H = h;
    }
  }
  best = FusedTiling{FW, H};
  return best;
}

cudaError_t launch_fused(const DevParams &p, int storage, const void *gs, void *gout,
                         const float *Tin, float *Tout, unsigned *status, const StepScalars *sc,
                         FusedTiling tl, cudaStream_t s) {
  if (tl.H < 1 || tl.W < 1 || tl.W > FW) return cudaErrorInvalidValue;
  switch (storage) {
    case STORAGE_BF16: return launch_t<StoreBF16>(p, gs, gout, Tin, Tout, status, sc, tl, s);
    case STORAGE_F16: return launch_t<StoreF16>(p, gs, gout, Tin, Tout, status, sc, tl, s);
    default: return launch_t<StoreF32>(p, gs, gout, Tin, Tout, status, sc, tl, s);
  }
}

}  // namespace lbm
