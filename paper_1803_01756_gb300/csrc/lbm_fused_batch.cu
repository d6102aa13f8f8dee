// Batched fused update: one persistent launch per step over the tiles of many
// lattices.  The per-tile sweep is in lbm_fused_tile.cuh.
#include "lbm_fused_tile.cuh"

namespace lbm {

namespace {

// Persistent batched update: resident CTAs take tiles of many lattices from one
// work-list (largest lattices first), so uneven lattice sizes balance across the SMs.
// Block b starts with tile b (a batch with fewer tiles than resident CTAs is launched with
// one CTA per tile, which the hardware spreads over the SMs); later tiles come from an
// atomic counter.
// The last CTA to leave resets the counters.
// (Reading the bulk physics from a constant-bank copy when all lattices share it
// measured 2 % faster than the shared-memory copy used here, and a kernel holding
// both paths 12 % slower, so there is one path.)
template <bool YW, bool XO, bool TH, bool MP, class ST>
__global__ void __launch_bounds__(FNT, LBM_FUSED_MIN_CTAS)
    k_fused_batch(const BatchChannel *__restrict__ ch, int nch, const StepScalars *__restrict__ sc,
                  int ntiles, int *counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmem &S = *reinterpret_cast<FusedSmem *>(smem_raw);
  __shared__ DevParams sp;
  __shared__ int s_tile, s_ch;
  int tile = (int)blockIdx.x;  // thread 0: the CTA's next tile
  for (;;) {
    if (threadIdx.x == 0) {
      int k = 0;
      if (tile < ntiles) {
        int lo = 0, hi = nch - 1;  // last channel whose first tile <= tile
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (ch[mid].tile_begin <= tile) lo = mid;
          else hi = mid - 1;
        }
        k = lo;
      }
      s_tile = tile;
      s_ch = k;
    }
    __syncthreads();
    const int cur = s_tile;
    if (cur >= ntiles) break;
    const BatchChannel &C = ch[s_ch];
    {
      // the lattice parameters live in shared memory for the tile
      const int *src = reinterpret_cast<const int *>(&C.p);
      int *dst = reinterpret_cast<int *>(&sp);
      for (int i = threadIdx.x; i < (int)(sizeof(DevParams) / sizeof(int)); i += FNT) dst[i] = src[i];
    }
    __syncthreads();
    const int local = cur - C.tile_begin;
    const int bx = local % C.strips, by = local / C.strips;
    const int Y0 = by * C.H;
    const typename ST::T *gs = static_cast<const typename ST::T *>(C.gs);
    typename ST::T *gout = static_cast<typename ST::T *>(C.gout);
    fused_tile<YW, XO, TH, MP, ST, 1, FNT, 1>(sp, sp, gs, gout, C.Tin, C.Tout, C.status,
                                             sc[s_ch], bx * C.W, C.W, Y0,
                                             min(Y0 + C.H, sp.ny), S);
    __syncthreads();
    if (threadIdx.x == 0) tile = (int)gridDim.x + atomicAdd(&counter[0], 1);
  }
  if (threadIdx.x == 0 && atomicAdd(&counter[1], 1) == (int)gridDim.x - 1) {
    counter[0] = 0;
    counter[1] = 0;
  }
}

template <class ST>
using BatchFn = void (*)(const BatchChannel *, int, const StepScalars *, int, int *);

template <class ST>
BatchFn<ST> batch_variant(const DevParams &p) {
  static const BatchFn<ST> table[16] = {
      k_fused_batch<false, false, false, false, ST>, k_fused_batch<false, false, false, true, ST>,
      k_fused_batch<false, false, true, false, ST>,  k_fused_batch<false, false, true, true, ST>,
      k_fused_batch<false, true, false, false, ST>,  k_fused_batch<false, true, false, true, ST>,
      k_fused_batch<false, true, true, false, ST>,   k_fused_batch<false, true, true, true, ST>,
      k_fused_batch<true, false, false, false, ST>,  k_fused_batch<true, false, false, true, ST>,
      k_fused_batch<true, false, true, false, ST>,   k_fused_batch<true, false, true, true, ST>,
      k_fused_batch<true, true, false, false, ST>,   k_fused_batch<true, true, false, true, ST>,
      k_fused_batch<true, true, true, false, ST>,    k_fused_batch<true, true, true, true, ST>};
  const int k = (p.y_walls ? 8 : 0) | (p.x_open ? 4 : 0) | (p.thermal ? 2 : 0) |
                (p.multiphase ? 1 : 0);
  return table[k];
}

template <class ST>
int batch_grid_t(const DevParams &mode, int device) {
  int sms = 0, occ = 0;
  const BatchFn<ST> fn = batch_variant<ST>(mode);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(FusedSmem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, FNT, sizeof(FusedSmem)) !=
          cudaSuccess ||
      occ < 1)
    return 0;
  return sms * occ;
}

template <class ST>
cudaError_t launch_batch_t(const DevParams &mode, const BatchChannel *ch, int nch,
                           const StepScalars *sc, int ntiles, int *counter, int grid,
                           cudaStream_t s) {
  batch_variant<ST>(mode)<<<grid, FNT, sizeof(FusedSmem), s>>>(ch, nch, sc, ntiles, counter);
  return cudaGetLastError();
}

}  // namespace

int fused_batch_grid(const DevParams &mode, int storage, int device) {
  return storage == STORAGE_BF16  ? batch_grid_t<StoreBF16>(mode, device)
         : storage == STORAGE_F16 ? batch_grid_t<StoreF16>(mode, device)
                                  : batch_grid_t<StoreF32>(mode, device);
}

cudaError_t launch_fused_batch(const DevParams &mode, int storage, const BatchChannel *ch, int nch,
                               const StepScalars *sc, int ntiles, int *counter, int grid,
                               cudaStream_t s) {
  switch (storage) {
    case STORAGE_BF16: return launch_batch_t<StoreBF16>(mode, ch, nch, sc, ntiles, counter, grid, s);
    case STORAGE_F16: return launch_batch_t<StoreF16>(mode, ch, nch, sc, ntiles, counter, grid, s);
    default: return launch_batch_t<StoreF32>(mode, ch, nch, sc, ntiles, counter, grid, s);
  }
}

}  // namespace lbm
