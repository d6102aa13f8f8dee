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
template <bool YW, bool XO, bool TH, bool MP, class ST, int NT, int CPT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_fused_batch(const BatchChannel *__restrict__ ch, int nch, const StepScalars *__restrict__ sc,
                  int ntiles, int *counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmemT<NT * CPT> &S = *reinterpret_cast<FusedSmemT<NT * CPT> *>(smem_raw);
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
      for (int i = threadIdx.x; i < (int)(sizeof(DevParams) / sizeof(int)); i += NT) dst[i] = src[i];
    }
    __syncthreads();
    const int local = cur - C.tile_begin;
    const int bx = local % C.strips, by = local / C.strips;
    const int Y0 = by * C.H;
    const typename ST::T *gs = static_cast<const typename ST::T *>(C.gs);
    typename ST::T *gout = static_cast<typename ST::T *>(C.gout);
    // (C.W is even with two columns per thread, so every strip starts at an even column)
    fused_tile<YW, XO, TH, MP, ST, 1, NT, CPT>(sp, sp, gs, gout, C.Tin, C.Tout, C.status,
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

// two columns per thread: 128-thread CTAs, two per SM (the registers allow no more)
constexpr int B2T = 128;

template <class ST>
using BatchFn = void (*)(const BatchChannel *, int, const StepScalars *, int, int *);

// the kernel of a mode and column count; with two columns per thread only the modes with
// the energy equation and the pseudopotential forces are built (nullptr otherwise)
template <class ST>
BatchFn<ST> batch_variant(const DevParams &p, int cpt) {
#define KB(a, b, c, d)                                                                      \
  k_fused_batch<a, b, c, d, ST, FNT, 1,                                                     \
                std::is_same<ST, StoreF32>::value && (c) && (d) ? FMIN_F32 : FMIN_16>
  static const BatchFn<ST> table[16] = {
      KB(false, false, false, false), KB(false, false, false, true), KB(false, false, true, false),
      KB(false, false, true, true),   KB(false, true, false, false), KB(false, true, false, true),
      KB(false, true, true, false),   KB(false, true, true, true),   KB(true, false, false, false),
      KB(true, false, false, true),   KB(true, false, true, false),  KB(true, false, true, true),
      KB(true, true, false, false),   KB(true, true, false, true),   KB(true, true, true, false),
      KB(true, true, true, true)};
#undef KB
#define KB2(a, b) k_fused_batch<a, b, true, true, ST, B2T, 2, 256 / B2T>
  static const BatchFn<ST> table2[4] = {KB2(false, false), KB2(false, true), KB2(true, false),
                                        KB2(true, true)};
#undef KB2
  if (cpt == 2)
    return p.thermal && p.multiphase ? table2[(p.y_walls ? 2 : 0) | (p.x_open ? 1 : 0)] : nullptr;
  if (cpt != 1) return nullptr;
  const int k = (p.y_walls ? 8 : 0) | (p.x_open ? 4 : 0) | (p.thermal ? 2 : 0) |
                (p.multiphase ? 1 : 0);
  return table[k];
}

template <class ST>
int batch_grid_t(const DevParams &mode, int cpt, int device) {
  int sms = 0, occ = 0;
  const BatchFn<ST> fn = batch_variant<ST>(mode, cpt);
  if (!fn) return 0;
  const int nt = cpt == 2 ? B2T : FNT;
  const int smem = cpt == 2 ? (int)sizeof(FusedSmemT<2 * B2T>) : (int)sizeof(FusedSmem);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, smem) != cudaSuccess || occ < 1)
    return 0;
  return sms * occ;
}

template <class ST>
cudaError_t launch_batch_t(const DevParams &mode, int cpt, const BatchChannel *ch, int nch,
                           const StepScalars *sc, int ntiles, int *counter, int grid,
                           cudaStream_t s) {
  const BatchFn<ST> fn = batch_variant<ST>(mode, cpt);
  if (!fn) return cudaErrorInvalidValue;
  const int nt = cpt == 2 ? B2T : FNT;
  const size_t smem = cpt == 2 ? sizeof(FusedSmemT<2 * B2T>) : sizeof(FusedSmem);
  fn<<<grid, nt, smem, s>>>(ch, nch, sc, ntiles, counter);
  return cudaGetLastError();
}

}  // namespace

int fused_batch_grid(const DevParams &mode, int storage, int cpt, int device) {
  return storage == STORAGE_BF16  ? batch_grid_t<StoreBF16>(mode, cpt, device)
         : storage == STORAGE_F16 ? batch_grid_t<StoreF16>(mode, cpt, device)
                                  : batch_grid_t<StoreF32>(mode, cpt, device);
}

int fused_batch_width(int cpt) { return cpt == 2 ? fused_width(B2T, 2) : FW; }

cudaError_t launch_fused_batch(const DevParams &mode, int storage, int cpt, const BatchChannel *ch,
                               int nch, const StepScalars *sc, int ntiles, int *counter, int grid,
                               cudaStream_t s) {
  switch (storage) {
    case STORAGE_BF16:
      return launch_batch_t<StoreBF16>(mode, cpt, ch, nch, sc, ntiles, counter, grid, s);
    case STORAGE_F16:
      return launch_batch_t<StoreF16>(mode, cpt, ch, nch, sc, ntiles, counter, grid, s);
    default:
      return launch_batch_t<StoreF32>(mode, cpt, ch, nch, sc, ntiles, counter, grid, s);
  }
}

}  // namespace lbm
