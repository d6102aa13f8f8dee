// Fused lattice update, one launch per step: the CPT = 1 instantiation of the
// single-lattice kernel (lbm_fused_step.cuh), the tiling of both column widths, and
// the launch that dispatches on the tiling.
#include "lbm_fused_step.cuh"

namespace lbm {

// 32-bit element offsets cover all nine population planes
bool fused_supported(const DevParams &p) {
  return p.nx >= 1 && p.ny >= 1 && 9LL * p.plane + p.pitch < 2147483647LL;
}

int fused_max_width(int cpt) {
  return cpt == 2 ? fused_width(fused_c2_threads(), 2) : FW;
}

namespace {

cudaError_t prepare(const DevParams &p, int storage, int cpt, int *occ) {
  if (cpt == 2) return fused_c2_prepare(p, storage, occ);
  return prepare_any<FNT, 1, FMIN_F32, FMIN_16>(p, storage, occ);
}

// CTAs across the lattice: at least ceil(nx / W) strips; with CPT = 2 also enough that
// the even-aligned strips of the kernel (2 ceil(ceil(nx/2) / strips) columns at most) fit
// the CTA's output width
int strips_of(const DevParams &p, int W, int cpt) {
  int s = (p.nx + W - 1) / W;
  if (cpt == 2) {
    const int half = fused_max_width(2) / 2, m = (p.nx + 1) / 2;
    s = std::max(s, (m + half - 1) / half);
  }
  return s;
}

}  // namespace

FusedTiling fused_tiling(const DevParams &p, int storage, int device, int cpt) {
  FusedTiling best{0, 0, cpt};
  int sms = 0, occ = 0;
  if (cpt != 1 && cpt != 2) return best;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return best;
  if (prepare(p, storage, cpt, &occ) != cudaSuccess || occ < 1) return best;
  // Widest strips (fewest halo columns), then the row-chunk height H with the shortest
  // estimated launch time over one wave of resident CTAs.  Every CTA sweeps H + 15 row
  // steps, and a row step takes longer the more CTAs share the SM: one CTA alone is bound
  // by the latency of the row step, a full SM shares its issue slots.  kStep[k] is the
  // measured time of one row step with k CTAs of 128 threads per SM, relative, for the
  // build that fits three per SM (FP32 storage; 4096 x 512: 1.20 us with three, 1.04 us
  // with two; 1024 x 128 and 200 x 50: one CTA about 0.83 of two) and the one that fits
  // four (16-bit storage, and two columns per thread, whose k CTAs count as 2k: a CTA's
  // row step carries twice the work).  Beyond one wave the time grows with k.  Equal-work
  // tilings with narrower strips or two waves were 2-35 % slower on 4096 x 512.  A small
  // lattice thus gets short chunks spread over idle SMs (1 row on 200 x 50, 2x the rate of
  // 16-row chunks), a large one one wave of tall chunks (FP32: 40 rows on 4096 x 512, 683
  // on 16384 x 2048).
  static const double kStep3[4] = {0.0, 0.85, 1.0, 1.15};
  static const double kStep4[5] = {0.0, 0.85, 0.97, 1.42, 1.64};
  const bool four = occ >= 4 || cpt == 2;
  const double *kStep = four ? kStep4 : kStep3;
  const int kmax = four ? 4 : 3;
  const int W = fused_max_width(cpt);
  const long long slots = (long long)sms * occ;
  const int strips = strips_of(p, W, cpt);
  long long max_chunks = slots / strips;
  if (max_chunks < 1) max_chunks = 1;
  if (max_chunks > p.ny) max_chunks = p.ny;
  int H = p.ny;
  double best_cost = -1.0;
  for (long long c = 1; c <= max_chunks; c++) {
    const int h = (int)((p.ny + c - 1) / c);
    const long long tiles = (long long)strips * ((p.ny + h - 1) / h);
    const long long k = ((tiles + sms - 1) / sms) * cpt;  // CTA-equivalents per SM
    const double step = k <= kmax ? kStep[k] : kStep[kmax] * (double)k / kmax;
    const double cost = (h + 15) * step;
    if (best_cost < 0.0 || cost < best_cost) {  // ties keep the taller chunk
      best_cost = cost;
      H = h;
    }
  }
  best = FusedTiling{W, H, cpt, 0};
  // Programmatic dependent launch when the grid fills at least 90 % of one wave of resident
  // CTAs: the next update's CTAs then take the SMs as this update's CTAs finish (4096 x 512:
  // 65.0 against 65.8 us per update; 16384 x 2048 unchanged).  A grid that leaves SMs free
  // keeps plain stream order: there the waiting CTAs of the next update slowed the update
  // (1024 x 128: 16.6 against 15.7 us).
  const long long tiles = (long long)strips * ((p.ny + H - 1) / H);
  best.pdl = cpt == 1 && tiles * 10 >= slots * 9 && tiles <= slots ? 1 : 0;
  return best;
}

cudaError_t launch_fused(const DevParams &p, int storage, const void *gs, void *gout,
                         const float *Tin, float *Tout, unsigned *status, const StepScalars *sc,
                         FusedTiling tl, cudaStream_t s) {
  if (tl.H < 1 || tl.W < 1 || tl.W > fused_max_width(tl.cpt)) return cudaErrorInvalidValue;
  // strips and row chunks of at most W columns (see strips_of) and H rows
  const dim3 grid(strips_of(p, tl.W, tl.cpt), (p.ny + tl.H - 1) / tl.H);
  if (tl.cpt == 2) return fused_c2_launch(p, storage, gs, gout, Tin, Tout, status, sc, grid, s);
  if (tl.cpt != 1) return cudaErrorInvalidValue;
  return launch_any<FNT, 1, FMIN_F32, FMIN_16>(p, storage, gs, gout, Tin, Tout, status, sc, grid,
                                                tl.pdl != 0, s);
}

}  // namespace lbm
