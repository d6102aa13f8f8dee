// Batched updates of many lattices in one persistent launch per step.
#include <algorithm>
#include <cstring>
#include <new>
#include <queue>
#include <vector>

#include "lbm_handle.h"

using lbm::BatchChannel;
using lbm::StepScalars;

struct lbm_batch {
  int device = 0;
  int storage = 0;
  lbm::DevParams mode{};  // boundary modes and physics switches shared by all lattices
  std::vector<lbm_lattice *> lat;  // work-list order: most tiles first
  int tile_rows = 64;              // output rows per tile (default_rows, or set / autotuned)
  int tile_cols = 0;               // output columns per tile (even with two columns per thread)
  int cpt = 1;                     // lattice columns per thread of the batched kernel
  int grid_of[3] = {0, 0, 0};      // resident CTAs with 1 and 2 columns per thread (0: none)
  int ntiles = 0, grid = 0, sms = 1;
  BatchChannel *d_ch[2] = {nullptr, nullptr};  // tables for even and odd steps of a call
  std::vector<BatchChannel> h_ch[2];
  StepScalars *d_sc = nullptr;                  // [chunk][n] scalars of the next chunk
  StepScalars *h_sc[2] = {nullptr, nullptr};    // pinned host staging, double buffered
  cudaEvent_t sc_ev[2] = {nullptr, nullptr};
  bool sc_used[2] = {false, false};
  int sc_buf = 0;
  int *d_counter = nullptr;
  int chunk = 16;  // steps per scalar upload; also the graph length (even)
  bool use_graph = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap_stream = nullptr;
};

namespace {

using lbm_host::cuda_fail;

int tiles_of(const lbm_lattice *h, int rows, int cols) {
  const int H = std::min(rows, h->ny);
  return ((h->nx + cols - 1) / cols) * ((h->ny + H - 1) / H);
}

void drop_graph(lbm_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
}

// Work-list layout for the current tile height: lattices with the most work first
void layout(lbm_batch *b) {
  std::stable_sort(b->lat.begin(), b->lat.end(), [&](const lbm_lattice *x, const lbm_lattice *y) {
    return (long long)tiles_of(x, b->tile_rows, b->tile_cols) * x->nx >
           (long long)tiles_of(y, b->tile_rows, b->tile_cols) * y->nx;
  });
  b->ntiles = 0;
  for (auto *h : b->lat) b->ntiles += tiles_of(h, b->tile_rows, b->tile_cols);
  b->grid = b->grid_of[b->cpt];
  drop_graph(b);
}

// Greedy list schedule of the work-list at tile height H over `grid` CTA slots (tiles in
// launch order, each taken by the first free slot, a tile costing its row steps H + 15):
// returns the makespan in row steps and the number of tiles.
double schedule(const lbm_batch *b, const std::vector<const lbm_lattice *> &order, int H,
                long long &ntiles) {
  const int W = b->tile_cols;
  std::priority_queue<double, std::vector<double>, std::greater<double>> slots;
  for (int k = 0; k < b->grid; k++) slots.push(0.0);
  double makespan = 0.0;
  ntiles = 0;
  for (const lbm_lattice *h : order) {
    const int rows = std::min(H, h->ny), strips = (h->nx + W - 1) / W;
    for (int y0 = 0; y0 < h->ny; y0 += rows) {
      const double len = std::min(rows, h->ny - y0) + 15.0;
      for (int x = 0; x < strips; x++) {
        const double t = slots.top() + len;
        slots.pop();
        slots.push(t);
        makespan = std::max(makespan, t);
        ntiles++;
      }
    }
  }
  return makespan;
}

// Default tile height.  Each candidate of 128 .. 16 rows is scored by the makespan of its
// greedy schedule and the shortest wins, the taller on a tie.  Measured on GB300 against
// fixed heights, this picks the best or within 4 % of it on four shapes: 12 channels of
// 512 x 64 (16 rows, 2.8x the 64-row rate), 20 of 1024 x 256, one of 4096 x 512 and 96
// uneven channels.  When that leaves fewer tiles than SMs, most of the GPU would idle:
// then heights down to one row compete, each makespan weighted by the time of a row step
// with k tiles per SM (relative, as in the single-lattice tiling: 0.85, 1.0, 1.15 for
// k = 1 .. 3 with FP32 storage, three CTAs per SM; 0.85, 0.97, 1.42, 1.64 for k = 1 .. 4
// with 16-bit storage, four: one CTA alone is bound by the latency of its row step, a
// full SM shares the issue slots), so that a few small lattices spread over the SMs
// (200 x 50 alone: 1 row, 17.0 against 39.3 us per update with 16; 1024 x 128: 4 rows,
// 22.8 against 39.6 us).
int default_rows(const lbm_batch *b) {
  static const int tall[] = {128, 96, 64, 48, 32, 24, 16};
  static const int small[] = {16, 12, 8, 6, 4, 3, 2, 1};
  static const double kStep3[4] = {0.0, 0.85, 1.0, 1.15};
  static const double kStep4[5] = {0.0, 0.85, 0.97, 1.42, 1.64};
  std::vector<const lbm_lattice *> order(b->lat.begin(), b->lat.end());
  std::stable_sort(order.begin(), order.end(), [](const lbm_lattice *x, const lbm_lattice *y) {
    return (long long)x->nx * x->ny > (long long)y->nx * y->ny;
  });
  int best = 16;
  long long best_tiles = 0;
  double best_cost = 0.0;
  for (int H : tall) {
    long long n = 0;
    const double cost = schedule(b, order, H, n);
    if (best_cost == 0.0 || cost < best_cost) {
      best = H;
      best_cost = cost;
      best_tiles = n;
    }
  }
  if (best_tiles >= b->sms) return best;
  const int occ = std::max(1, std::min(4, b->grid / b->sms));
  const double *kStep = occ >= 4 ? kStep4 : kStep3;
  best_cost = 0.0;
  for (int H : small) {
    long long n = 0;
    const double span = schedule(b, order, H, n);
    const int k = (int)std::max(1LL, std::min<long long>(occ, (n + b->sms - 1) / b->sms));
    const double cost = span * kStep[k];
    if (best_cost == 0.0 || cost < best_cost) {
      best = H;
      best_cost = cost;
    }
  }
  return best;
}

// Channel tables for the lattices' current buffers: table 0 for steps at even
// offsets from now, table 1 for odd offsets.
int upload_tables(lbm_batch *b, cudaStream_t s) {
  const int W = b->tile_cols;
  int begin = 0;
  for (int par = 0; par < 2; par++) b->h_ch[par].resize(b->lat.size());
  for (size_t i = 0; i < b->lat.size(); i++) {
    lbm_lattice *h = b->lat[i];
    const int H = std::min(b->tile_rows, h->ny);
    for (int par = 0; par < 2; par++) {
      const int gc = h->cur ^ par;
      const int tc = h->dp.thermal ? (h->tcur ^ par) : h->tcur;
      BatchChannel &c = b->h_ch[par][i];
      c.p = h->dp;
      c.gs = h->g[gc];
      c.gout = h->g[1 - gc];
      c.Tin = h->T[tc];
      c.Tout = h->dp.thermal ? h->T[1 - tc] : h->T[tc];
      c.status = h->status;
      c.W = W;
      c.H = H;
      c.strips = (h->nx + W - 1) / W;
      c.tile_begin = begin;
    }
    begin += tiles_of(h, b->tile_rows, b->tile_cols);
  }
  const size_t bytes = sizeof(BatchChannel) * b->lat.size();
  for (int par = 0; par < 2; par++)
    LBM_CUDA(cudaMemcpyAsync(b->d_ch[par], b->h_ch[par].data(), bytes, cudaMemcpyHostToDevice, s));
  return LBM_OK;
}

// CTAs of one launch: the resident grid, or one per tile when there are fewer tiles
int launch_grid(const lbm_batch *b) { return std::min(b->grid, b->ntiles); }

int launch_one(lbm_batch *b, int k, cudaStream_t s) {
  const int n = (int)b->lat.size();
  return cuda_fail(lbm::launch_fused_batch(b->mode, b->storage, b->cpt, b->d_ch[k & 1], n,
                                           b->d_sc + (size_t)k * n, b->ntiles, b->d_counter,
                                           launch_grid(b), s));
}

int build_graph(lbm_batch *b) {
  drop_graph(b);
  LBM_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = LBM_OK;
  for (int k = 0; k < b->chunk && rc == LBM_OK; k++) rc = launch_one(b, k, b->cap_stream);
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &b->graph);
  if (rc != LBM_OK) return rc;
  LBM_CUDA(e);
  LBM_CUDA(cudaGraphInstantiate(&b->gexec, b->graph, 0));
  return LBM_OK;
}

void free_batch(lbm_batch *b) {
  drop_graph(b);
  cudaFree(b->d_ch[0]);
  cudaFree(b->d_ch[1]);
  cudaFree(b->d_sc);
  cudaFree(b->d_counter);
  for (int k = 0; k < 2; k++) {
    if (b->h_sc[k]) cudaFreeHost(b->h_sc[k]);
    if (b->sc_ev[k]) cudaEventDestroy(b->sc_ev[k]);
  }
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_h *lattices, int n, lbm_batch_h *out) {
  if (!lattices || n < 1 || !out) return LBM_ERR_ARG;
  *out = nullptr;
  lbm_lattice *first = lattices[0];
  if (!first) return LBM_ERR_ARG;
  for (int i = 0; i < n; i++) {
    lbm_lattice *h = lattices[i];
    // lattices on the fused or the two-pass path (both keep the fused kernel's 32-bit
    // element offsets, which the batched kernel uses)
    if (!h || h->device != first->device ||
        (h->kernel != LBM_KERNEL_FUSED && h->kernel != LBM_KERNEL_TWOPASS))
      return LBM_ERR_ARG;
    if (h->dp.y_walls != first->dp.y_walls || h->dp.x_open != first->dp.x_open ||
        h->dp.thermal != first->dp.thermal || h->dp.multiphase != first->dp.multiphase ||
        h->p.storage != first->p.storage)
      return LBM_ERR_ARG;
    for (int j = 0; j < i; j++)
      if (lattices[j] == h) return LBM_ERR_ARG;
  }
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_OOM;
  b->device = first->device;
  b->storage = first->p.storage;
  b->mode = first->dp;
  b->lat.assign(lattices, lattices + n);
  cudaError_t e = cudaSetDevice(b->device);
  for (int c = 1; c <= 2 && e == cudaSuccess; c++)
    b->grid_of[c] = lbm::fused_batch_grid(b->mode, b->storage, c, b->device);
  b->grid = b->grid_of[1];
  b->tile_cols = lbm::fused_batch_width(1);
  if (b->grid > 0 &&
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
    b->grid = 0;
  if (b->grid < 1) {
    delete b;
    return LBM_ERR_CUDA;
  }
  for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMalloc(&b->d_ch[k], sizeof(BatchChannel) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_sc, sizeof(StepScalars) * n * b->chunk);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_counter, 0, 2 * sizeof(int));
  for (int k = 0; k < 2 && e == cudaSuccess; k++)
    e = cudaMallocHost((void **)&b->h_sc[k], sizeof(StepScalars) * n * b->chunk);
  for (int k = 0; k < 2 && e == cudaSuccess; k++)
    e = cudaEventCreateWithFlags(&b->sc_ev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_batch(b);
    delete b;
    return cuda_fail(e);
  }
  b->tile_rows = default_rows(b);
  layout(b);
  *out = b;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch_h b, long nsteps, void *stream) {
  if (!b || nsteps < 0) return LBM_ERR_ARG;
  LBM_CUDA(cudaSetDevice(b->device));
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  LBM_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return LBM_ERR_ARG;  // as lbm_step
  int rc = upload_tables(b, s);
  if (rc) return rc;
  const int n = (int)b->lat.size();
  long done = 0;
  int phase = 0;  // parity of the steps taken in this call
  while (done < nsteps) {
    const int m = (int)std::min<long>(b->chunk, nsteps - done);
    const int buf = b->sc_buf;
    if (b->sc_used[buf]) LBM_CUDA(cudaEventSynchronize(b->sc_ev[buf]));
    StepScalars *hs = b->h_sc[buf];
    for (int k = 0; k < m; k++)
      for (int i = 0; i < n; i++)
        hs[(size_t)k * n + i] = lbm_host::scalars_at(b->lat[i], b->lat[i]->t + done + k);
    LBM_CUDA(cudaMemcpyAsync(b->d_sc, hs, sizeof(StepScalars) * n * m, cudaMemcpyHostToDevice, s));
    LBM_CUDA(cudaEventRecord(b->sc_ev[buf], s));
    b->sc_used[buf] = true;
    b->sc_buf ^= 1;
    if (b->use_graph && m == b->chunk && phase == 0) {
      if (!b->gexec) {
        rc = build_graph(b);
        if (rc) return rc;
      }
      LBM_CUDA(cudaGraphLaunch(b->gexec, s));
    } else {
      for (int k = 0; k < m; k++) {
        // k-th step of this chunk runs with the table of its parity in the call
        const int par = (phase + k) & 1;
        rc = cuda_fail(lbm::launch_fused_batch(b->mode, b->storage, b->cpt, b->d_ch[par], n,
                                               b->d_sc + (size_t)k * n, b->ntiles, b->d_counter,
                                               launch_grid(b), s));
        if (rc) return rc;
      }
    }
    phase = (phase + m) & 1;
    done += m;
  }
  for (auto *h : b->lat) {
    h->t += nsteps;
    if (nsteps & 1) {
      h->cur ^= 1;
      if (h->dp.thermal) h->tcur ^= 1;
    }
  }
  return LBM_OK;
}

int lbm_batch_set_graph(lbm_batch_h b, int enable) {
  if (!b) return LBM_ERR_ARG;
  b->use_graph = enable != 0;
  if (!b->use_graph) drop_graph(b);
  return LBM_OK;
}

int lbm_batch_set_tile_rows(lbm_batch_h b, int rows) {
  if (!b || rows < 1) return LBM_ERR_ARG;
  b->tile_rows = rows;
  layout(b);
  return LBM_OK;
}

int lbm_batch_set_tiling(lbm_batch_h b, int rows, int cols, int cols_per_thread) {
  if (!b || rows < 1 || cols < 1) return LBM_ERR_ARG;
  if (cols_per_thread != 1 && cols_per_thread != 2) return LBM_ERR_ARG;
  if (b->grid_of[cols_per_thread] < 1) return LBM_ERR_ARG;
  if (cols > lbm::fused_batch_width(cols_per_thread)) return LBM_ERR_ARG;
  if (cols_per_thread == 2 && (cols & 1)) return LBM_ERR_ARG;
  b->tile_rows = rows;
  b->tile_cols = cols;
  b->cpt = cols_per_thread;
  layout(b);
  return LBM_OK;
}

int lbm_batch_tiling(lbm_batch_h b, int *rows, int *cols, int *cols_per_thread) {
  if (!b) return LBM_ERR_ARG;
  if (rows) *rows = b->tile_rows;
  if (cols) *cols = b->tile_cols;
  if (cols_per_thread) *cols_per_thread = b->cpt;
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch_h b, int steps_per_candidate, int *best_rows, void *stream) {
  if (!b || steps_per_candidate < 2) return LBM_ERR_ARG;
  LBM_CUDA(cudaSetDevice(b->device));
  cudaStream_t s = (cudaStream_t)stream;
  struct Cand {
    int rows, cols, cpt;
  };
  static const int heights[] = {16, 24, 32, 48, 64, 96, 128};
  cudaEvent_t e0, e1;
  LBM_CUDA(cudaEventCreate(&e0));
  LBM_CUDA(cudaEventCreate(&e1));
  const bool graph = b->use_graph;
  b->use_graph = false;
  float best = -1.0f;
  Cand win{b->tile_rows, b->tile_cols, b->cpt};
  int rc = LBM_OK;
  auto time_one = [&](const Cand &c) -> int {
    b->tile_rows = c.rows;
    b->tile_cols = c.cols;
    b->cpt = c.cpt;
    layout(b);
    int r = lbm_batch_step(b, 2, stream);  // warm-up
    if (r) return r;
    LBM_CUDA(cudaEventRecord(e0, s));
    r = lbm_batch_step(b, steps_per_candidate, stream);
    if (r) return r;
    LBM_CUDA(cudaEventRecord(e1, s));
    LBM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    LBM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (best < 0.0f || ms < best) {
      best = ms;
      win = c;
    }
    return LBM_OK;
  };
  // tile heights at the widest tiles, for each column count the mode has a kernel for
  for (int cpt = 1; cpt <= 2 && rc == LBM_OK; cpt++) {
    if (b->grid_of[cpt] < 1) continue;
    for (int H : heights) {
      rc = time_one(Cand{H, lbm::fused_batch_width(cpt), cpt});
      if (rc) break;
    }
  }
  // then narrower tiles (three quarters and half the width) at the winner's height
  if (rc == LBM_OK) {
    const Cand base = win;
    const int Wmax = lbm::fused_batch_width(base.cpt);
    for (int num : {3, 2}) {
      int W = Wmax * num / 4;
      if (base.cpt == 2) W &= ~1;
      rc = time_one(Cand{base.rows, W, base.cpt});
      if (rc) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->use_graph = graph;
  b->tile_rows = win.rows;
  b->tile_cols = win.cols;
  b->cpt = win.cpt;
  layout(b);
  if (best_rows) *best_rows = win.rows;
  return rc;
}

int lbm_batch_info(lbm_batch_h b, int *ntiles, int *grid, int *tile_rows) {
  if (!b) return LBM_ERR_ARG;
  if (ntiles) *ntiles = b->ntiles;
  if (grid) *grid = b->grid;
  if (tile_rows) *tile_rows = b->tile_rows;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch_h b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  free_batch(b);
  delete b;
}

}  // extern "C"
