// Handle of one lattice (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm_host {

enum { KN_DENSITY = 0, KN_COLLIDE, KN_ENERGY, KN_FUSED, KN_STREAM_COLLIDE, KN_ENERGY_RK4, KN_COUNT };

struct TimedLaunch {
  int kind;
  cudaEvent_t a, b;
};

}  // namespace lbm_host

struct lbm_lattice {
  int device = 0;
  int nx = 0, ny = 0, pitch = 0;
  long long plane = 0;
  lbm_params_t p{};
  lbm::DevParams dp{};
  double Tc = 0, T_ref = 0, rho_ref = 0;
  double rho_branch_end = 0;  // vapour-branch end of the isotherm at T_inlet (pressure inlet)
  long long t = 0;
  int kernel = LBM_KERNEL_SPLIT;
  lbm::FusedTiling fused{0, 0, 1};  // CTA tiling of the fused kernel
  lbm::TwoPassTiling twopass{0, 0};  // row-chunk heights of the two-pass path
  int cur = 0;   // g[cur]: post-collision populations of the previous update
  int tcur = 0;  // T[tcur]: temperature deviation of time t
  void *g[2] = {nullptr, nullptr};  // populations, storage-typed elements
  int esize = 4;                    // bytes per stored population
  float *T[2] = {nullptr, nullptr};
  float *rho = nullptr, *psi = nullptr, *ux = nullptr, *uy = nullptr;
  unsigned *status = nullptr;
  double *partials = nullptr, *sums = nullptr;
  int nblocks = 1;
  double *rho0 = nullptr;  // device staging (nx * ny doubles) for the field copies in and out
  double *host_sums = nullptr;  // pinned, 2 doubles
  size_t device_bytes = 0;
  // Fused updates run in chunks of kChunk: the chunk's boundary scalars (one StepScalars per
  // update) go from a pinned staging buffer (two, alternating) to d_sc, then a full chunk
  // replays a captured CUDA graph of kChunk launches when graphs are on.  A chunk has an
  // even length, so it starts and ends at the same buffer parity: gexec[cur][tcur].
  static constexpr int kChunk = 16;
  lbm::StepScalars *d_sc = nullptr;
  lbm::StepScalars *h_sc[2] = {nullptr, nullptr};
  cudaEvent_t sc_ev[2] = {nullptr, nullptr};
  bool sc_used[2] = {false, false};
  int sc_buf = 0;
  bool use_graph = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  // timing
  bool timing = false;
  std::vector<lbm_host::TimedLaunch> pending;
  std::vector<cudaEvent_t> pool;
  double total_ms[lbm_host::KN_COUNT] = {};
  long launches[lbm_host::KN_COUNT] = {};
};


namespace lbm_host {

// per-update scalars of time t (inlet velocity or density, body-force phase)
lbm::StepScalars scalars_at(const lbm_lattice *h, long long t);
int cuda_fail(cudaError_t e);

}  // namespace lbm_host

#define LBM_CUDA(expr)                                     \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return lbm_host::cuda_fail(_e); \
  } while (0)
