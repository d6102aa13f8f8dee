// Mass and heat sums for callers that cannot allocate device memory.
//
// Some callers can't call cudaMalloc: a host framework or serving loop that owns
// the whole device-memory budget and hands out buffers only from its own pool,
// or a latency-critical loop that must not risk the device-wide synchronisation
// that cudaMalloc and cudaFree can cause.  lbm_mass_heat_noalloc runs the same
// two-stage FP64 reduction as lbm_reduce on caller-owned fields, but keeps the
// per-block partial sums in a fixed array in this library's device memory, so
// the call allocates nothing.
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

// One (mass, heat) pair per block of the first reduction stage.  The first stage
// never uses more than 1216 blocks (8 per SM on 152 SMs), whatever the field size.
constexpr int kNoallocPairs = 1216;
// Every GPU that loads the library holds this array (19 KB) until the process exits.
static __device__ __align__(256) double g_noalloc_partials[2 * kNoallocPairs];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_partials_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
int partials_address(int device, double **addr) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[device]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr)
      return LBM_ERR_CUDA;
    g_partials_addr[device] = static_cast<double *>(ptr);
  }
  *addr = g_partials_addr[device];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_mass_heat_noalloc(const float *rho, const float *T_dev, int nx, int ny,
                                     int pitch, double T_ref, double Cv, double *out,
                                     void *stream) {
  if (!rho || !T_dev || !out) return LBM_ERR_ARG;
  if (nx < 1 || ny < 1 || nx > LBM_NOALLOC_MAX_DIM || ny > LBM_NOALLOC_MAX_DIM) return LBM_ERR_ARG;
  if (pitch < nx || pitch > 2 * LBM_NOALLOC_MAX_DIM) return LBM_ERR_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return LBM_ERR_CUDA;
  if (device < 0 || device >= kMaxDevices) return LBM_ERR_ARG;
  double *partials = nullptr;
  int rc = partials_address(device, &partials);
  if (rc != LBM_OK) return rc;
  lbm::DevParams d{};
  d.nx = nx;
  d.ny = ny;
  d.pitch = pitch;
  d.plane = (long long)ny * pitch;
  const int nblocks = lbm::mass_heat_blocks(d);
  if (nblocks < 1 || nblocks > kNoallocPairs) return LBM_ERR_ARG;
  // every block overwrites its own pair and the second stage reads only those
  // pairs, so nothing left by an earlier call needs clearing
  cudaError_t e = lbm::launch_mass_heat(d, rho, T_dev, T_ref, Cv, partials, nblocks, out,
                                        static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
