// Set-up and reduction kernels.
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int IBX = 32, IBY = 8;

// Post-collision populations whose pull (Eq. 12 read per destination) yields the
// rest equilibrium f_i = w_i rho0(x) at every node: the population that node
// x + e_i pulls from x holds w_i rho0(x + e_i); populations that no fluid node
// pulls, and those a wall row returns by bounce-back, hold w_i rho0(x).
template <class S>
__global__ void k_init(DevParams p, const double *__restrict__ rho0,
                       typename S::T *__restrict__ gout) {
  const int tx = ceil_div(p.nx, IBX);
  const int x = (int)(blockIdx.x % tx) * IBX + threadIdx.x, y = (int)(blockIdx.x / tx) * IBY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const long long c = (long long)y * p.pitch + x;
  const double own = rho0[(long long)y * p.nx + x];
#pragma unroll
  for (int i = 0; i < 9; i++) {
    double r = own;
    if (i > 0) {
      int xo, yo;
      if (classify(p, x, y, ex(i), ey(i), xo, yo) == NB_FLUID) r = rho0[(long long)yo * p.nx + xo];
    }
    gout[i * p.plane + c] = S::pack((float)((double)wlat(i) * (r - (double)p.rho_ref)), i);
  }
}

// FP64 partial sums of rho and rho Cv T, one pair per block (fixed order).
constexpr int RT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(RT)
    k_mass_heat_partial(DevParams p, const float *__restrict__ rho, const float *__restrict__ Tdev,
                        double T_ref, double Cv, double *__restrict__ partials) {
  double m = 0.0, h = 0.0;
  const long long n = (long long)p.nx * p.ny;
  for (long long k = (long long)blockIdx.x * RT + threadIdx.x; k < n; k += (long long)gridDim.x * RT) {
    const long long y = k / p.nx, x = k - y * p.nx;
    const long long c = y * p.pitch + x;
    const double r = (double)rho[c];
    m += r;
    h += r * Cv * (T_ref + (double)Tdev[c]);
  }
  __shared__ double sm[RT / 32], sh[RT / 32];
  m = warp_sum(m);
  h = warp_sum(h);
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5] = m;
    sh[threadIdx.x >> 5] = h;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < RT / 32; w++) {
      a += sm[w];
      b += sh[w];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

__global__ void __launch_bounds__(RT)
    k_mass_heat_final(const double *__restrict__ partials, int nblocks, double *__restrict__ out) {
  double m = 0.0, h = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += RT) {
    m += partials[2 * k];
    h += partials[2 * k + 1];
  }
  __shared__ double sm[RT / 32], sh[RT / 32];
  m = warp_sum(m);
  h = warp_sum(h);
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5] = m;
    sh[threadIdx.x >> 5] = h;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < RT / 32; w++) {
      a += sm[w];
      b += sh[w];
    }
    out[0] = a;
    out[1] = b;
  }
}

__global__ void k_unpitch(const float *__restrict__ src, int nx, int ny, int pitch, double add,
                          double *__restrict__ dst) {
  const int tx = ceil_div(nx, IBX);
  const int x = (int)(blockIdx.x % tx) * IBX + threadIdx.x, y = (int)(blockIdx.x / tx) * IBY + threadIdx.y;
  if (x >= nx || y >= ny) return;
  dst[(long long)y * nx + x] = (double)src[(long long)y * pitch + x] + add;
}

__global__ void k_pitch_T(const double *__restrict__ T, int nx, int ny, int pitch, double T_ref,
                          float *__restrict__ dst) {
  const int tx = ceil_div(pitch, IBX);
  const int x = (int)(blockIdx.x % tx) * IBX + threadIdx.x, y = (int)(blockIdx.x / tx) * IBY + threadIdx.y;
  if (x >= pitch || y >= ny) return;
  double v = 0.0;
  if (x < nx) v = T[(long long)y * nx + x] - T_ref;
  dst[(long long)y * pitch + x] = (float)v;
}

}  // namespace

cudaError_t launch_unpitch(const float *src, int nx, int ny, int pitch, double add, double *dst,
                           cudaStream_t s) {
  dim3 grid;
  cudaError_t e = tile_grid(ceil_div(nx, IBX), ceil_div(ny, IBY), grid);
  if (e != cudaSuccess) return e;
  k_unpitch<<<grid, dim3(IBX, IBY), 0, s>>>(src, nx, ny, pitch, add, dst);
  return cudaGetLastError();
}

cudaError_t launch_pitch_T(const double *T, int nx, int ny, int pitch, double T_ref, float *dst,
                           cudaStream_t s) {
  dim3 grid;
  cudaError_t e = tile_grid(ceil_div(pitch, IBX), ceil_div(ny, IBY), grid);
  if (e != cudaSuccess) return e;
  k_pitch_T<<<grid, dim3(IBX, IBY), 0, s>>>(T, nx, ny, pitch, T_ref, dst);
  return cudaGetLastError();
}

cudaError_t launch_init(const DevParams &p, int storage, const double *rho0, void *gout,
                        cudaStream_t s) {
  dim3 grid;
  cudaError_t e = tile_grid(ceil_div(p.nx, IBX), ceil_div(p.ny, IBY), grid);
  if (e != cudaSuccess) return e;
  switch (storage) {
    case STORAGE_BF16:
      k_init<StoreBF16><<<grid, dim3(IBX, IBY), 0, s>>>(p, rho0, static_cast<__nv_bfloat16 *>(gout));
      break;
    case STORAGE_F16:
      k_init<StoreF16><<<grid, dim3(IBX, IBY), 0, s>>>(p, rho0, static_cast<__half *>(gout));
      break;
    default:
      k_init<StoreF32><<<grid, dim3(IBX, IBY), 0, s>>>(p, rho0, static_cast<float *>(gout));
  }
  return cudaGetLastError();
}

int mass_heat_blocks(const DevParams &p) {
  long long n = (long long)p.nx * p.ny;
  long long b = (n + RT * 8 - 1) / (RT * 8);
  if (b < 1) b = 1;
  if (b > 1216) b = 1216;  // 8 blocks per SM on 152 SMs
  return (int)b;
}

cudaError_t launch_mass_heat(const DevParams &p, const float *rho, const float *Tdev, double T_ref,
                             double Cv, double *partials, int nblocks, double *out,
                             cudaStream_t s) {
  k_mass_heat_partial<<<nblocks, RT, 0, s>>>(p, rho, Tdev, T_ref, Cv, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mass_heat_final<<<1, RT, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

}  // namespace lbm
