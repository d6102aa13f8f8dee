// Split lattice update: three launches per step.
//  1. k_density_psi: pull-stream (Eq. 12 with boundary rules), rho (Eq. 13),
//     pseudopotential (Eqs. 10-11) -> rho and psi - psi_r arrays.
//  2. k_collide: pull-stream again, forces from the psi of the 8 neighbours
//     (Eqs. 9, 14, 15), velocity (Eq. 13), MRT collision with Li forcing
//     (Eqs. 6-8) -> post-collision populations and u.
//  3. k_energy: four RK4 stages (Eqs. 17-18) of the energy equation (Eq. 16)
//     on a shared-memory tile with a halo of 4 nodes.
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int BX = 32, BY = 8;

template <class S>
__global__ void __launch_bounds__(BX *BY)
    k_density_psi(DevParams p, const typename S::T *__restrict__ gs, const float *__restrict__ Tdev,
                  float *__restrict__ rho_o, float *__restrict__ psi_o, unsigned *status,
                  StepScalars sc) {
  const int tx = ceil_div(p.nx, BX);
  const int x = (int)(blockIdx.x % tx) * BX + threadIdx.x, y = (int)(blockIdx.x / tx) * BY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  float g[9];
  pull<S>(p, gs, x, y, sc, g);
  const float rho = p.rho_ref + sum9(g);
  const long long c = (long long)y * p.pitch + x;
  unsigned st = 0;
  if (!(rho > 0.0f)) st |= ST_RHO_NONPOS;
  if (p.eos_b * rho >= 1.0f) st |= ST_EOS_POLE;
  float dpsi = 0.0f;
  if (p.multiphase) {
    const float dT = Tdev[c];
    if (!(p.T_ref + dT > 0.0f)) st |= ST_T_NONPOS;
    dpsi = pseudopotential_dev(p, sum9(g), dT, st);
  }
  rho_o[c] = rho;
  psi_o[c] = dpsi;
  set_status(status, st);
}

template <class S, bool WRITE_POP>
__global__ void __launch_bounds__(BX *BY)
    k_collide(DevParams p, const typename S::T *__restrict__ gs, typename S::T *__restrict__ gout,
              const float *__restrict__ Tdev, const float *__restrict__ psi,
              float *__restrict__ ux_o, float *__restrict__ uy_o, unsigned *status,
              StepScalars sc) {
  const int tx = ceil_div(p.nx, BX);
  const int x = (int)(blockIdx.x % tx) * BX + threadIdx.x, y = (int)(blockIdx.x / tx) * BY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  float g[9];
  pull<S>(p, gs, x, y, sc, g);
  const long long c = (long long)y * p.pitch + x;
  Force F{0.0f, 0.0f, 0.0f};
  if (p.multiphase) {
    float dpsin[9];
    unsigned solid = 0;
    const bool interior = x > 0 && x < p.nx - 1 && y > 0 && y < p.ny - 1;
#pragma unroll
    for (int i = 1; i < 9; i++) {
      if (interior) {
        dpsin[i] = psi[c + ey(i) * p.pitch + ex(i)];
      } else {
        int xo, yo;
        int k = classify(p, x, y, ex(i), ey(i), xo, yo);
        if (k == NB_SOLID) {
          solid |= 1u << i;
          dpsin[i] = 0.0f;
        } else {
          dpsin[i] = psi[(long long)yo * p.pitch + xo];
        }
      }
    }
    float psiw = 0.0f;
    if (p.rho_w > 0.0f && solid) {
      unsigned st_unused = 0;
      psiw = pseudopotential(p, p.rho_w, p.T_ref + Tdev[c], st_unused);
    }
    F = interaction_force(p, psi[c], dpsin, solid, psiw);
  }
  const float drho = sum9(g);
  const float rho_v = p.drho_ref_g + drho;  // rho - rho_v of Eq. 15
  F.Fx += rho_v * p.gx * sc.gcos;
  F.Fy += rho_v * p.gy * sc.gcos;
  float gn[9], rho, ux, uy;
  collide(p, g, drho, F.Fx, F.Fy, F.fm2, gn, rho, ux, uy);
  if (WRITE_POP) {
#pragma unroll
    for (int i = 0; i < 9; i++) gout[i * p.plane + c] = S::pack(gn[i], i);
  }
  ux_o[c] = ux;
  uy_o[c] = uy;
  if (!isfinite(rho + ux + uy)) set_status(status, ST_NAN);
}

// ---------------------------------------------------------------------------
// Energy equation, RK4 on a tile with halo 4 (each stage is a 9-point stencil)
// ---------------------------------------------------------------------------
constexpr int ETX = 32, ETY = 16, EH = 4;
constexpr int ERX = ETX + 2 * EH, ERY = ETY + 2 * EH, ERN = ERX * ERY;
constexpr int ETHREADS = 256;
enum : unsigned char { K_DOMAIN = 0, K_WALL = 1, K_INLET = 2, K_OUTLET = 3 };

__device__ __forceinline__ int modi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__global__ void __launch_bounds__(ETHREADS)
    k_energy(DevParams p, const float *__restrict__ Tin, float *__restrict__ Tout,
             const float *__restrict__ rho, const float *__restrict__ ux,
             const float *__restrict__ uy, unsigned *status, StepScalars sc) {
  __shared__ float sTb[ERN], sX[ERN], sY[ERN], sux[ERN], suy[ERN];
  __shared__ float scl[ERN], se1[ERN], se2[ERN];
  __shared__ float sacc[ETX * ETY];
  __shared__ short sred[ERN];
  __shared__ unsigned char skind[ERN];

  const int tx = ceil_div(p.nx, ETX);
  const int x0 = (int)(blockIdx.x % tx) * ETX - EH, y0 = (int)(blockIdx.x / tx) * ETY - EH;
  const int tid = threadIdx.x;

  for (int i = tid; i < ERN; i += ETHREADS) {
    const int lx = i % ERX, ly = i / ERX;
    int gx = x0 + lx, gy = y0 + ly;
    unsigned char kind = K_DOMAIN;
    int red = i;
    float T = 0.0f, vx = 0.0f, vy = 0.0f, cl = 0.0f, cA = 0.0f, cB = 0.0f;
    bool load = true;
    if (p.y_walls && (gy < 0 || gy >= p.ny)) {
      kind = K_WALL;
      const bool top = gy >= p.ny;
      const int wx = p.x_open ? gx : modi(gx, p.nx);  // periodic image of the wall column
      if (p.adiabatic && wall_adiabatic(p, wx, top)) {
        // adiabatic: every stage reads the fluid node across the wall (same column);
        // x is periodic here, so that node lies inside this tile's halo region
        red = ((top ? p.ny - 1 : 0) - y0) * ERX + lx;
      } else {
        T = top ? wall_T_top_dev(p, wx) : wall_T_dev(p, wx);
      }
      load = false;
    } else {
      if (!p.y_walls) gy = modi(gy, p.ny);
      if (!p.x_open) {
        gx = modi(gx, p.nx);
      } else if (gx < 0) {
        kind = K_INLET;
        T = p.T_inlet_dev;
        vx = sc.u_in;
        load = false;
        if (p.p_inlet) {  // pressure inlet: the velocity ghost copies column 0
          const long long c0 = (long long)gy * p.pitch;
          vx = ux[c0];
          vy = uy[c0];
        }
      } else if (gx >= p.nx) {
        kind = K_OUTLET;
        red = i - (gx - (p.nx - 1));
        gx = p.nx - 1;
      }
    }
    if (load) {
      const long long c = (long long)gy * p.pitch + gx;
      T = Tin[c];
      vx = ux[c];
      vy = uy[c];
      if (kind == K_DOMAIN) {
        const float r = rho[c];
        const float br = p.eos_b * r;
        const float inv_cv = 1.0f / p.Cv;
        cl = p.lambda * inv_cv / r;
        cA = p.eos_R * inv_cv / (1.0f - br);
        cB = p.eos_a * r * p.kappa * inv_cv / (1.0f + 2.0f * br - br * br);
      }
    }
    sTb[i] = T;
    sX[i] = T;
    sY[i] = T;
    sux[i] = vx;
    suy[i] = vy;
    scl[i] = cl;
    se1[i] = cA;
    se2[i] = cB;
    sred[i] = (short)red;
    skind[i] = kind;
  }
  __syncthreads();

  // div u on the halo-3 region: 3 sum w_i u(x+e_i).e_i
  {
    constexpr int W = ETX + 6, H = ETY + 6;
    for (int j = tid; j < W * H; j += ETHREADS) {
      const int lx = 1 + j % W, ly = 1 + j / W, i = ly * ERX + lx;
      if (skind[i] != K_DOMAIN) continue;
      float d = 0.0f;
#pragma unroll
      for (int k = 1; k < 9; k++) {
        const int nb = i + ey(k) * ERX + ex(k);
        d += wlat(k) * (sux[nb] * ex(k) + suy[nb] * ey(k));
      }
      d *= 3.0f;
      se1[i] *= d;
      se2[i] *= d;
    }
  }
  __syncthreads();

  float *src = sTb, *dst = sX;
#pragma unroll 1
  for (int s = 0; s < 4; s++) {
    const int h = 3 - s;
    const int W = ETX + 2 * h, H = ETY + 2 * h;
    for (int j = tid; j < W * H; j += ETHREADS) {
      const int lx = EH - h + j % W, ly = EH - h + j / W, i = ly * ERX + lx;
      if (skind[i] != K_DOMAIN) continue;
      const float c = src[i];
      float gxs = 0.0f, gys = 0.0f, lap = 0.0f;
#pragma unroll
      for (int k = 1; k < 9; k++) {
        const float v = src[sred[i + ey(k) * ERX + ex(k)]];
        gxs += wlat(k) * ex(k) * v;
        gys += wlat(k) * ey(k) * v;
        lap += wlat(k) * (v - c);
      }
      gxs *= 3.0f;
      gys *= 3.0f;
      lap *= 6.0f;
      const float Tabs = p.T_ref + c;
      const float sq = sqrtf(Tabs * p.inv_Tc);
      const float hv = -(sux[i] * gxs + suy[i] * gys) + scl[i] * lap - se1[i] * Tabs -
                       se2[i] * sq * (1.0f + p.kappa - p.kappa * sq);
      if (s < 3) dst[i] = sTb[i] + (s == 2 ? 1.0f : 0.5f) * hv;
      const int ix = lx - EH, iy = ly - EH;
      if (ix >= 0 && ix < ETX && iy >= 0 && iy < ETY) {
        if (s == 0)
          sacc[iy * ETX + ix] = hv;
        else
          sacc[iy * ETX + ix] += (s == 3 ? 1.0f : 2.0f) * hv;
      }
    }
    __syncthreads();
    src = dst;
    dst = (dst == sX) ? sY : sX;
  }

  unsigned st = 0;
  for (int j = tid; j < ETX * ETY; j += ETHREADS) {
    const int ix = j % ETX, iy = j / ETX;
    const int gx = x0 + EH + ix, gy = y0 + EH + iy;
    if (gx >= p.nx || gy >= p.ny) continue;
    const int i = (iy + EH) * ERX + ix + EH;
    const float Tn = sTb[i] + sacc[j] * (1.0f / 6.0f);
    if (!isfinite(Tn)) st |= ST_NAN;
    if (!(p.T_ref + Tn > 0.0f)) st |= ST_T_NONPOS;
    Tout[(long long)gy * p.pitch + gx] = Tn;
  }
  set_status(status, st);
}

template <class S>
cudaError_t density_psi_t(const DevParams &p, const void *gs, const float *Tdev, float *rho,
                          float *psi, unsigned *status, StepScalars sc, cudaStream_t s) {
  dim3 grid;
  cudaError_t e = tile_grid(ceil_div(p.nx, BX), ceil_div(p.ny, BY), grid);
  if (e != cudaSuccess) return e;
  k_density_psi<S><<<grid, dim3(BX, BY), 0, s>>>(p, static_cast<const typename S::T *>(gs), Tdev,
                                                 rho, psi, status, sc);
  return cudaGetLastError();
}

template <class S>
cudaError_t collide_t(const DevParams &p, const void *gs, void *gout, const float *Tdev,
                      const float *psi, float *ux, float *uy, unsigned *status, StepScalars sc,
                      bool write_populations, cudaStream_t s) {
  using T = typename S::T;
  dim3 grid;
  cudaError_t e = tile_grid(ceil_div(p.nx, BX), ceil_div(p.ny, BY), grid);
  if (e != cudaSuccess) return e;
  const T *in = static_cast<const T *>(gs);
  T *out = static_cast<T *>(gout);
  if (write_populations)
    k_collide<S, true><<<grid, dim3(BX, BY), 0, s>>>(p, in, out, Tdev, psi, ux, uy, status, sc);
  else
    k_collide<S, false><<<grid, dim3(BX, BY), 0, s>>>(p, in, out, Tdev, psi, ux, uy, status, sc);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_density_psi(const DevParams &p, int storage, const void *gs, const float *Tdev,
                               float *rho, float *psi, unsigned *status, StepScalars sc,
                               cudaStream_t s) {
  switch (storage) {
    case STORAGE_BF16: return density_psi_t<StoreBF16>(p, gs, Tdev, rho, psi, status, sc, s);
    case STORAGE_F16: return density_psi_t<StoreF16>(p, gs, Tdev, rho, psi, status, sc, s);
    default: return density_psi_t<StoreF32>(p, gs, Tdev, rho, psi, status, sc, s);
  }
}

cudaError_t launch_collide(const DevParams &p, int storage, const void *gs, void *gout,
                           const float *Tdev, const float *psi, float *ux, float *uy,
                           unsigned *status, StepScalars sc, bool write_populations,
                           cudaStream_t s) {
  switch (storage) {
    case STORAGE_BF16:
      return collide_t<StoreBF16>(p, gs, gout, Tdev, psi, ux, uy, status, sc, write_populations, s);
    case STORAGE_F16:
      return collide_t<StoreF16>(p, gs, gout, Tdev, psi, ux, uy, status, sc, write_populations, s);
    default:
      return collide_t<StoreF32>(p, gs, gout, Tdev, psi, ux, uy, status, sc, write_populations, s);
  }
}

cudaError_t launch_energy(const DevParams &p, const float *Tin, float *Tout, const float *rho,
                          const float *ux, const float *uy, unsigned *status, StepScalars sc,
                          cudaStream_t s) {
  dim3 grid;
  cudaError_t e = tile_grid(ceil_div(p.nx, ETX), ceil_div(p.ny, ETY), grid);
  if (e != cudaSuccess) return e;
  k_energy<<<grid, ETHREADS, 0, s>>>(p, Tin, Tout, rho, ux, uy, status, sc);
  return cudaGetLastError();
}

}  // namespace lbm
