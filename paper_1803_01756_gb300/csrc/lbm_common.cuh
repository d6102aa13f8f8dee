// Device-side physics of the D2Q9 pseudopotential MRT lattice update
// (arXiv:1803.01756, Section 2).  FP32 arithmetic; populations are carried as
// deviations g_i = f_i - w_i rho_ref and temperatures as T - T_ref, so that the
// stored numbers are small and FP32 rounding stays far below the field values.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

// D2Q9 velocity set of Eq. 2
__host__ __device__ constexpr int ex(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 5 + 2) & 3) + 5);
}
// D2Q9 lattice weights
__host__ __device__ constexpr float wlat(int i) {
  return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// Eq. 9 interaction weights w(1) = 1/3, w(2) = 1/12
__host__ __device__ constexpr float wpsi(int i) {
  return i == 0 ? 0.0f : (i <= 4 ? 1.0f / 3.0f : 1.0f / 12.0f);
}

// 1 / w_i
__host__ __device__ constexpr float inv_wlat(int i) {
  return i == 0 ? 9.0f / 4.0f : (i <= 4 ? 9.0f : 36.0f);
}

// Population storage.  Kernels always work on g_i = f_i - w_i rho_ref in FP32.
//  F32 : stores g_i.
//  BF16, F16 : store h_i = g_i / w_i = f_i / w_i - rho_ref, so that all nine
//              directions share one range (16-bit, round to nearest).
//  store2 writes the values of two adjacent columns (p 2-element aligned) with one
//  store, rounding each exactly as pack does.
struct StoreF32 {
  using T = float;
  static __device__ __forceinline__ float load(const T *p, int) { return __ldg(p); }
  static __device__ __forceinline__ T pack(float g, int) { return g; }
  static __device__ __forceinline__ void store2(T *p, float a, float b, int) {
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
  }
};
struct StoreBF16 {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float load(const T *p, int i) {
    return wlat(i) * __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ T pack(float g, int i) {
    return __float2bfloat16_rn(g * inv_wlat(i));
  }
  static __device__ __forceinline__ void store2(T *p, float a, float b, int i) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a * inv_wlat(i), b * inv_wlat(i));
  }
};
struct StoreF16 {
  using T = __half;
  static __device__ __forceinline__ float load(const T *p, int i) {
    return wlat(i) * __half2float(__ldg(p));
  }
  static __device__ __forceinline__ T pack(float g, int i) { return __float2half_rn(g * inv_wlat(i)); }
  static __device__ __forceinline__ void store2(T *p, float a, float b, int i) {
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a * inv_wlat(i), b * inv_wlat(i));
  }
};

enum : unsigned {
  ST_NAN = 1u, ST_PSI_NEG = 2u, ST_RHO_NONPOS = 4u, ST_EOS_POLE = 8u, ST_T_NONPOS = 16u
};

// Parameters as the kernels see them (derived on the host from lbm_params_t).
struct DevParams {
  int nx, ny, pitch;
  int x_open, y_walls, multiphase, thermal;
  int p_inlet;            // x = 0 is a pressure (density) inlet instead of a velocity inlet
  long long plane;        // ny * pitch, elements per population plane
  float rho_ref, T_ref;   // deviation references
  float Tc, inv_Tc;
  float eos_a, eos_b, eos_R, kappa;
  float G, Gw, rho_w;     // rho_w <= 0: psi_w = local psi
  // reference state (rho_ref, T_ref) of the deviation pseudopotential, with D(rho) =
  // 1 + 2 b rho - b^2 rho^2 and the factor 2/G of psi^2 folded into the coefficients
  float sr;               // sqrt(T_ref / Tc)
  float rphi_r;           // 1 + kappa (1 - sr)
  float kappa1;           // 1 + kappa
  float psi_r, psi_r2;    // psi(rho_ref, T_ref) and its square
  float ps_RT;            // (2/G) R
  float ps_R;             // (2/G) R T_ref / (1 - b rho_ref)
  float ps_g;             // 1 + 2 b rho_ref
  float ps_B;             // (2/G) a phi(T_ref) / D(rho_ref)
  float ps_phi;           // -(2/G) a kappa
  float ps_3;             // -(2/G) / 3
  float G3, G3r;          // -G / 3 and -G psi_r / 3 (bulk Eq. 9 force, 1/3 weight taken out)
  float wall_r;           // (G - Gw) psi_r: wall term of Eqs. 9 + 14 at the reference state
  float drho_ref_g;       // rho_ref - rho_g, the reference part of Eq. 15's (rho - rho_v)
  float c_theta_e;        // 12 theta s_e G^2   ((1 - s_e/2) 12 theta / (tau_e - 1/2) = 12 theta s_e)
  float c_theta_z;        // 12 theta s_zeta G^2
  float s_e, s_z, s_q;
  // collision coefficients with the 1/D_k of M^-1 = M^T D^-1 folded in (Eqs. 7-8):
  //   a1 = m1*/36 = k1[0] n1 + k1[1] drho + k1[2] rho|u|^2 + k1[3] u.F + k1[4] 9|q|^2
  //   a2 = m2*/36 = k2[0] n2 + k2[1] drho + k2[2] rho|u|^2 + k2[3] u.F + k2[4] 9|q|^2
  //   a4 = m4*/12 = kq[0] n4 + kq[1] rho u_x + kq[2] F_x   (same for a6 with y)
  float k1[5], k2[5], kq[3];
  float tau_g, dtau, rho_g, inv_drho;  // Eq. 5: tau_g + clamp((rho - rho_g) inv_drho) dtau
  int tau_const;          // tau_g == tau_l
  float s_nu_const;
  // with tau_const, the a7 / a8 coefficients of the collision (see collide):
  // 0.25 (1 - s_nu), 0.25 s_nu, 0.25 (2 - s_nu), 0.25 (1 - s_nu / 2)
  float kn[4];
  float gx, gy;
  int has_g;              // gx or gy nonzero
  float Cv, lambda;
  float lam_cv, R_cv, akap_cv;  // lambda/Cv, R/Cv, a kappa/Cv
  // energy coefficients of the fused kernel's RK4 stages (K(T) with the stencil and
  // sqrt(T/Tc) factors folded in): (2/3) lambda/Cv, R Tc/(3 Cv), a kappa (1 + kappa)/(3 Cv),
  // kappa/(1 + kappa), T_ref/Tc
  float lam23_cv, RTc_cv3, akap1_cv3, kappa_r, xr;
  float tw0, tw_slope;    // wall temperature deviation at x: tw0 + tw_slope * x (bottom wall)
  float tw0_top, tw_slope_top;  // the same for the top wall
  // isothermal windows [x0, x1) of the two walls; outside them the wall is adiabatic
  // (x1 <= x0: isothermal everywhere); adiabatic != 0 when some column is adiabatic
  int top_iso_x0, top_iso_x1, bot_iso_x0, bot_iso_x1;
  int adiabatic;
  float T_inlet_dev;
  float rho_out;
};

// Per-update scalars computed on the host in double precision.
struct StepScalars {
  float u_in;   // inlet velocity of time t
  float gcos;   // cos(g_omega t)
  float rho_in; // inlet density of time t (pressure inlet)
};

// 2D tilings launched as 1D grids: a grid's y dimension stops at 65535 blocks and a
// lattice may have 2^20 rows.  Block b covers tile (b % tiles_x, b / tiles_x).
__host__ __device__ constexpr int ceil_div(int a, int b) { return (a + b - 1) / b; }
inline cudaError_t tile_grid(int tiles_x, int tiles_y, dim3 &grid) {
  const long long n = (long long)tiles_x * tiles_y;
  if (n < 1 || n > 2147483647LL) return cudaErrorInvalidConfiguration;
  grid = dim3((unsigned)n);
  return cudaSuccess;
}

__device__ __forceinline__ int wrapi(int v, int n) {
  v = v < 0 ? v + n : v;
  return v >= n ? v - n : v;
}

__device__ __forceinline__ void set_status(unsigned *status, unsigned bits) {
  if (bits) atomicOr(status, bits);
}

// ---------------------------------------------------------------------------
// Peng-Robinson EOS (Eq. 11) and pseudopotential (Eq. 10)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float eos_pressure(const DevParams &p, float rho, float Tabs) {
  float r = 1.0f + p.kappa * (1.0f - sqrtf(Tabs * p.inv_Tc));
  float phi = r * r;
  float br = p.eos_b * rho;
  return rho * p.eos_R * Tabs / (1.0f - br) - p.eos_a * phi * rho * rho / (1.0f + 2.0f * br - br * br);
}

// psi = sqrt(2 (P - rho/3) / G); negative argument -> 0 and a status bit
__device__ __forceinline__ float pseudopotential(const DevParams &p, float rho, float Tabs,
                                                 unsigned &st) {
  float arg = 2.0f * (eos_pressure(p, rho, Tabs) - rho * (1.0f / 3.0f)) / p.G;
  if (!(arg >= 0.0f)) {
    st |= ST_PSI_NEG;
    return 0.0f;
  }
  return sqrtf(arg);
}

// Deviation of psi from psi_r = psi(rho_ref, T_ref), from the deviations
// drho = rho - rho_ref and dT = T - T_ref.  The pressure difference of Eq. 11 is
// formed term by term from exact difference identities,
//   rho T/(1-b rho) - rho_r T_r/(1-b rho_r) = (dT rho + T_r drho/(1-b rho_r)) / (1-b rho),
//   phi rho^2/D(rho) - phi_r rho_r^2/D(rho_r)
//       = (dphi rho^2 + phi_r drho (rho + rho_r + 2 b rho rho_r) / D(rho_r)) / D(rho),
//   dphi = phi(T) - phi(T_r) = -kappa (s - s_r) (r + r_r),  s - s_r = dT / (Tc (s + s_r)),
// so no large nearly equal numbers are subtracted; then
//   psi^2 - psi_r^2 = 2 (dP - drho/3) / G   and   psi - psi_r = (psi^2 - psi_r^2) / (psi + psi_r).
// Neighbour differences of psi therefore keep FP32 relative precision.
__device__ __forceinline__ float pseudopotential_dev(const DevParams &p, float drho, float dT,
                                                     unsigned &st) {
  const float rho = p.rho_ref + drho;
  const float br = p.eos_b * rho;
  const float inv1 = __fdividef(1.0f, 1.0f - br);
  const float invD = __fdividef(1.0f, fmaf(br, 2.0f - br, 1.0f));
  const float s = sqrtf((p.T_ref + dT) * p.inv_Tc);
  const float ds = __fdividef(dT * p.inv_Tc, s + p.sr);
  const float r = fmaf(-p.kappa, s, p.kappa1);
  const float g = fmaf(rho, p.ps_g, p.rho_ref);
  // (2/G) R of the pressure difference, and (2/G) a of its attraction part
  const float tR = inv1 * fmaf(p.ps_RT * dT, rho, p.ps_R * drho);
  const float tA = invD * fmaf(p.ps_phi * ds * (r + p.rphi_r), rho * rho, p.ps_B * drho * g);
  const float dpsi2 = fmaf(p.ps_3, drho, tR - tA);
  const float psi2 = p.psi_r2 + dpsi2;
  // a negative argument gives psi = 0 and a status bit (selects, no branch)
  const bool neg = !(psi2 >= 0.0f);
  st |= neg ? ST_PSI_NEG : 0u;
  const float den = sqrtf(fmaxf(psi2, 0.0f)) + p.psi_r;
  const float d = den > 0.0f ? __fdividef(dpsi2, den) : 0.0f;
  return neg ? -p.psi_r : d;
}

// ---------------------------------------------------------------------------
// Geometry: classification of the site (x + dx, y + dy) seen from a fluid node
// ---------------------------------------------------------------------------
enum : int { NB_FLUID = 0, NB_SOLID = 1, NB_INLET = 2, NB_OUTLET = 3 };

// Returns the kind; for FLUID/INLET/OUTLET (xo, yo) is the fluid node supplying
// a copied value (wrapped, or clamped at the open ends).
__device__ __forceinline__ int classify(const DevParams &p, int x, int y, int dx, int dy,
                                        int &xo, int &yo) {
  int xs = x + dx, ys = y + dy;
  if (p.y_walls) {
    if (ys < 0 || ys >= p.ny) {
      xo = p.x_open ? min(max(xs, 0), p.nx - 1) : wrapi(xs, p.nx);
      yo = ys < 0 ? 0 : p.ny - 1;
      return NB_SOLID;
    }
  } else {
    ys = wrapi(ys, p.ny);
  }
  yo = ys;
  if (!p.x_open) {
    xo = wrapi(xs, p.nx);
    return NB_FLUID;
  }
  if (xs < 0) { xo = 0; return NB_INLET; }
  if (xs >= p.nx) { xo = p.nx - 1; return NB_OUTLET; }
  xo = xs;
  return NB_FLUID;
}

// ---------------------------------------------------------------------------
// Pull-streaming (Eq. 12 indexed by destination) with half-way bounce-back on
// wall rows and Zou-He on the open columns (force-free form).
// gs: post-collision deviations of the previous update.  g: pulled deviations.
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ void pull_load(const DevParams &p, const typename S::T *__restrict__ gs,
                                          int x, int y, float g[9], unsigned &unknown) {
  const long long c = (long long)y * p.pitch + x;
  unknown = 0u;
  const bool interior = x > 0 && x < p.nx - 1 && y > 0 && y < p.ny - 1;
  if (interior) {
#pragma unroll
    for (int i = 0; i < 9; i++)
      g[i] = S::load(gs + i * p.plane + c - ey(i) * p.pitch - ex(i), i);
    return;
  }
#pragma unroll
  for (int i = 0; i < 9; i++) {
    int xo, yo;
    int k = classify(p, x, y, -ex(i), -ey(i), xo, yo);
    if (i == 0) {
      g[0] = S::load(gs + c, 0);
    } else if (k == NB_FLUID) {
      g[i] = S::load(gs + i * p.plane + (long long)yo * p.pitch + xo, i);
    } else {
      g[i] = S::load(gs + opp(i) * p.plane + c, opp(i));
      if (k == NB_INLET || k == NB_OUTLET) unknown |= 1u << i;
    }
  }
}

// Zou-He on the populations that entered from outside the x range (force-free form)
__device__ __forceinline__ void pull_fix(const DevParams &p, int x, const StepScalars &sc,
                                         float g[9], unsigned unknown) {
  if (!unknown) return;
  if (x == 0) {
    // f0+f2+f4+2(f3+f6+f7) has weight sum 1 -> rho_ref + deviations
    const float known = g[0] + g[2] + g[4] + 2.0f * (g[3] + g[6] + g[7]);
    float U, rb;
    if (p.p_inlet) {
      rb = sc.rho_in;  // pressure inlet: density given, velocity from the knowns
      U = (sc.rho_in - p.rho_ref - known) / sc.rho_in;
    } else {
      U = sc.u_in;     // velocity inlet
      rb = (known + p.rho_ref) / (1.0f - U);
    }
    if (unknown & (1u << 1)) g[1] = g[3] + (2.0f / 3.0f) * rb * U;
    const float d24 = 0.5f * (g[2] - g[4]), m6 = rb * U * (1.0f / 6.0f);
    if (unknown & (1u << 5)) g[5] = (g[7] - d24) + m6;
    if (unknown & (1u << 8)) g[8] = (g[6] + d24) + m6;
  }
  if (x == p.nx - 1) {
    const float ro = p.rho_out;
    const float U = (g[0] + g[2] + g[4] + 2.0f * (g[1] + g[5] + g[8]) + (p.rho_ref - ro)) / ro;
    if (unknown & (1u << 3)) g[3] = g[1] - (2.0f / 3.0f) * ro * U;
    const float d24 = 0.5f * (g[2] - g[4]), m6 = ro * U * (1.0f / 6.0f);
    if (unknown & (1u << 7)) g[7] = (g[5] + d24) - m6;
    if (unknown & (1u << 6)) g[6] = (g[8] - d24) - m6;
  }
}

template <class S>
__device__ __forceinline__ void pull(const DevParams &p, const typename S::T *__restrict__ gs, int x,
                                     int y, const StepScalars &sc, float g[9]) {
  unsigned unknown;
  pull_load<S>(p, gs, x, y, g, unknown);
  pull_fix(p, x, sc, g, unknown);
}

// Two-lane FP32 arithmetic: the packed add, multiply and fused multiply-add of sm_100 and
// later compute an x and a y term in one instruction.  Each lane rounds as the scalar
// operation does (round to nearest even; a - b as the fused (-1) b + a, which rounds once,
// like the subtraction), so a paired expression gives the bits of its scalar form.
struct P2 {
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) {
    return __ffma2_rn(make_float2(-1.0f, -1.0f), b, a);
  }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
  }
};

// rho u = sum e_i g_i + F/2 (Eq. 13; sum e_i w_i rho_ref = 0), summed in one fixed order
// wherever a velocity is formed, so that a node's velocity has the same bits whichever
// code path (collision or halo row) computes it
__device__ __forceinline__ void momentum(const float g[9], float Fx, float Fy, float &jxe,
                                         float &jye) {
  // x and y pairwise: (g1 - g3, g2 - g4) + (d57 - d68, d57 + d68), then + F/2
  const float2 d1324 = P2::sub(make_float2(g[1], g[2]), make_float2(g[3], g[4]));
  const float2 d5768 = P2::sub(make_float2(g[5], g[6]), make_float2(g[7], g[8]));
  const float2 dxy = make_float2(d5768.x - d5768.y, d5768.x + d5768.y);
  const float2 je = P2::fma(make_float2(0.5f, 0.5f), make_float2(Fx, Fy), P2::add(d1324, dxy));
  jxe = je.x;
  jye = je.y;
}

// sum of the nine deviations (density deviation, Eq. 13), opposite directions first and
// the x and y pairs in one two-lane add each
__device__ __forceinline__ float sum9(const float g[9]) {
  const float2 s1324 = P2::add(make_float2(g[1], g[2]), make_float2(g[3], g[4]));
  const float2 s5768 = P2::add(make_float2(g[5], g[6]), make_float2(g[7], g[8]));
  return g[0] + (s1324.x + s1324.y) + (s5768.x + s5768.y);
}

// ---------------------------------------------------------------------------
// Forces of Eqs. 9, 14 from the psi deviations of the 8 neighbours.
// dpsin[i]: psi(x+e_i) - psi_r (ignored when solid); dpsi_c: own psi - psi_r.
// With S = 3 sum_solid w e (exact: 3 w is 1 or 1/4) and the fluid part
// Q = 3 sum_fluid w dpsi e = (d1 - d3) + (d5 - d7 + d8 - d6) / 4 (x; y alike, solid
// neighbours counted as 0), the sum of Eq. 9 and Eq. 14 with the local psi as psi_w is
//   F = psi_c [ -G Q + ((G - Gw) psi_r - Gw dpsi_c) S ] / 3
//     = (-G psi_c / 3) Q + psi_c wc S / 3,
// written so that no two psi-sized terms cancel in FP32 and so that, with no solid
// neighbour (S = 0), F is the bulk product (-G psi_c / 3) Q bit for bit.
// Returns F and 9 |F_m|^2 / psi^2 = G^2 |Q - psi_r S|^2 (G^2 folded into c_theta).
// ---------------------------------------------------------------------------
struct Force {
  float Fx, Fy, fm2;
};

__device__ __forceinline__ Force interaction_force(const DevParams &p, float dpsi_c,
                                                   const float dpsin[9], unsigned solid_mask,
                                                   float psi_w_fixed) {
  float d[9];
  float Sx = 0.f, Sy = 0.f;
#pragma unroll
  for (int i = 1; i < 9; i++) {
    const bool sol = (solid_mask >> i) & 1u;
    d[i] = sol ? 0.0f : dpsin[i];
    Sx += sol ? (i <= 4 ? 1.0f : 0.25f) * ex(i) : 0.0f;
    Sy += sol ? (i <= 4 ? 1.0f : 0.25f) * ey(i) : 0.0f;
  }
  const float d57 = d[5] - d[7], d86 = d[8] - d[6];
  const float Qx = fmaf(0.25f, d57 + d86, d[1] - d[3]);
  const float Qy = fmaf(0.25f, d57 - d86, d[2] - d[4]);
  const float psi_c = p.psi_r + dpsi_c;
  // wall coefficient: local psi_w by default, a fixed psi(rho_w) when rho_w > 0
  const float wc = psi_w_fixed > 0.0f ? p.G * p.psi_r - p.Gw * psi_w_fixed
                                      : p.wall_r - p.Gw * dpsi_c;
  const float gpsi = fmaf(p.G3, dpsi_c, p.G3r);  // -G psi_c / 3
  const float ws = psi_c * wc * (1.0f / 3.0f);
  Force F;
  F.Fx = fmaf(ws, Sx, gpsi * Qx);
  F.Fy = fmaf(ws, Sy, gpsi * Qy);
  const float fx = fmaf(-p.psi_r, Sx, Qx), fy = fmaf(-p.psi_r, Sy, Qy);
  F.fm2 = fmaf(fx, fx, fy * fy);
  return F;
}

// ---------------------------------------------------------------------------
// Moment-space collision of Eq. 7 with Li's forcing (Eq. 8), written in closed
// form on the deviation populations.  In: pulled g, their sum drho = sum9(g),
// total force F, fm2 = 9 |sum w psi e|^2.  Out: post-collision deviations gs.
// Returns rho and u.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void collide(const DevParams &p, const float g[9], float drho, float Fx,
                                        float Fy, float fm2, float gs[9], float &rho_out,
                                        float &ux_out, float &uy_out) {
  // n = M g (Eq. 6 on deviations; m = n + rho_ref (1, -2, 1, 0, ...))
  // sums and differences of opposite directions, shared by the moments; the x and y
  // halves of each pair of like terms go through one two-lane instruction (P2 below)
  const float2 g12 = make_float2(g[1], g[2]), g34 = make_float2(g[3], g[4]);
  const float2 g56 = make_float2(g[5], g[6]), g78 = make_float2(g[7], g[8]);
  const float2 s1324 = P2::add(g12, g34), d1324 = P2::sub(g12, g34);
  const float2 s5768 = P2::add(g56, g78), d5768 = P2::sub(g56, g78);
  const float s13 = s1324.x, s24 = s1324.y, s57 = s5768.x, s68 = s5768.y;
  const float d57 = d5768.x, d68 = d5768.y;
  const float sa = s13 + s24, sd = s57 + s68;
  const float2 dxy = make_float2(d57 - d68, d57 + d68);  // diagonal parts of j
  const float n1 = fmaf(2.0f, sd, fmaf(-4.0f, g[0], -sa));
  const float n2 = fmaf(-2.0f, sa, fmaf(4.0f, g[0], sd));
  const float2 jxy = P2::add(d1324, dxy);
  const float2 n46 = P2::fma(make_float2(-2.0f, -2.0f), d1324, dxy);
  const float n7 = s13 - s24, n8 = s57 - s68;

  const float rho = p.rho_ref + drho;
  const float inv_rho = __fdividef(1.0f, rho);
  // rho u (Eq. 13): the tree of momentum() pairwise
  const float2 Fxy = make_float2(Fx, Fy);
  const float2 je = P2::fma(make_float2(0.5f, 0.5f), Fxy, jxy);
  const float2 uxy = P2::mul(je, make_float2(inv_rho, inv_rho));
  const float jxe = je.x, jye = je.y, ux = uxy.x, uy = uxy.y;
  // products are fused explicitly (fmaf) throughout, so that every copy of this code
  // rounds the same way
  const float uu = fmaf(jxe, ux, jye * uy);  // rho |u|^2 (the factor 3 is in k1[2], k2[2])
  const float uF = fmaf(ux, Fx, uy * Fy);

  // coefficients of a7 and a8 below: 0.25 (1 - s_nu), 0.25 s_nu, 0.25 (2 - s_nu) and
  // 0.25 (1 - s_nu / 2), from the parameters when s_nu is constant
  float c7a, c7b, c7c, c8c;
  if (p.tau_const) {
    c7a = p.kn[0];
    c7b = p.kn[1];
    c7c = p.kn[2];
    c8c = p.kn[3];
  } else {
    float fr = fminf(fmaxf((rho - p.rho_g) * p.inv_drho, 0.0f), 1.0f);
    const float s_nu = __fdividef(1.0f, p.tau_g + fr * p.dtau);  // Eq. 5
    c7b = 0.25f * s_nu;
    c7a = 0.25f - c7b;
    c7c = 0.5f - c7b;
    c8c = fmaf(-0.5f, c7b, 0.25f);
  }

  // m* - rho_ref c, moment by moment (Eq. 7) with (1 - s/2) S from Eq. 8, each already
  // divided by its D_k: a_k = (m*_k - rho_ref c_k) / D_k
  const float a0 = drho * (1.0f / 9.0f);
  const float a1 = fmaf(p.k1[4], fm2, fmaf(p.k1[3], uF, fmaf(p.k1[2], uu,
                                                               fmaf(p.k1[1], drho, p.k1[0] * n1))));
  const float a2 = fmaf(p.k2[4], fm2, fmaf(p.k2[3], uF, fmaf(p.k2[2], uu,
                                                               fmaf(p.k2[1], drho, p.k2[0] * n2))));
  const float2 a35 = P2::mul(P2::add(jxy, Fxy), make_float2(1.0f / 6.0f, 1.0f / 6.0f));
  const float2 a46 = P2::fma(make_float2(p.kq[2], p.kq[2]), Fxy,
                             P2::fma(make_float2(p.kq[1], p.kq[1]), je,
                                     P2::mul(make_float2(p.kq[0], p.kq[0]), n46)));
  const float a7 = fmaf(c7c, fmaf(ux, Fx, -(uy * Fy)),
                        fmaf(c7b, fmaf(jxe, ux, -(jye * uy)), c7a * n7));
  const float a8 = fmaf(c8c, fmaf(ux, Fy, uy * Fx), fmaf(c7b, jxe * uy, c7a * n8));
  // f* = M^-1 m* = M^T D^-1 m*
  const float b_ax = a0 - a1 - 2.0f * a2;   // common part of f1..f4
  const float b_dg = a0 + 2.0f * a1 + a2;   // common part of f5..f8
  const float2 pxy = P2::fma(make_float2(-2.0f, -2.0f), a46, a35);  // a3 - 2 a4, a5 - 2 a6
  const float2 t = P2::add(a35, a46);                                // a3 + a4, a5 + a6
  const float2 q = make_float2(t.x + t.y, t.y - t.x);               // qs, qd
  const float2 bx = make_float2(b_ax + a7, b_ax - a7), bd = make_float2(b_dg + a8, b_dg - a8);
  gs[0] = a0 - 4.0f * a1 + 4.0f * a2;
  const float2 g12o = P2::add(bx, pxy), g34o = P2::sub(bx, pxy);
  const float2 g56o = P2::add(bd, q), g78o = P2::sub(bd, q);
  gs[1] = g12o.x;
  gs[2] = g12o.y;
  gs[3] = g34o.x;
  gs[4] = g34o.y;
  gs[5] = g56o.x;
  gs[6] = g56o.y;
  gs[7] = g78o.x;
  gs[8] = g78o.y;
  rho_out = rho;
  ux_out = ux;
  uy_out = uy;
}

// wall temperature deviation at column x (linear between the two end values)
__device__ __forceinline__ float wall_T_dev(const DevParams &p, int x) {
  x = min(max(x, 0), p.nx - 1);
  return p.tw0 + p.tw_slope * (float)x;
}

__device__ __forceinline__ float wall_T_top_dev(const DevParams &p, int x) {
  x = min(max(x, 0), p.nx - 1);
  return p.tw0_top + p.tw_slope_top * (float)x;
}

// column x of the top (bottom) wall is adiabatic: outside the wall's isothermal window
__device__ __forceinline__ bool wall_adiabatic(const DevParams &p, int x, bool top) {
  const int x0 = top ? p.top_iso_x0 : p.bot_iso_x0, x1 = top ? p.top_iso_x1 : p.bot_iso_x1;
  return x1 > x0 && (x < x0 || x >= x1);
}

}  // namespace lbm
