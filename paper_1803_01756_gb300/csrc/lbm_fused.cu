// Fused lattice update: one launch per step, every intermediate on chip.
//
// A CTA owns FW output columns and a chunk of H output rows.  Its FNT threads
// each own one lattice column of [X0 - 5, X0 + FW + 5) and sweep the rows of the
// chunk (plus 5 halo rows on each side) from bottom to top.  Per swept row the
// update runs as six stages that trail each other by two rows:
//   S0 row r     : pull-streaming with boundary rules (Eq. 12), density (Eq. 13),
//                  pseudopotential deviation (Eqs. 10-11)            -> psi ring
//   S1 row r-2   : forces (Eqs. 9, 14, 15), velocity (Eq. 13), MRT collision with
//                  Li forcing (Eqs. 6-8) and the store of the populations
//   S2 row r-4   : div u and the first RK4 slope h1 of Eq. 16 (Eq. 18)
//   S3 row r-6   : h2      S4 row r-8 : h3      S5 row r-10 : h4 and Eq. 17
// Because each stage reads only rows that the stage before it finished in an
// earlier row step, one __syncthreads per row step orders all of them.  The
// 9-point stencils of psi, u and the stage temperatures need neighbour columns,
// which live in shared-memory row rings; own-column values (pulled populations
// of the two newest rows) stay in registers.  Global traffic per cell-update is
// the algorithmic minimum: the populations and T read once and written once,
// plus halo re-reads that hit L2.
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int FNT = 128;             // threads per CTA, one lattice column each
constexpr int FHALO = 5;             // psi is needed 5 nodes beyond the outputs
constexpr int FW = FNT - 2 * FHALO;  // output columns per CTA

struct FusedSmem {
  float psi[4][FNT];                         // psi - psi_r, rows j-3 .. j
  float ux[4][FNT], uy[4][FNT];              // velocity, rows j-5 .. j-2
  float cl[4][FNT], cA[4][FNT], cB[4][FNT];  // energy coefficients of rho, same rows
  float T[8][FNT];                           // T - T_ref, rows j-5 .. j
  float T2[4][FNT], T3[4][FNT], T4[4][FNT];  // RK stage fields
  // own-column values of rows j-10 .. j-4
  float oux[8][FNT], ouy[8][FNT], ocl[8][FNT], oe1[8][FNT], oe2[8][FNT], oTb[8][FNT],
      oacc[8][FNT];
};

__device__ __forceinline__ int modi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// K(T) of Eq. 16 at one node from a 3-row ring window of the stage field.
//   grad = 3 sum w_i T(x+e_i) e_i,  lap = 6 sum w_i (T(x+e_i) - T(x)),
//   K = -u.grad T + cl lap - e1 T - e2 s (1 + kappa - kappa s),  s = sqrt(T/Tc)
// where cl = lambda/(rho Cv) and e1, e2 carry (dP/dT)_rho T div u / (rho Cv).
__device__ __forceinline__ float rk_rate(const DevParams &p, const float *__restrict__ Rm,
                                         const float *__restrict__ R0,
                                         const float *__restrict__ Rp, int tl, int t, int tr,
                                         float ux, float uy, float cl, float e1, float e2) {
  const float c = R0[t];
  const float v1 = R0[tr], v3 = R0[tl], v2 = Rp[t], v4 = Rm[t];
  const float v5 = Rp[tr], v6 = Rp[tl], v7 = Rm[tl], v8 = Rm[tr];
  const float gx = (1.0f / 3.0f) * (v1 - v3) + (1.0f / 12.0f) * ((v5 - v7) + (v8 - v6));
  const float gy = (1.0f / 3.0f) * (v2 - v4) + (1.0f / 12.0f) * ((v5 - v7) + (v6 - v8));
  const float lap = (2.0f / 3.0f) * ((v1 + v3) + (v2 + v4) - 4.0f * c) +
                    (1.0f / 6.0f) * ((v5 + v7) + (v6 + v8) - 4.0f * c);
  const float Tabs = p.T_ref + c;
  const float s = sqrtf(Tabs * p.inv_Tc);
  return -(ux * gx + uy * gy) + cl * lap - e1 * Tabs - e2 * s * (1.0f + p.kappa - p.kappa * s);
}

__global__ void __launch_bounds__(FNT, 4)
    k_fused_step(DevParams p, const float *__restrict__ gs, float *__restrict__ gout,
                 const float *__restrict__ Tin, float *__restrict__ Tout, unsigned *status,
                 StepScalars sc, int H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmem &S = *reinterpret_cast<FusedSmem *>(smem_raw);

  const int t = threadIdx.x;
  const int X0 = blockIdx.x * FW;
  const int Y0 = blockIdx.y * H;
  const int ye = min(Y0 + H, p.ny);
  const int c = X0 - FHALO + t;  // lattice column of this thread

  // column kind: domain (wrapped when periodic) or a ghost beyond an open end
  bool col_in = false, col_out = false;
  int cx;
  if (!p.x_open) {
    cx = modi(c, p.nx);
  } else {
    col_in = c < 0;
    col_out = c >= p.nx;
    cx = min(max(c, 0), p.nx - 1);
  }
  const int xe = min(X0 + FW, p.nx);
  const int dxo = c < X0 ? X0 - c : (c >= xe ? c - xe + 1 : 0);  // columns outside the outputs
  const int tl = t - 1;
  // the outlet ghost copies column nx-1 for u and temperatures
  const int tr = (p.x_open && c + 1 >= p.nx) ? (p.nx - 1) - (X0 - FHALO) : t + 1;
  const float twall = wall_T_dev(p, cx);

  // pull offsets of an interior node relative to its own index (Eq. 12, f_i(x) = f*_i(x - e_i))
  int poff[9];
#pragma unroll
  for (int i = 0; i < 9; i++) poff[i] = i * (int)p.plane - ey(i) * p.pitch - ex(i);

  unsigned st = 0;
  float fA[9], fB[9];
#pragma unroll
  for (int i = 0; i < 9; i++) {
    fA[i] = 0.0f;
    fB[i] = 0.0f;
  }

  const int J = (ye - Y0) + 3 * FHALO;
#pragma unroll 1
  for (int j = 0; j < J; j++) {
    const int r = Y0 - FHALO + j;

    // ---------------- S0 loads: row r ----------------
    const bool s0_row = r < ye + FHALO;
    const bool r_solid = p.y_walls && (r < 0 || r >= p.ny);
    const int ry = p.y_walls ? r : modi(r, p.ny);
    float fc[9];
    unsigned unk = 0u;
    float Tc = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; i++) fc[i] = 0.0f;
    if (s0_row && !r_solid) {
      const int own = ry * p.pitch + cx;
      if (cx > 0 && cx < p.nx - 1 && ry > 0 && ry < p.ny - 1) {
        const float *src = gs + own;
#pragma unroll
        for (int i = 0; i < 9; i++) fc[i] = __ldg(src + poff[i]);
      } else {
        pull_load(p, gs, cx, ry, fc, unk);
      }
      Tc = __ldg(Tin + own);
    }

    // ---------------- S1: row r-2 (forces, velocity, collision) ----------------
    {
      const int q = r - 2;
      if (j >= 3 && q < ye + 4 && dxo <= 4) {
        const int sl = (j - 2) & 3;
        const bool solid = p.y_walls && (q < 0 || q >= p.ny);
        if (solid) {
          S.ux[sl][t] = 0.0f;
          S.uy[sl][t] = 0.0f;
        } else if (col_in) {
          S.ux[sl][t] = sc.u_in;
          S.uy[sl][t] = 0.0f;
        } else if (!col_out) {
          const int qy = p.y_walls ? q : modi(q, p.ny);
          const float drho = sum9(fB);
          const float rho = p.rho_ref + drho;
          Force F{0.0f, 0.0f, 0.0f};
          if (p.multiphase) {
            const int pm = (j - 3) & 3, p0 = (j - 2) & 3, pp = (j - 1) & 3;
            const bool sdn = p.y_walls && q - 1 < 0;
            const bool sup = p.y_walls && q + 1 >= p.ny;
            float dn[9];
            dn[0] = 0.0f;
            dn[1] = S.psi[p0][t + 1];
            dn[2] = S.psi[pp][t];
            dn[3] = S.psi[p0][t - 1];
            dn[4] = S.psi[pm][t];
            dn[5] = S.psi[pp][t + 1];
            dn[6] = S.psi[pp][t - 1];
            dn[7] = S.psi[pm][t - 1];
            dn[8] = S.psi[pm][t + 1];
            const float dpc = S.psi[p0][t];
            if (!sdn && !sup) {
              // no wall neighbour: F = -G psi sum w dpsi e  (Eq. 9; sum w e = 0)
              const float qx = (1.0f / 3.0f) * (dn[1] - dn[3]) +
                               (1.0f / 12.0f) * ((dn[5] - dn[7]) + (dn[8] - dn[6]));
              const float qy2 = (1.0f / 3.0f) * (dn[2] - dn[4]) +
                                (1.0f / 12.0f) * ((dn[5] - dn[7]) + (dn[6] - dn[8]));
              const float gpsi = -p.G * (p.psi_r + dpc);
              F.Fx = gpsi * qx;
              F.Fy = gpsi * qy2;
              F.fm2 = qx * qx + qy2 * qy2;
            } else {
              unsigned solid_mask = 0u;
              if (sup) solid_mask |= (1u << 2) | (1u << 5) | (1u << 6);
              if (sdn) solid_mask |= (1u << 4) | (1u << 7) | (1u << 8);
              float psiw = 0.0f;
              if (p.rho_w > 0.0f) {
                unsigned st_unused = 0;
                psiw = pseudopotential(p, p.rho_w, p.T_ref + S.T[(j - 2) & 7][t], st_unused);
              }
              F = interaction_force(p, dpc, dn, solid_mask, psiw);
            }
          }
          const float rho_v = p.drho_ref_g + drho;  // rho - rho_v of Eq. 15
          F.Fx += rho_v * p.gx * sc.gcos;
          F.Fy += rho_v * p.gy * sc.gcos;
          float ux, uy, inv_rho;
          if (dxo == 0 && q >= Y0 && q < ye) {
            float gn[9], rr;
            collide(p, fB, F.Fx, F.Fy, F.fm2, gn, rr, ux, uy);
            float *dst = gout + (qy * p.pitch + c);
#pragma unroll
            for (int i = 0; i < 9; i++) dst[i * (int)p.plane] = gn[i];
            if (!isfinite(rr + ux + uy)) st |= ST_NAN;
            inv_rho = 1.0f / rho;
          } else {
            inv_rho = 1.0f / rho;
            const float jx = (fB[1] - fB[3]) + (fB[5] - fB[7]) - (fB[6] - fB[8]);
            const float jy = (fB[2] - fB[4]) + (fB[5] - fB[7]) + (fB[6] - fB[8]);
            ux = (jx + 0.5f * F.Fx) * inv_rho;
            uy = (jy + 0.5f * F.Fy) * inv_rho;
          }
          S.ux[sl][t] = ux;
          S.uy[sl][t] = uy;
          const float br = p.eos_b * rho;
          S.cl[sl][t] = p.lam_cv * inv_rho;
          S.cA[sl][t] = p.R_cv / (1.0f - br);
          S.cB[sl][t] = p.akap_cv * rho / (1.0f + 2.0f * br - br * br);
        }
      }
    }

    if (p.thermal) {
      // ---------------- S2: row r-4 (div u, h1) ----------------
      {
        const int q = r - 4;
        if (j >= 6 && q < ye + 3 && dxo <= 3) {
          const int sl = (j - 4) & 3;
          const bool solid = p.y_walls && (q < 0 || q >= p.ny);
          if (solid) {
            S.T2[sl][t] = twall;
          } else if (col_in) {
            S.T2[sl][t] = p.T_inlet_dev;
          } else if (!col_out) {
            const int um = (j - 5) & 3, u0 = (j - 4) & 3, up = (j - 3) & 3;
            // div u = 3 sum w_i u(x+e_i).e_i
            const float divu =
                (1.0f / 3.0f) * ((S.ux[u0][tr] - S.ux[u0][tl]) + (S.uy[up][t] - S.uy[um][t])) +
                (1.0f / 12.0f) * ((S.ux[up][tr] + S.uy[up][tr]) - (S.ux[up][tl] - S.uy[up][tl]) -
                                  (S.ux[um][tl] + S.uy[um][tl]) + (S.ux[um][tr] - S.uy[um][tr]));
            const float uxo = S.ux[u0][t], uyo = S.uy[u0][t];
            const float cl = S.cl[u0][t];
            const float e1 = S.cA[u0][t] * divu, e2 = S.cB[u0][t] * divu;
            const float Tb = S.T[(j - 4) & 7][t];
            const float h1 = rk_rate(p, S.T[(j - 5) & 7], S.T[(j - 4) & 7], S.T[(j - 3) & 7], tl,
                                     t, tr, uxo, uyo, cl, e1, e2);
            S.T2[sl][t] = Tb + 0.5f * h1;
            const int o = (j - 4) & 7;
            S.oux[o][t] = uxo;
            S.ouy[o][t] = uyo;
            S.ocl[o][t] = cl;
            S.oe1[o][t] = e1;
            S.oe2[o][t] = e2;
            S.oTb[o][t] = Tb;
            S.oacc[o][t] = h1;
          }
        }
      }
      // ---------------- S3: row r-6 (h2) ----------------
      {
        const int q = r - 6;
        if (j >= 9 && q < ye + 2 && dxo <= 2) {
          const int sl = (j - 6) & 3;
          const bool solid = p.y_walls && (q < 0 || q >= p.ny);
          if (solid) {
            S.T3[sl][t] = twall;
          } else if (col_in) {
            S.T3[sl][t] = p.T_inlet_dev;
          } else if (!col_out) {
            const int o = (j - 6) & 7;
            const float h2 = rk_rate(p, S.T2[(j - 7) & 3], S.T2[(j - 6) & 3], S.T2[(j - 5) & 3], tl,
                                     t, tr, S.oux[o][t], S.ouy[o][t], S.ocl[o][t], S.oe1[o][t],
                                     S.oe2[o][t]);
            S.T3[sl][t] = S.oTb[o][t] + 0.5f * h2;
            S.oacc[o][t] += 2.0f * h2;
          }
        }
      }
      // ---------------- S4: row r-8 (h3) ----------------
      {
        const int q = r - 8;
        if (j >= 12 && q < ye + 1 && dxo <= 1) {
          const int sl = (j - 8) & 3;
          const bool solid = p.y_walls && (q < 0 || q >= p.ny);
          if (solid) {
            S.T4[sl][t] = twall;
          } else if (col_in) {
            S.T4[sl][t] = p.T_inlet_dev;
          } else if (!col_out) {
            const int o = (j - 8) & 7;
            const float h3 = rk_rate(p, S.T3[(j - 9) & 3], S.T3[(j - 8) & 3], S.T3[(j - 7) & 3], tl,
                                     t, tr, S.oux[o][t], S.ouy[o][t], S.ocl[o][t], S.oe1[o][t],
                                     S.oe2[o][t]);
            S.T4[sl][t] = S.oTb[o][t] + h3;
            S.oacc[o][t] += 2.0f * h3;
          }
        }
      }
      // ---------------- S5: row r-10 (h4, new temperature) ----------------
      {
        const int q = r - 10;
        if (j >= 15 && q < ye && dxo == 0) {
          const int o = (j - 10) & 7;
          const float h4 = rk_rate(p, S.T4[(j - 11) & 3], S.T4[(j - 10) & 3], S.T4[(j - 9) & 3],
                                   tl, t, tr, S.oux[o][t], S.ouy[o][t], S.ocl[o][t], S.oe1[o][t],
                                   S.oe2[o][t]);
          const float Tn = S.oTb[o][t] + (S.oacc[o][t] + h4) * (1.0f / 6.0f);
          if (!isfinite(Tn)) st |= ST_NAN;
          if (!(p.T_ref + Tn > 0.0f)) st |= ST_T_NONPOS;
          Tout[q * p.pitch + c] = Tn;
        }
      }
    }

    // ---------------- S0 finish: row r ----------------
    if (s0_row) {
      const int sl = j & 3, sT = j & 7;
      if (r_solid) {
        S.T[sT][t] = twall;
        S.psi[sl][t] = 0.0f;
      } else {
        pull_fix(p, cx, sc.u_in, fc, unk);
        S.T[sT][t] = col_in ? p.T_inlet_dev : Tc;
        float dpsi = 0.0f;
        const float drho = sum9(fc);
        if (p.multiphase) dpsi = pseudopotential_dev(p, drho, Tc, st);
        S.psi[sl][t] = dpsi;
        if (!col_in && !col_out) {
          const float rho = p.rho_ref + drho;
          if (!(rho > 0.0f)) st |= ST_RHO_NONPOS;
          if (p.eos_b * rho >= 1.0f) st |= ST_EOS_POLE;
          if (!(p.T_ref + Tc > 0.0f)) st |= ST_T_NONPOS;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 9; i++) {
      fB[i] = fA[i];
      fA[i] = fc[i];
    }
    __syncthreads();
  }
  set_status(status, st);
}

}  // namespace

// 32-bit element offsets cover all nine population planes
bool fused_supported(const DevParams &p) {
  return p.nx >= 1 && p.ny >= 1 && 9LL * p.plane + p.pitch < 2147483647LL;
}

int fused_chunk_rows(const DevParams &p, int device) {
  int sms = 0, occ = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(k_fused_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(FusedSmem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_step, FNT, sizeof(FusedSmem)) !=
          cudaSuccess ||
      occ < 1)
    return 0;
  const int strips = (p.nx + FW - 1) / FW;
  int chunks = (sms * occ) / strips;  // one wave of resident CTAs
  if (chunks < 1) chunks = 1;
  int H = (p.ny + chunks - 1) / chunks;
  if (H < 16) H = 16;  // keep the 10-row sweep overhead bounded
  return H;
}

cudaError_t launch_fused(const DevParams &p, const float *gs, float *gout, const float *Tin,
                         float *Tout, unsigned *status, StepScalars sc, int H, cudaStream_t s) {
  if (H < 1) return cudaErrorInvalidValue;
  dim3 grid((p.nx + FW - 1) / FW, (p.ny + H - 1) / H);
  k_fused_step<<<grid, FNT, sizeof(FusedSmem), s>>>(p, gs, gout, Tin, Tout, status, sc, H);
  return cudaGetLastError();
}

}  // namespace lbm
