// Fused lattice update: the per-tile sweep shared by the single-lattice kernel
// (lbm_fused.cu) and the batched kernel (lbm_fused_batch.cu).
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
#pragma once

#include "lbm_internal.h"

namespace lbm {

namespace {

#ifndef LBM_FUSED_THREADS
#define LBM_FUSED_THREADS 128
#endif
constexpr int FNT = LBM_FUSED_THREADS;  // threads per CTA, one lattice column each
#ifndef LBM_FUSED_MIN_CTAS
#define LBM_FUSED_MIN_CTAS (512 / LBM_FUSED_THREADS)
#endif
constexpr int FHALO = 5;             // psi is needed 5 nodes beyond the outputs
constexpr int FW = FNT - 2 * FHALO;  // output columns per CTA

struct FusedSmem {
  float4 pad_lo;        // neighbour reads of thread 0 below the first ring
  float psi[4][FNT];    // psi - psi_r, rows j-3 .. j
  float2 u[4][FNT];     // velocity, rows j-5 .. j-2
  float4 cf[4][FNT];    // energy coefficients of rho (cl, E1/(3 div u), E2/(3 div u), -), same rows
  float T[8][FNT];      // T - T_ref, rows j-5 .. j
  float T2[4][FNT], T3[4][FNT], T4[4][FNT];  // RK stage fields
  // own-column values of rows j-10 .. j-4: (ux/3, uy/3, cl, E1), (E2, Tb) and the RK4 sum
  float4 o1[8][FNT];
  float2 o2[8][FNT];
  float oacc[8][FNT];
  float4 pad_hi;        // neighbour reads of the last thread above the last ring
};

__device__ __forceinline__ int modi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Shared-memory ring access by a byte offset `off` of a float element (slot * FNT * 4 +
// column * 4; +-4 for the neighbouring columns); rings of float2 and float4 elements
// scale it by their element size, so one offset register serves every ring.
#define F1(ring, off) (*reinterpret_cast<float *>(reinterpret_cast<char *>(ring) + (off)))
#define F2(ring, off) (*reinterpret_cast<float2 *>(reinterpret_cast<char *>(ring) + 2 * (off)))
#define F4(ring, off) (*reinterpret_cast<float4 *>(reinterpret_cast<char *>(ring) + 4 * (off)))

// K(T) of Eq. 16 at one node from a 3-row ring window of the stage field, with
//   grad T = 3 sum w_i T(x+e_i) e_i = g / 3,    g_x = (T1 - T3) + (T5 - T7 + T8 - T6) / 4,
//   lap T = 6 sum w_i (T(x+e_i) - T(x)) = 2 L / 3,
//                                         L = (T1 + T2 + T3 + T4) + (T5 + T6 + T7 + T8) / 4 - 5T,
//   T (dP/dT)_rho div u / (rho Cv) = e1 T + e2 s (1 + kappa - kappa s),  s = sqrt(T/Tc),
// and, with x = T/Tc = s^2, the last term equal to E1 x + E2 s (E1 = e1 Tc - e2 kappa,
// E2 = e2 (1 + kappa)).  The caller passes us = u/3, cl = (2/3) lambda/(rho Cv), E1, E2:
//   K = -us.g + cl L - E1 x - E2 s.
__device__ __forceinline__ float rk_rate(const DevParams &p, float *__restrict__ R, int im,
                                         int i0, int ip, float uxs, float uys, float cl, float E1,
                                         float E2) {
  const float c = F1(R, i0);
  const float v1 = F1(R, i0 + 4), v3 = F1(R, i0 - 4), v2 = F1(R, ip), v4 = F1(R, im);
  const float v5 = F1(R, ip + 4), v6 = F1(R, ip - 4), v7 = F1(R, im - 4), v8 = F1(R, im + 4);
  const float d57 = v5 - v7, d86 = v8 - v6;
  const float gx = fmaf(0.25f, d57 + d86, v1 - v3);
  const float gy = fmaf(0.25f, d57 - d86, v2 - v4);
  const float lap = fmaf(-5.0f, c, fmaf(0.25f, (v5 + v7) + (v6 + v8), (v1 + v3) + (v2 + v4)));
  const float x = fmaf(c, p.inv_Tc, p.xr);  // T/Tc > 0 on fluid nodes
  const float s = x * rsqrtf(x);
  return fmaf(-E2, s, fmaf(-E1, x, fmaf(cl, lap, -fmaf(uxs, gx, uys * gy))));
}

// One tile of the fused update: output columns [X0, X0 + W) and rows [Y0, ye) of
// one lattice.  p supplies the bulk physics constants, pg the lattice's geometry and
// boundary data (sizes, walls, inlet/outlet, gravity).  Both kernels pass the same
// parameter set for the two; the split keeps the per-lattice fields apart from the
// constants that the single-lattice kernel reads from its constant bank.  Boundary modes and physics switches are
// compile-time parameters: YW walls in y, XO open ends in x, TH energy equation,
// MP pseudopotential forces; ST the population storage.
template <bool YW, bool XO, bool TH, bool MP, class ST, int U>
__device__ __forceinline__ void fused_tile(const DevParams &p, const DevParams &pg,
                                           const typename ST::T *__restrict__ gs,
                                           typename ST::T *__restrict__ gout,
                                           const float *__restrict__ Tin,
                                           float *__restrict__ Tout, unsigned *status,
                                           const StepScalars &sc, int X0, int W, int Y0, int ye,
                                           FusedSmem &S) {
  const int t = threadIdx.x;
  const int c = X0 - FHALO + t;  // lattice column of this thread

  // column kind: domain (wrapped when periodic) or a ghost beyond an open end
  bool col_in = false, col_out = false;
  int cx;
  if (!XO) {
    cx = modi(c, pg.nx);
  } else {
    col_in = c < 0;
    col_out = c >= pg.nx;
    cx = min(max(c, 0), pg.nx - 1);
  }
  const int xe = min(X0 + W, pg.nx);
  const int dxo = c < X0 ? X0 - c : (c >= xe ? c - xe + 1 : 0);  // columns outside the outputs
  // Ghost columns beyond an open end hold copies that the thread of the adjacent
  // boundary column writes into their ring slots (same thread, no race): the outlet
  // ghost copies column nx-1 (psi, T, u and the RK4 stage fields), the inlet ghost
  // copies psi of column 0 (zero gradient) and holds T_inlet, and with a pressure inlet
  // also copies the velocity of column 0.  Only the ghost column next to the domain is
  // read by a needed stencil, so the other ghost threads do no work in S0.
  const bool ghost = col_in || col_out;
  const bool mirror = XO && c == pg.nx - 1 && t + 1 < FNT;
  const bool mirror_in0 = XO && c == 0 && t >= 1;
  const bool mirror_in = mirror_in0 && pg.p_inlet;
  // the CTA holds a column of an open end (uniform over the CTA): only such CTAs have
  // Zou-He unknowns to fix
  const bool xb = XO && (c - t <= 0 || c - t + FNT - 1 >= pg.nx - 1);
  // Energy-equation ghosts of the walls (Section 3.2): isothermal columns hold the wall
  // temperature of their wall; on adiabatic columns every stage field's ghost copies the
  // fluid node across the wall: at the top the ghost row takes the value of row ny - 1
  // written one row step earlier, at the bottom row 0 writes its value into the slot of
  // row -1 (not read by any stage before then).  Adiabatic columns come with periodic x.
  const float twall = wall_T_dev(pg, cx), twall_top = wall_T_top_dev(pg, cx);
  // (lbm_create accepts adiabatic columns only with periodic x: compile-time false for open x)
  const bool adi_bot = YW && !XO && pg.adiabatic && wall_adiabatic(pg, cx, false);
  const bool adi_top = YW && !XO && pg.adiabatic && wall_adiabatic(pg, cx, true);

  // Pull offsets relative to the node's own index (Eq. 12, f_i(x) = f*_i(x - e_i)), used
  // on every row not next to a wall.  Next to a periodic seam the source column wraps;
  // at an open end the populations entering from outside (Zou-He unknowns) read any
  // in-bounds element of their plane and are replaced by pull_fix.
  int poff[9];
  unsigned unk_edge = 0u;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    poff[i] = i * (int)pg.plane - ey(i) * pg.pitch - ex(i);
    if (!XO) {
      if (cx == 0 && ex(i) == 1) poff[i] += pg.nx;
      if (cx == pg.nx - 1 && ex(i) == -1) poff[i] -= pg.nx;
    } else {
      if (cx == 0 && ex(i) == 1) unk_edge |= 1u << i;
      if (cx == pg.nx - 1 && ex(i) == -1) unk_edge |= 1u << i;
    }
  }

  unsigned st = 0;
  // running checks folded into status bits once at the end
  // (on deviations; the references are added once at the end)
  float chk = 0.0f;         // NaN propagates through the sum
  float drho_min = 0.0f;    // density must stay positive
  float drho_max = 0.0f;    // b rho must stay below the pole of Eq. 11
  float dT_min = 0.0f;      // absolute temperature must stay positive
  float fA[9], fB[9];
  float drhoA = 0.0f, drhoB = 0.0f;  // density deviations of the two newest pulled rows
#pragma unroll
  for (int i = 0; i < 9; i++) {
    fA[i] = 0.0f;
    fB[i] = 0.0f;
  }

  // float byte offset of ring row (j - k) at this thread's column, shared by every ring
  // and stage (R4(k), R8(k) below): q4[d] = 4 (((j + d) & 3) FNT + t),
  // q8[d] = 4 (((j + d) & 7) FNT + t), rotated by one position per row step
  int q4[4], q8[8];
#pragma unroll
  for (int d = 0; d < 4; d++) q4[d] = 4 * (d * FNT + t);
#pragma unroll
  for (int d = 0; d < 8; d++) q8[d] = 4 * (d * FNT + t);

  // Stage conditions depend on the row only (uniform over the CTA).  Within a stage every
  // thread computes, including halo threads outside the cone their stage is needed in
  // (stage k is needed for dxo <= 5 - k) and ghost columns beyond an open end: those
  // values are neither stored to global memory nor read by a needed column, and the
  // ring writes that a boundary column mirrors into a ghost slot are predicated off in
  // the ghost thread.  The pads around the rings keep the outermost threads' neighbour
  // reads in bounds.
  // Row ranges as one unsigned compare each: stage k (S1..S5) runs for 3k <= j < HR + 10 + k,
  // S0 for j < HR + 10, where HR is the number of output rows.
  const int HR = ye - Y0;
  const unsigned uny = (unsigned)pg.ny;
  const int J = HR + 3 * FHALO;
  // U = 2: two row steps per iteration, so that the compiler renames the rotated registers
  // within the pair (a step past J, when J is odd, runs no stage: every stage range ends
  // by J).  Measured, this pays in the single-lattice kernel (72.8 against 76.3 us on
  // 4096 x 512) and costs in the batched one (23.5 against 25.5 GLUPS on 96 channels).
  auto row_step = [&](const int j) {
    const int r = Y0 - FHALO + j;
#define R4(k) q4[(4 - ((k) & 3)) & 3]
#define R8(k) q8[(8 - ((k) & 7)) & 7]
    float *const ring_psi = &S.psi[0][0];
    float2 *const ring_u = &S.u[0][0];
    float4 *const ring_cf = &S.cf[0][0];
    float *const ring_T = &S.T[0][0];
    float *const ring_T2 = &S.T2[0][0];
    float *const ring_T3 = &S.T3[0][0];
    float *const ring_T4 = &S.T4[0][0];
    float4 *const ring_o1 = &S.o1[0][0];
    float2 *const ring_o2 = &S.o2[0][0];
    float *const ring_acc = &S.oacc[0][0];

    // ---------------- S0 loads: row r ----------------
    const bool s0_row = j < HR + 2 * FHALO;
    const bool r_solid = YW && (unsigned)r >= uny;
    const int ry = YW ? r : modi(r, pg.ny);
    float fc[9];
    unsigned unk = 0u;
    float Tc = 0.0f, drhoC = 0.0f;
    if (s0_row && !r_solid) {
      // ghost threads load their clamped column (in bounds) and never use it
      const int own = ry * pg.pitch + cx;
      if ((unsigned)(ry - 1) < (unsigned)(pg.ny - 2)) {  // 0 < ry < ny - 1
        const typename ST::T *src = gs + own;
#pragma unroll
        for (int i = 0; i < 9; i++) fc[i] = ST::load(src + poff[i], i);
        unk = ghost ? 0u : unk_edge;
      } else {
        pull_load<ST>(pg, gs, cx, ry, fc, unk);
        if (ghost) unk = 0u;
      }
      Tc = __ldg(Tin + own);
    } else {
#pragma unroll
      for (int i = 0; i < 9; i++) fc[i] = 0.0f;
    }

    // ---------------- S1: row r-2 (forces, velocity, collision) ----------------
    {
      const int q = r - 2;
      if ((unsigned)(j - 3) < (unsigned)(HR + 8)) {
        const int sl = R4(2);
        const bool solid = YW && (unsigned)q >= uny;
        if (solid) {
          if (TH) F2(ring_u, sl) = make_float2(0.0f, 0.0f);
        } else {
          const int qy = YW ? q : modi(q, pg.ny);
          const float drho = drhoB;
          const float rho = p.rho_ref + drho;
          Force F{0.0f, 0.0f, 0.0f};
          if (MP) {
            const int pm = R4(3), p0 = R4(2), pp = R4(1);
            const bool sdn = YW && q == 0;  // q is a fluid row here
            const bool sup = YW && q == pg.ny - 1;
            float dn[9];
            dn[0] = 0.0f;
            dn[1] = F1(ring_psi, p0 + 4);
            dn[2] = F1(ring_psi, pp);
            dn[3] = F1(ring_psi, p0 - 4);
            dn[4] = F1(ring_psi, pm);
            dn[5] = F1(ring_psi, pp + 4);
            dn[6] = F1(ring_psi, pp - 4);
            dn[7] = F1(ring_psi, pm - 4);
            dn[8] = F1(ring_psi, pm + 4);
            const float dpc = F1(ring_psi, p0);
            if (!sdn && !sup) {
              // no wall neighbour: F = -G psi sum w dpsi e  (Eq. 9; sum w e = 0), with
              // Q = 3 sum w dpsi e and fm2 = |Q|^2 = 9 |q|^2
              const float d57 = dn[5] - dn[7], d86 = dn[8] - dn[6];
              const float Qx = fmaf(0.25f, d57 + d86, dn[1] - dn[3]);
              const float Qy = fmaf(0.25f, d57 - d86, dn[2] - dn[4]);
              const float gpsi = fmaf(p.G3, dpc, p.G3r);  // -G psi / 3
              F.Fx = gpsi * Qx;
              F.Fy = gpsi * Qy;
              F.fm2 = fmaf(Qx, Qx, Qy * Qy);
            } else {
              unsigned solid_mask = 0u;
              if (sup) solid_mask |= (1u << 2) | (1u << 5) | (1u << 6);
              if (sdn) solid_mask |= (1u << 4) | (1u << 7) | (1u << 8);
              float psiw = 0.0f;
              if (pg.rho_w > 0.0f) {
                unsigned st_unused = 0;
                psiw = pseudopotential(pg, pg.rho_w, p.T_ref + F1(ring_T, R8(2)), st_unused);
              }
              F = interaction_force(pg, dpc, dn, solid_mask, psiw);
            }
          }
          if (pg.has_g) {
            const float rho_v = pg.drho_ref_g + drho;  // rho - rho_v of Eq. 15
            F.Fx += rho_v * pg.gx * sc.gcos;
            F.Fy += rho_v * pg.gy * sc.gcos;
          }
          float ux, uy;
          const float inv_rho = __fdividef(1.0f, rho);
          if ((unsigned)(q - Y0) < (unsigned)HR) {
            float gn[9], rr;
            collide(p, fB, drho, F.Fx, F.Fy, F.fm2, gn, rr, ux, uy);
            if (dxo == 0) {
              typename ST::T *dst = gout + (qy * pg.pitch + c);
#pragma unroll
              for (int i = 0; i < 9; i++) dst[i * (int)pg.plane] = ST::pack(gn[i], i);
              chk += ux + uy;  // rho enters at S0
            }
          } else {
            float jxe, jye;
            momentum(fB, F.Fx, F.Fy, jxe, jye);
            ux = jxe * inv_rho;
            uy = jye * inv_rho;
          }
          if (TH) {
            // the velocity inlet's ghost holds the inlet velocity; with a pressure inlet
            // column 0 mirrors its velocity there
            const float2 uu = col_in ? make_float2(sc.u_in, 0.0f) : make_float2(ux, uy);
            if (!col_out && !(col_in && pg.p_inlet)) F2(ring_u, sl) = uu;
            if (mirror) F2(ring_u, sl + 4) = uu;
            if (mirror_in) F2(ring_u, sl - 4) = uu;
            // energy coefficients of the node (see rk_rate): cl, E1 / (3 div u), E2 / (3 div u)
            const float br = p.eos_b * rho;
            const float z = __fdividef(p.akap1_cv3 * rho, fmaf(br, 2.0f - br, 1.0f));
            F4(ring_cf, sl) = make_float4(p.lam23_cv * inv_rho,
                                      __fdividef(p.RTc_cv3, 1.0f - br) - p.kappa_r * z, z, 0.0f);
          }
        }
      }
    }

    if (TH) {
      // ---------------- S2: row r-4 (div u, h1) ----------------
      {
        const int q = r - 4;
        if ((unsigned)(j - 6) < (unsigned)(HR + 6)) {
          const int sl = R4(4);
          const bool solid = YW && (unsigned)q >= uny;
          if (solid) {
            F1(ring_T2, sl) = q < 0 ? twall : (adi_top ? F1(ring_T2, R4(5)) : twall_top);
          } else {
            const int um = R4(5), u0 = R4(4), up = R4(3);
            const float2 a1 = F2(ring_u, u0 + 4), a3 = F2(ring_u, u0 - 4);
            const float2 a2 = F2(ring_u, up), a4 = F2(ring_u, um);
            const float2 a5 = F2(ring_u, up + 4), a6 = F2(ring_u, up - 4);
            const float2 a7 = F2(ring_u, um - 4), a8 = F2(ring_u, um + 4);
            // 3 div u = 9 sum w_i u(x+e_i).e_i (the 1/3 is folded into the cf coefficients)
            const float divu3 = ((a1.x - a3.x) + (a2.y - a4.y)) +
                                0.25f * ((a5.x + a5.y) - (a6.x - a6.y) - (a7.x + a7.y) +
                                         (a8.x - a8.y));
            const float2 uo = F2(ring_u, u0);
            const float4 cf = F4(ring_cf, u0);
            const float E1 = cf.y * divu3, E2 = cf.z * divu3;
            const float uxs = uo.x * (1.0f / 3.0f), uys = uo.y * (1.0f / 3.0f);
            const int t0 = R8(4);
            const float Tb = F1(ring_T, t0);
            const float h1 = rk_rate(p, ring_T, R8(5), t0, R8(3), uxs, uys, cf.x, E1, E2);
            const float v = col_in ? pg.T_inlet_dev : Tb + 0.5f * h1;
            if (!col_out) F1(ring_T2, sl) = v;
            if (mirror) F1(ring_T2, sl + 4) = v;
            if (adi_bot && q == 0) F1(ring_T2, R4(5)) = v;
            F4(ring_o1, t0) = make_float4(uxs, uys, cf.x, E1);
            F2(ring_o2, t0) = make_float2(E2, Tb);
            F1(ring_acc, t0) = h1;
          }
        }
      }
      // ---------------- S3: row r-6 (h2) ----------------
      {
        const int q = r - 6;
        if ((unsigned)(j - 9) < (unsigned)(HR + 4)) {
          const int sl = R4(6);
          const bool solid = YW && (unsigned)q >= uny;
          if (solid) {
            F1(ring_T3, sl) = q < 0 ? twall : (adi_top ? F1(ring_T3, R4(7)) : twall_top);
          } else {
            const int o = R8(6);
            const float4 w1 = F4(ring_o1, o);
            const float2 w2 = F2(ring_o2, o);
            const float h2 = rk_rate(p, ring_T2, R4(7), sl, R4(5), w1.x, w1.y, w1.z, w1.w, w2.x);
            const float v = col_in ? pg.T_inlet_dev : w2.y + 0.5f * h2;
            if (!col_out) F1(ring_T3, sl) = v;
            if (mirror) F1(ring_T3, sl + 4) = v;
            if (adi_bot && q == 0) F1(ring_T3, R4(7)) = v;
            F1(ring_acc, o) += 2.0f * h2;
          }
        }
      }
      // ---------------- S4: row r-8 (h3) ----------------
      {
        const int q = r - 8;
        if ((unsigned)(j - 12) < (unsigned)(HR + 2)) {
          const int sl = R4(8);
          const bool solid = YW && (unsigned)q >= uny;
          if (solid) {
            F1(ring_T4, sl) = q < 0 ? twall : (adi_top ? F1(ring_T4, R4(9)) : twall_top);
          } else {
            const int o = R8(8);
            const float4 w1 = F4(ring_o1, o);
            const float2 w2 = F2(ring_o2, o);
            const float h3 = rk_rate(p, ring_T3, R4(9), sl, R4(7), w1.x, w1.y, w1.z, w1.w, w2.x);
            const float v = col_in ? pg.T_inlet_dev : w2.y + h3;
            if (!col_out) F1(ring_T4, sl) = v;
            if (mirror) F1(ring_T4, sl + 4) = v;
            if (adi_bot && q == 0) F1(ring_T4, R4(9)) = v;
            F1(ring_acc, o) += 2.0f * h3;
          }
        }
      }
      // ---------------- S5: row r-10 (h4, new temperature) ----------------
      {
        const int q = r - 10;
        if ((unsigned)(j - 15) < (unsigned)HR) {
          const int o = R8(10);
          const float4 w1 = F4(ring_o1, o);
          const float2 w2 = F2(ring_o2, o);
          const float h4 = rk_rate(p, ring_T4, R4(11), R4(10), R4(9), w1.x, w1.y, w1.z, w1.w,
                                   w2.x);
          const float Tn = w2.y + (F1(ring_acc, o) + h4) * (1.0f / 6.0f);
          if (dxo == 0) {
            chk += Tn;
            dT_min = fminf(dT_min, Tn);
            Tout[q * pg.pitch + c] = Tn;
          }
        }
      }
    }

    // ---------------- S0 finish: row r ----------------
    if (s0_row) {
      const int sl = R4(0), sT = R8(0);
      if (r_solid) {
        F1(ring_T, sT) = r < 0 ? twall : (adi_top ? F1(ring_T, R8(1)) : twall_top);
        F1(ring_psi, sl) = 0.0f;
      } else {
        if (xb) pull_fix(pg, cx, sc, fc, unk);
        float dpsi = 0.0f;
        const float drho = sum9(fc);
        drhoC = drho;
        unsigned st_psi = 0u;
        if (MP) dpsi = pseudopotential_dev(p, drho, Tc, st_psi);
        if (!ghost) {
          st |= st_psi;  // a ghost's populations include unfixed placeholders
          F1(ring_T, sT) = Tc;
          F1(ring_psi, sl) = dpsi;
          drho_min = fminf(drho_min, drho);
          drho_max = fmaxf(drho_max, drho);
          dT_min = fminf(dT_min, Tc);
          chk += drho;
        }
        if (mirror) {
          F1(ring_T, sT + 4) = Tc;
          F1(ring_psi, sl + 4) = dpsi;
        }
        if (mirror_in0) {
          F1(ring_T, sT - 4) = pg.T_inlet_dev;
          F1(ring_psi, sl - 4) = dpsi;
        }
        if (adi_bot && r == 0) F1(ring_T, R8(1)) = Tc;
      }
    }
#pragma unroll
    for (int i = 0; i < 9; i++) {
      fB[i] = fA[i];
      fA[i] = fc[i];
    }
    drhoB = drhoA;
    drhoA = drhoC;
    {
      const int a = q4[0];
#pragma unroll
      for (int d = 0; d < 3; d++) q4[d] = q4[d + 1];
      q4[3] = a;
      const int b = q8[0];
#pragma unroll
      for (int d = 0; d < 7; d++) q8[d] = q8[d + 1];
      q8[7] = b;
    }
#undef R4
#undef R8
  };
  if constexpr (U == 2) {
#pragma unroll 1
    for (int j = 0; j < J; j += 2) {
      row_step(j);
      __syncthreads();
      row_step(j + 1);
      __syncthreads();
    }
  } else {
#pragma unroll 1
    for (int j = 0; j < J; j++) {
      row_step(j);
      __syncthreads();
    }
  }
  if (!isfinite(chk)) st |= ST_NAN;
  if (!(p.rho_ref + drho_min > 0.0f)) st |= ST_RHO_NONPOS;
  if (!(p.eos_b * (p.rho_ref + drho_max) < 1.0f)) st |= ST_EOS_POLE;
  if (!(p.T_ref + dT_min > 0.0f)) st |= ST_T_NONPOS;
  set_status(status, st);
}

}  // namespace

}  // namespace lbm
