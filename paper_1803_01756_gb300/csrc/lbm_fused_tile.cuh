// Fused lattice update: the per-tile sweep shared by the single-lattice kernel
// (lbm_fused_step.cuh) and the batched kernel (lbm_fused_batch.cu).
//
// A CTA of NT threads owns FW output columns and a chunk of H output rows.  Each
// thread owns CPT adjacent lattice columns of [X0 - FH, X0 - FH + NT * CPT) (FH halo
// columns on the left, at least 5 on the right) and sweeps the rows of the chunk
// (plus 5 halo rows on each side) from bottom to top.  Per swept row the update runs
// as six stages that trail each other by two rows:
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
//
// With CPT = 2 a thread reads the stencil rows of its two columns and their two
// outer neighbours with three shared-memory loads per row instead of six, shares
// the per-row bookkeeping between the columns, gives the scheduler two independent
// chains, and stores the populations and T of its column pair with 64-bit (FP32) or
// 32-bit (16-bit storage) stores; FH = 6 keeps every pair's first column even.
// Every column runs the same instructions whichever thread and slot hold it, so
// a node gets the same bits for any tiling and either CPT.
#pragma once

#include <type_traits>

#include "lbm_internal.h"

namespace lbm {

namespace {

#ifndef LBM_FUSED_THREADS
#define LBM_FUSED_THREADS 128
#endif
constexpr int FNT = LBM_FUSED_THREADS;  // threads per CTA of the CPT = 1 kernel
// Resident CTAs per SM that the register budget of the one-column kernels is sized for.
// For the full update (energy equation and pseudopotential forces) with FP32 storage three
// 128-thread CTAs (168 registers a thread) beat four (128): the six stages of a row step
// are independent chains, and the extra registers let the compiler overlap them (4096 x 512:
// 65.9 against 66.5 us per update, 1024 x 128: 15.7 against 16.3 us, the batched kernel
// 3 % faster).  Every other variant keeps four: with 16-bit storage (4096 x 512: 71.5
// against 76.2 us; the BF16 job server 27,200 against 24,700 jobs/h) and without the
// energy equation or the forces (58.0 against 52.9 us, 68.8 against 63.4 us), where the
// shorter row step needs the fourth CTA's warps to cover its latency.
constexpr int FMIN_F32 = 384 / FNT, FMIN_16 = 512 / FNT;

// left halo columns of a CTA: psi is needed 5 nodes beyond the outputs; with two columns
// per thread one more keeps the pairs aligned
__host__ __device__ constexpr int fused_halo(int cpt) { return cpt == 1 ? 5 : 6; }
// output columns of a CTA of nt threads with cpt columns each
__host__ __device__ constexpr int fused_width(int nt, int cpt) {
  return nt * cpt - fused_halo(cpt) - 5 - (cpt == 1 ? 0 : 1);
}
constexpr int FW = fused_width(FNT, 1);  // output columns of the CPT = 1 CTA

template <int NC>
struct FusedSmemT {
  float4 pad_lo;         // neighbour reads of the first column below the first ring
  float psi[4][NC];      // psi - psi_r, rows j-3 .. j
  float2 u[4][NC];       // velocity, rows j-5 .. j-2
  float4 cf[4][NC];      // energy coefficients of rho (E1/(3 div u), E2/(3 div u), cl, -), same rows
  float T[8][NC];        // T - T_ref, rows j-5 .. j
  float T2[4][NC], T3[4][NC], T4[4][NC];  // RK stage fields
  // own-column values of rows j-10 .. j-4: (ux/3, uy/3, cl, E1), (E2, Tb) and the RK4 sum
  float4 o1[8][NC];
  float2 o2[8][NC];
  float oacc[8][NC];
  float4 pad_hi;         // neighbour reads of the last column above the last ring
};
using FusedSmem = FusedSmemT<FNT>;

__device__ __forceinline__ int modi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Shared-memory ring access by a byte offset `off` of a float element (slot * NC * 4 +
// column * 4; +-4 for the neighbouring columns); rings of float2 and float4 elements
// scale it by their element size, so one offset register serves every ring.  PF1 and PF2
// address the pair of a thread's two columns in a float and a float2 ring.
#define F1(ring, off) (*reinterpret_cast<float *>(reinterpret_cast<char *>(ring) + (off)))
#define F2(ring, off) (*reinterpret_cast<float2 *>(reinterpret_cast<char *>(ring) + 2 * (off)))
#define F4(ring, off) (*reinterpret_cast<float4 *>(reinterpret_cast<char *>(ring) + 4 * (off)))
#define PF1(ring, off) (*reinterpret_cast<float2 *>(reinterpret_cast<char *>(ring) + (off)))
#define PF2(ring, off) (*reinterpret_cast<float4 *>(reinterpret_cast<char *>(ring) + 2 * (off)))

// One row of a float ring at the thread's CPT columns and one neighbour on each side:
// v[0] = first column - 1, v[1 .. CPT] the own columns, v[CPT + 1] = last column + 1.
template <int CPT>
__device__ __forceinline__ void ring_row(float *ring, int off, float (&v)[CPT + 2]) {
  v[0] = F1(ring, off - 4);
  if constexpr (CPT == 1) {
    v[1] = F1(ring, off);
  } else {
    const float2 a = PF1(ring, off);
    v[1] = a.x;
    v[2] = a.y;
  }
  v[CPT + 1] = F1(ring, off + 4 * CPT);
}

// the same for a float2 ring
template <int CPT>
__device__ __forceinline__ void ring_row2(float2 *ring, int off, float2 (&v)[CPT + 2]) {
  v[0] = F2(ring, off - 4);
  if constexpr (CPT == 1) {
    v[1] = F2(ring, off);
  } else {
    const float4 a = PF2(ring, off);
    v[1] = make_float2(a.x, a.y);
    v[2] = make_float2(a.z, a.w);
  }
  v[CPT + 1] = F2(ring, off + 4 * CPT);
}

// Store the thread's column values into a float ring: one vector store when every column
// writes, else one predicated store per column.
template <int CPT>
__device__ __forceinline__ void ring_put(float *ring, int off, const float (&v)[CPT], bool all,
                                         const bool (&w)[CPT]) {
  if constexpr (CPT == 2) {
    if (all) {
      PF1(ring, off) = make_float2(v[0], v[1]);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < CPT; k++)
    if (w[k]) F1(ring, off + 4 * k) = v[k];
}

template <int CPT>
__device__ __forceinline__ void ring_put2(float2 *ring, int off, const float2 (&v)[CPT], bool all,
                                          const bool (&w)[CPT]) {
  if constexpr (CPT == 2) {
    if (all) {
      PF2(ring, off) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < CPT; k++)
    if (w[k]) F2(ring, off + 4 * k) = v[k];
}

// K(T) of Eq. 16 at column k of a 3-row window of the stage field (rows m = q - 1,
// z = q, p = q + 1; index k + 1 is the node), with
//   grad T = 3 sum w_i T(x+e_i) e_i = g / 3,    g_x = (T1 - T3) + (T5 - T7 + T8 - T6) / 4,
//   lap T = 6 sum w_i (T(x+e_i) - T(x)) = 2 L / 3,
//                                         L = (T1 + T2 + T3 + T4) + (T5 + T6 + T7 + T8) / 4 - 5T,
//   T (dP/dT)_rho div u / (rho Cv) = e1 T + e2 s (1 + kappa - kappa s),  s = sqrt(T/Tc),
// and, with x = T/Tc = s^2, the last term equal to E1 x + E2 s (E1 = e1 Tc - e2 kappa,
// E2 = e2 (1 + kappa)).  The caller passes us = u/3, cl = (2/3) lambda/(rho Cv), E1, E2:
//   K = -us.g + cl L - E1 x - E2 s.
template <int CPT>
__device__ __forceinline__ float rk_rate(const DevParams &p, const float (&m)[CPT + 2],
                                         const float (&z)[CPT + 2], const float (&pp)[CPT + 2],
                                         int k, float uxs, float uys, float cl, float E1,
                                         float E2) {
  const float c = z[k + 1];
  // the x and y terms pairwise: (v1, v2) -+ (v3, v4) and (v5, v8) -+ (v7, v6)
  const float2 v12 = make_float2(z[k + 2], pp[k + 1]), v34 = make_float2(z[k], m[k + 1]);
  const float2 v58 = make_float2(pp[k + 2], m[k + 2]), v76 = make_float2(m[k], pp[k]);
  const float2 d1324 = P2::sub(v12, v34), s1324 = P2::add(v12, v34);
  const float2 d5786 = P2::sub(v58, v76), s5786 = P2::add(v58, v76);
  const float d57 = d5786.x, d86 = d5786.y;
  const float2 g = P2::fma(make_float2(0.25f, 0.25f), make_float2(d57 + d86, d57 - d86), d1324);
  const float gx = g.x, gy = g.y;
  const float lap = fmaf(-5.0f, c, fmaf(0.25f, s5786.x + s5786.y, s1324.x + s1324.y));
  const float x = fmaf(c, p.inv_Tc, p.xr);  // T/Tc > 0 on fluid nodes
  const float s = x * rsqrtf(x);
  return fmaf(-E2, s, fmaf(-E1, x, fmaf(cl, lap, -fmaf(uxs, gx, uys * gy))));
}

// Store the populations of the thread's output columns of one row: a vector store of the
// column pair when both are outputs (the first column is even, so the pair is aligned).
template <class ST, int CPT>
__device__ __forceinline__ void store_pops(typename ST::T *__restrict__ dst, int plane,
                                           const float (&gn)[CPT][9], const bool (&out)[CPT]) {
  if constexpr (CPT == 2) {
    if (out[0] && out[1]) {
#pragma unroll
      for (int i = 0; i < 9; i++) ST::store2(dst + i * plane, gn[0][i], gn[1][i], i);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < CPT; k++)
    if (out[k]) {
#pragma unroll
      for (int i = 0; i < 9; i++) dst[i * plane + k] = ST::pack(gn[k][i], i);
    }
}

// One tile of the fused update: output columns [X0, X0 + W) and rows [Y0, ye) of
// one lattice.  p supplies the bulk physics constants, pg the lattice's geometry and
// boundary data (sizes, walls, inlet/outlet, gravity).  Both kernels pass the same
// parameter set for the two; the split keeps the per-lattice fields apart from the
// constants that the single-lattice kernel reads from its constant bank.  Boundary modes and physics switches are
// compile-time parameters: YW walls in y, XO open ends in x, TH energy equation,
// MP pseudopotential forces; ST the population storage; U row steps per loop
// iteration; NT threads of CPT columns each.  With CPT = 2, X0 must be even.
template <bool YW, bool XO, bool TH, bool MP, class ST, int U, int NT, int CPT>
__device__ __forceinline__ void fused_tile(const DevParams &p, const DevParams &pg,
                                           const typename ST::T *__restrict__ gs,
                                           typename ST::T *__restrict__ gout,
                                           const float *__restrict__ Tin,
                                           float *__restrict__ Tout, unsigned *status,
                                           const StepScalars &sc, int X0, int W, int Y0, int ye,
                                           FusedSmemT<NT * CPT> &S) {
  constexpr int NC = NT * CPT;
  constexpr int FH = fused_halo(CPT);
  const int t = threadIdx.x;
  const int c0 = X0 - FH + CPT * t;  // lattice column of this thread's first column
  const int xe = min(X0 + W, pg.nx);

  // Per column: kind (domain, wrapped when periodic, or a ghost beyond an open end).
  // Ghost columns beyond an open end hold copies that the thread of the adjacent
  // boundary column writes into their ring slots (no race: a ghost never writes its own
  // slot): the outlet ghost copies column nx-1 (psi, T, u and the RK4 stage fields), the
  // inlet ghost copies psi of column 0 (zero gradient) and holds T_inlet, and with a
  // pressure inlet also copies the velocity of column 0.  Only the ghost column next to
  // the domain is read by a needed stencil, so the other ghosts' values do not matter.
  // Energy-equation ghosts of the walls (Section 3.2): isothermal columns hold the wall
  // temperature of their wall; on adiabatic columns every stage field's ghost copies the
  // fluid node across the wall: at the top the ghost row takes the value of row ny - 1
  // written one row step earlier, at the bottom row 0 writes its value into the slot of
  // row -1 (not read by any stage before then).  Adiabatic columns come with periodic x
  // (lbm_create accepts them only then: compile-time false for open x).
  // per-column cases as bits of one register per column (the kernel runs at its register
  // bound): FL_IN / FL_OUT ghost beyond the inlet / outlet, FL_OUTC output column, FL_MIR /
  // FL_MIN0 the boundary column that mirrors into the outlet / inlet ghost slot (FL_MIN:
  // also the velocity, pressure inlet), FL_ADB / FL_ADT adiabatic bottom / top wall column
  enum : unsigned { FL_IN = 1u, FL_OUT = 2u, FL_OUTC = 4u, FL_MIR = 8u, FL_MIN0 = 16u,
                    FL_MIN = 32u, FL_ADB = 64u, FL_ADT = 128u };
  int cx[CPT];
  unsigned fl[CPT];
  // Pull offsets relative to the node's own index (Eq. 12, f_i(x) = f*_i(x - e_i)), used
  // on every row not next to a wall.  Next to a periodic seam the source column wraps;
  // at an open end the populations entering from outside (Zou-He unknowns) read any
  // in-bounds element of their plane and are replaced by pull_fix.
  int poff[CPT][9];
  unsigned unk_edge[CPT];
#pragma unroll
  for (int k = 0; k < CPT; k++) {
    const int c = c0 + k, lc = CPT * t + k;
    unsigned f = 0u;
    if (!XO) {
      cx[k] = modi(c, pg.nx);
    } else {
      f |= c < 0 ? FL_IN : 0u;
      f |= c >= pg.nx ? FL_OUT : 0u;
      cx[k] = min(max(c, 0), pg.nx - 1);
    }
    f |= c >= X0 && c < xe ? FL_OUTC : 0u;
    f |= XO && c == pg.nx - 1 && lc + 1 < NC ? FL_MIR : 0u;
    f |= XO && c == 0 && lc >= 1 ? FL_MIN0 : 0u;
    f |= XO && c == 0 && lc >= 1 && pg.p_inlet ? FL_MIN : 0u;
    f |= YW && !XO && pg.adiabatic && wall_adiabatic(pg, cx[k], false) ? FL_ADB : 0u;
    f |= YW && !XO && pg.adiabatic && wall_adiabatic(pg, cx[k], true) ? FL_ADT : 0u;
    fl[k] = f;
    unk_edge[k] = 0u;
#pragma unroll
    for (int i = 0; i < 9; i++) {
      poff[k][i] = i * (int)pg.plane - ey(i) * pg.pitch - ex(i);
      if (!XO) {
        if (cx[k] == 0 && ex(i) == 1) poff[k][i] += pg.nx;
        if (cx[k] == pg.nx - 1 && ex(i) == -1) poff[k][i] -= pg.nx;
      } else {
        if (cx[k] == 0 && ex(i) == 1) unk_edge[k] |= 1u << i;
        if (cx[k] == pg.nx - 1 && ex(i) == -1) unk_edge[k] |= 1u << i;
      }
    }
  }
#define HAS(k, b) ((fl[k] & (b)) != 0u)
  // the column writes its own ring slot in S0 (not a ghost), in S1's velocity ring (not
  // the outlet ghost, not the pressure inlet's ghost) and in the stage rings (not the
  // outlet ghost); wall temperatures are formed where a wall row needs them
  bool wS0[CPT], wU[CPT], wT[CPT], outc[CPT];
  bool allS0 = true, allU = true, allT = true;
#pragma unroll
  for (int k = 0; k < CPT; k++) {
    wS0[k] = !HAS(k, FL_IN | FL_OUT);
    wU[k] = !HAS(k, FL_OUT) && !(HAS(k, FL_IN) && pg.p_inlet);
    wT[k] = !HAS(k, FL_OUT);
    outc[k] = HAS(k, FL_OUTC);
    allS0 = allS0 && wS0[k];
    allU = allU && wU[k];
    allT = allT && wT[k];
  }
#define TWALL(k) wall_T_dev(pg, cx[k])
#define TWALL_TOP(k) wall_T_top_dev(pg, cx[k])
  // the CTA holds a column of an open end (uniform over the CTA): only such CTAs have
  // Zou-He unknowns to fix
  const bool xb = XO && (X0 - FH <= 0 || X0 - FH + NC - 1 >= pg.nx - 1);

  unsigned st = 0;
  // running checks folded into status bits once at the end
  // (on deviations; the references are added once at the end)
  float chk = 0.0f;         // NaN propagates through the sum
  float drho_min = 0.0f;    // density must stay positive
  float drho_max = 0.0f;    // b rho must stay below the pole of Eq. 11
  float dT_min = 0.0f;      // absolute temperature must stay positive
  float fA[CPT][9], fB[CPT][9];
  float drhoA[CPT], drhoB[CPT];  // density deviations of the two newest pulled rows
#pragma unroll
  for (int k = 0; k < CPT; k++) {
    drhoA[k] = 0.0f;
    drhoB[k] = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; i++) {
      fA[k][i] = 0.0f;
      fB[k][i] = 0.0f;
    }
  }

  // float byte offset of ring row (j - k) at this thread's first column, shared by every
  // ring and stage (R4(k), R8(k) below): q4[d] = 4 (((j + d) & 3) NC + CPT t),
  // q8[d] = 4 (((j + d) & 7) NC + CPT t), rotated by one position per row step.  The rings
  // of own-column values (cf, o1, o2, oacc) hold column k of thread t at k NT + t of the
  // slot (column-major over the thread's columns, so each column's access is
  // conflict-free): OWN(q, k) = q - 4 (CPT - 1) t + 4 k NT.
  int q4[4], q8[8];
#pragma unroll
  for (int d = 0; d < 4; d++) q4[d] = 4 * (d * NC + CPT * t);
#pragma unroll
  for (int d = 0; d < 8; d++) q8[d] = 4 * (d * NC + CPT * t);
  const int tsh = 4 * (CPT - 1) * t;
#define OWN(q, k) ((q) - tsh + 4 * (k) * NT)

  // Stage conditions depend on the row only (uniform over the CTA).  Within a stage every
  // thread computes, including halo columns outside the cone their stage is needed in
  // (stage k is needed within 5 - k columns of the outputs) and ghost columns beyond an
  // open end: those values are neither stored to global memory nor read by a needed
  // column, and the ring writes that a boundary column mirrors into a ghost slot are
  // predicated off in the ghost's own write.  The pads around the rings keep the
  // outermost threads' neighbour reads in bounds.
  // Row ranges as one unsigned compare each: stage k (S1..S5) runs for 3k <= j < HR + 10 + k,
  // S0 for j < HR + 10, where HR is the number of output rows.
  const int HR = ye - Y0;
  const unsigned uny = (unsigned)pg.ny;
  const int J = HR + 15;
  // U = 2: two row steps per loop iteration, so that the compiler renames the rotated
  // registers within the pair (a step past J, when J is odd, runs no stage: every stage
  // range ends by J).  Each stage stores its ring values as soon as it has them: deferring
  // all of a row step's ring stores to its end (no stage reads a slot another stage
  // writes in the same step) raised the issue rate of the one-column kernel from 2.55 to
  // 2.74 per cycle but added 14 % instructions at its 128-register bound, a net loss.
  auto row_step = [&](const int j) {
    const int r = Y0 - 5 + j;
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
    const bool s0_row = j < HR + 10;
    const bool r_solid = YW && (unsigned)r >= uny;
    const int ry = YW ? r : modi(r, pg.ny);
    float fc[CPT][9];
    unsigned unk[CPT];
    float Tc[CPT], drhoC[CPT];
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      unk[k] = 0u;
      Tc[k] = 0.0f;
      drhoC[k] = 0.0f;
    }
    if (s0_row && !r_solid) {
#pragma unroll
      for (int k = 0; k < CPT; k++) {
        // ghost columns load their clamped column (in bounds) and never use it
        const int own = ry * pg.pitch + cx[k];
        if ((unsigned)(ry - 1) < (unsigned)(pg.ny - 2)) {  // 0 < ry < ny - 1
          const typename ST::T *src = gs + own;
#pragma unroll
          for (int i = 0; i < 9; i++) fc[k][i] = ST::load(src + poff[k][i], i);
          unk[k] = HAS(k, FL_IN | FL_OUT) ? 0u : unk_edge[k];
        } else {
          pull_load<ST>(pg, gs, cx[k], ry, fc[k], unk[k]);
          if (HAS(k, FL_IN | FL_OUT)) unk[k] = 0u;
        }
        Tc[k] = __ldg(Tin + own);
      }
    } else {
#pragma unroll
      for (int k = 0; k < CPT; k++)
#pragma unroll
        for (int i = 0; i < 9; i++) fc[k][i] = 0.0f;
    }

    // ---------------- S1: row r-2 (forces, velocity, collision) ----------------
    {
      const int q = r - 2;
      if ((unsigned)(j - 3) < (unsigned)(HR + 8)) {
        const int sl = R4(2);
        const bool solid = YW && (unsigned)q >= uny;
        if (solid) {
          if (TH) {
            float2 z2[CPT];
            bool yes[CPT];
#pragma unroll
            for (int k = 0; k < CPT; k++) {
              z2[k] = make_float2(0.0f, 0.0f);
              yes[k] = true;
            }
            ring_put2<CPT>(ring_u, sl, z2, true, yes);
          }
        } else {
          const int qy = YW ? q : modi(q, pg.ny);
          Force F[CPT];
#pragma unroll
          for (int k = 0; k < CPT; k++) F[k] = Force{0.0f, 0.0f, 0.0f};
          if (MP) {
            float wm[CPT + 2], w0[CPT + 2], wp[CPT + 2];
            ring_row<CPT>(ring_psi, R4(3), wm);
            ring_row<CPT>(ring_psi, R4(2), w0);
            ring_row<CPT>(ring_psi, R4(1), wp);
            const bool sdn = YW && q == 0;  // q is a fluid row here
            const bool sup = YW && q == pg.ny - 1;
#pragma unroll
            for (int k = 0; k < CPT; k++) {
              float dn[9];
              dn[0] = 0.0f;
              dn[1] = w0[k + 2];
              dn[2] = wp[k + 1];
              dn[3] = w0[k];
              dn[4] = wm[k + 1];
              dn[5] = wp[k + 2];
              dn[6] = wp[k];
              dn[7] = wm[k];
              dn[8] = wm[k + 2];
              const float dpc = w0[k + 1];
              if (!sdn && !sup) {
                // no wall neighbour: F = -G psi sum w dpsi e  (Eq. 9; sum w e = 0), with
                // Q = 3 sum w dpsi e and fm2 = |Q|^2 = 9 |q|^2
                // (x and y terms pairwise, as in rk_rate)
                const float2 d5786 = P2::sub(make_float2(dn[5], dn[8]), make_float2(dn[7], dn[6]));
                const float2 d1324 = P2::sub(make_float2(dn[1], dn[2]), make_float2(dn[3], dn[4]));
                const float d57 = d5786.x, d86 = d5786.y;
                const float2 Q = P2::fma(make_float2(0.25f, 0.25f),
                                         make_float2(d57 + d86, d57 - d86), d1324);
                const float gpsi = fmaf(p.G3, dpc, p.G3r);  // -G psi / 3
                const float2 Fq = P2::mul(make_float2(gpsi, gpsi), Q);
                F[k].Fx = Fq.x;
                F[k].Fy = Fq.y;
                F[k].fm2 = fmaf(Q.x, Q.x, Q.y * Q.y);
              } else {
                unsigned solid_mask = 0u;
                if (sup) solid_mask |= (1u << 2) | (1u << 5) | (1u << 6);
                if (sdn) solid_mask |= (1u << 4) | (1u << 7) | (1u << 8);
                float psiw = 0.0f;
                if (pg.rho_w > 0.0f) {
                  unsigned st_unused = 0;
                  psiw = pseudopotential(pg, pg.rho_w, p.T_ref + F1(ring_T, R8(2) + 4 * k),
                                         st_unused);
                }
                F[k] = interaction_force(pg, dpc, dn, solid_mask, psiw);
              }
            }
          }
          float ux[CPT], uy[CPT], rho[CPT], inv_rho[CPT];
#pragma unroll
          for (int k = 0; k < CPT; k++) {
            const float drho = drhoB[k];
            rho[k] = p.rho_ref + drho;
            if (pg.has_g) {
              const float rho_v = pg.drho_ref_g + drho;  // rho - rho_v of Eq. 15
              F[k].Fx += rho_v * pg.gx * sc.gcos;
              F[k].Fy += rho_v * pg.gy * sc.gcos;
            }
            inv_rho[k] = __fdividef(1.0f, rho[k]);
          }
          if ((unsigned)(q - Y0) < (unsigned)HR) {
            float gn[CPT][9];
#pragma unroll
            for (int k = 0; k < CPT; k++) {
              float rr;
              collide(p, fB[k], drhoB[k], F[k].Fx, F[k].Fy, F[k].fm2, gn[k], rr, ux[k], uy[k]);
              if (outc[k]) chk += ux[k] + uy[k];  // rho enters at S0
            }
            store_pops<ST, CPT>(gout + (qy * pg.pitch + c0), (int)pg.plane, gn, outc);
          } else {
#pragma unroll
            for (int k = 0; k < CPT; k++) {
              float jxe, jye;
              momentum(fB[k], F[k].Fx, F[k].Fy, jxe, jye);
              const float2 u2 = P2::mul(make_float2(jxe, jye), make_float2(inv_rho[k], inv_rho[k]));
              ux[k] = u2.x;
              uy[k] = u2.y;
            }
          }
          if (TH) {
            // the velocity inlet's ghost holds the inlet velocity; with a pressure inlet
            // column 0 mirrors its velocity there
            float2 uu[CPT];
#pragma unroll
            for (int k = 0; k < CPT; k++)
              uu[k] = HAS(k, FL_IN) ? make_float2(sc.u_in, 0.0f) : make_float2(ux[k], uy[k]);
            ring_put2<CPT>(ring_u, sl, uu, allU, wU);
#pragma unroll
            for (int k = 0; k < CPT; k++) {
              if (HAS(k, FL_MIR)) F2(ring_u, sl + 4 * k + 4) = uu[k];
              if (HAS(k, FL_MIN)) F2(ring_u, sl + 4 * k - 4) = uu[k];
              // energy coefficients of the node (see rk_rate): E1 / (3 div u), E2 / (3 div u), cl
              const float br = p.eos_b * rho[k];
              const float z = __fdividef(p.akap1_cv3 * rho[k], fmaf(br, 2.0f - br, 1.0f));
              F4(ring_cf, OWN(sl, k)) =
                  make_float4(__fdividef(p.RTc_cv3, 1.0f - br) - p.kappa_r * z, z,
                              p.lam23_cv * inv_rho[k], 0.0f);
            }
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
#pragma unroll
            for (int k = 0; k < CPT; k++)
              F1(ring_T2, sl + 4 * k) =
                  q < 0 ? TWALL(k) : (HAS(k, FL_ADT) ? F1(ring_T2, R4(5) + 4 * k) : TWALL_TOP(k));
          } else {
            float2 um[CPT + 2], u0[CPT + 2], up[CPT + 2];
            ring_row2<CPT>(ring_u, R4(5), um);
            ring_row2<CPT>(ring_u, R4(4), u0);
            ring_row2<CPT>(ring_u, R4(3), up);
            float tm[CPT + 2], t0[CPT + 2], tp[CPT + 2];
            ring_row<CPT>(ring_T, R8(5), tm);
            ring_row<CPT>(ring_T, R8(4), t0);
            ring_row<CPT>(ring_T, R8(3), tp);
            const int o = R8(4);
            float v[CPT];
#pragma unroll
            for (int k = 0; k < CPT; k++) {
              const float2 a1 = u0[k + 2], a3 = u0[k];
              const float2 a2 = up[k + 1], a4 = um[k + 1];
              const float2 a5 = up[k + 2], a6 = up[k];
              const float2 a7 = um[k], a8 = um[k + 2];
              // 3 div u = 9 sum w_i u(x+e_i).e_i (the 1/3 is folded into the cf coefficients);
              // the diagonal part (u5 - u7) + (u8 - u6) with x and y pairwise
              const float2 d57 = P2::sub(a5, a7), d86 = P2::sub(a8, a6);
              const float divu3 = ((a1.x - a3.x) + (a2.y - a4.y)) +
                                  0.25f * ((d57.x + d86.x) + (d57.y - d86.y));
              const float4 cf = F4(ring_cf, OWN(R4(4), k));
              const float2 E = P2::mul(make_float2(cf.x, cf.y), make_float2(divu3, divu3));
              const float2 us = P2::mul(u0[k + 1], make_float2(1.0f / 3.0f, 1.0f / 3.0f));
              const float Tb = t0[k + 1];
              const float h1 = rk_rate<CPT>(p, tm, t0, tp, k, us.x, us.y, cf.z, E.x, E.y);
              v[k] = HAS(k, FL_IN) ? pg.T_inlet_dev : Tb + 0.5f * h1;
              F4(ring_o1, OWN(o, k)) = make_float4(us.x, us.y, cf.z, E.x);
              F2(ring_o2, OWN(o, k)) = make_float2(E.y, Tb);
              F1(ring_acc, OWN(o, k)) = h1;
            }
            ring_put<CPT>(ring_T2, sl, v, allT, wT);
#pragma unroll
            for (int k = 0; k < CPT; k++) {
              if (HAS(k, FL_MIR)) F1(ring_T2, sl + 4 * k + 4) = v[k];
              if (HAS(k, FL_ADB) && q == 0) F1(ring_T2, R4(5) + 4 * k) = v[k];
            }
          }
        }
      }
      // ---------------- S3: row r-6 (h2) and S4: row r-8 (h3) ----------------
      // T2 -> T3 with the half step, T3 -> T4 with the full step
      auto mid_stage = [&](const int q, const bool active, const int sl, const int below,
                           const int above, const int o, float *const src, float *const dst,
                           const bool full) {
        if (!active) return;
        const bool solid = YW && (unsigned)q >= uny;
        if (solid) {
#pragma unroll
          for (int k = 0; k < CPT; k++)
            F1(dst, sl + 4 * k) =
                q < 0 ? TWALL(k) : (HAS(k, FL_ADT) ? F1(dst, below + 4 * k) : TWALL_TOP(k));
        } else {
          float sm[CPT + 2], s0[CPT + 2], sp[CPT + 2];
          ring_row<CPT>(src, below, sm);
          ring_row<CPT>(src, sl, s0);
          ring_row<CPT>(src, above, sp);
          float v[CPT];
#pragma unroll
          for (int k = 0; k < CPT; k++) {
            const float4 w1 = F4(ring_o1, OWN(o, k));
            const float2 w2 = F2(ring_o2, OWN(o, k));
            const float h = rk_rate<CPT>(p, sm, s0, sp, k, w1.x, w1.y, w1.z, w1.w, w2.x);
            v[k] = HAS(k, FL_IN) ? pg.T_inlet_dev : (full ? w2.y + h : w2.y + 0.5f * h);
            F1(ring_acc, OWN(o, k)) += 2.0f * h;
          }
          ring_put<CPT>(dst, sl, v, allT, wT);
#pragma unroll
          for (int k = 0; k < CPT; k++) {
            if (HAS(k, FL_MIR)) F1(dst, sl + 4 * k + 4) = v[k];
            if (HAS(k, FL_ADB) && q == 0) F1(dst, below + 4 * k) = v[k];
          }
        }
      };
      mid_stage(r - 6, (unsigned)(j - 9) < (unsigned)(HR + 4), R4(6), R4(7), R4(5), R8(6),
                ring_T2, ring_T3, false);
      mid_stage(r - 8, (unsigned)(j - 12) < (unsigned)(HR + 2), R4(8), R4(9), R4(7), R8(8),
                ring_T3, ring_T4, true);
      // ---------------- S5: row r-10 (h4, new temperature) ----------------
      {
        const int q = r - 10;
        if ((unsigned)(j - 15) < (unsigned)HR) {
          float sm[CPT + 2], s0[CPT + 2], sp[CPT + 2];
          ring_row<CPT>(ring_T4, R4(11), sm);
          ring_row<CPT>(ring_T4, R4(10), s0);
          ring_row<CPT>(ring_T4, R4(9), sp);
          const int o = R8(10);
          float Tn[CPT];
#pragma unroll
          for (int k = 0; k < CPT; k++) {
            const float4 w1 = F4(ring_o1, OWN(o, k));
            const float2 w2 = F2(ring_o2, OWN(o, k));
            const float h4 = rk_rate<CPT>(p, sm, s0, sp, k, w1.x, w1.y, w1.z, w1.w, w2.x);
            Tn[k] = w2.y + (F1(ring_acc, OWN(o, k)) + h4) * (1.0f / 6.0f);
            if (outc[k]) {
              chk += Tn[k];
              dT_min = fminf(dT_min, Tn[k]);
            }
          }
          float *dst = Tout + (q * pg.pitch + c0);
          bool pair = false;
          if constexpr (CPT == 2) {
            pair = outc[0] && outc[1];
            if (pair) *reinterpret_cast<float2 *>(dst) = make_float2(Tn[0], Tn[1]);
          }
          if (!pair) {
#pragma unroll
            for (int k = 0; k < CPT; k++)
              if (outc[k]) dst[k] = Tn[k];
          }
        }
      }
    }

    // ---------------- S0 finish: row r ----------------
    if (s0_row) {
      const int sl = R4(0), sT = R8(0);
      if (r_solid) {
#pragma unroll
        for (int k = 0; k < CPT; k++) {
          F1(ring_T, sT + 4 * k) =
              r < 0 ? TWALL(k) : (HAS(k, FL_ADT) ? F1(ring_T, R8(1) + 4 * k) : TWALL_TOP(k));
          F1(ring_psi, sl + 4 * k) = 0.0f;
        }
      } else {
        float dpsi[CPT];
#pragma unroll
        for (int k = 0; k < CPT; k++) {
          if (xb) pull_fix(pg, cx[k], sc, fc[k], unk[k]);
          dpsi[k] = 0.0f;
          const float drho = sum9(fc[k]);
          drhoC[k] = drho;
          unsigned st_psi = 0u;
          if (MP) dpsi[k] = pseudopotential_dev(p, drho, Tc[k], st_psi);
          if (!HAS(k, FL_IN | FL_OUT)) {
            st |= st_psi;  // a ghost's populations include unfixed placeholders
            drho_min = fminf(drho_min, drho);
            drho_max = fmaxf(drho_max, drho);
            dT_min = fminf(dT_min, Tc[k]);
            chk += drho;
          }
        }
        ring_put<CPT>(ring_T, sT, Tc, allS0, wS0);
        ring_put<CPT>(ring_psi, sl, dpsi, allS0, wS0);
#pragma unroll
        for (int k = 0; k < CPT; k++) {
          if (HAS(k, FL_MIR)) {
            F1(ring_T, sT + 4 * k + 4) = Tc[k];
            F1(ring_psi, sl + 4 * k + 4) = dpsi[k];
          }
          if (HAS(k, FL_MIN0)) {
            F1(ring_T, sT + 4 * k - 4) = pg.T_inlet_dev;
            F1(ring_psi, sl + 4 * k - 4) = dpsi[k];
          }
          if (HAS(k, FL_ADB) && r == 0) F1(ring_T, R8(1) + 4 * k) = Tc[k];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < CPT; k++) {
#pragma unroll
      for (int i = 0; i < 9; i++) {
        fB[k][i] = fA[k][i];
        fA[k][i] = fc[k][i];
      }
      drhoB[k] = drhoA[k];
      drhoA[k] = drhoC[k];
    }
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
#undef OWN
#undef HAS
#undef TWALL
#undef TWALL_TOP
}

}  // namespace

}  // namespace lbm
