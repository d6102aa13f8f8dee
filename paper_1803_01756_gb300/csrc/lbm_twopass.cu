// Two-pass lattice update: the update of Section 2 as two launches.
//
//   pass A (k_stream_collide): pull-streaming with the boundary rules (Eq. 12), density
//     (Eq. 13), pseudopotential (Eqs. 10-11), forces (Eqs. 9, 14, 15), velocity (Eq. 13) and
//     the MRT collision with Li forcing (Eqs. 6-8); writes the post-collision populations
//     and, with the energy equation on, the density and velocity of every node.
//   pass B (k_energy_rk4): the four RK4 stages (Eqs. 17-18) of the energy equation
//     (Eq. 16) with density and velocity frozen at time t; writes T of time t + 1.
//
// Against the fused kernel (one launch, six stages per swept row), each pass keeps only
// the halo its own stencils need: pass A one row and one column of psi for the force of
// Eq. 9, pass B four rows and columns for the four stencil stages.  The fused kernel
// recomputes pass A's work on the energy equation's four halo rows as well (its
// collision stage must deliver u there), and its six stages in one loop body hold
// enough registers that three CTAs fit an SM; the two passes are lighter and run with
// more warps per SM (four and five CTAs).  The price is 24 B per node of extra traffic
// (rho, u written by A and read by B) and a second launch.  Measured on GB300, the path is
// faster than the fused kernel on small lattices (up to about 2^18 nodes, where the fused
// kernel's short row chunks spend most row steps filling its pipeline) and slower on large
// ones (4096 x 512: 75.0 against 65.8 us per update), where the two passes together execute
// more instructions per node than the fused kernel.
//
// Both passes sweep a strip of lattice columns (one column per thread) over a chunk of
// rows from bottom to top, like the fused kernel, with stages that trail each other in
// shared-memory row rings and one __syncthreads per row step.  Every node is computed by
// the same instructions whichever CTA owns it, so the results do not depend on the tiling.
#include <algorithm>

#include "lbm_fused_tile.cuh"

namespace lbm {

namespace {

constexpr int ANT = 128;       // threads of a pass-A CTA: one psi halo column on each side
constexpr int AW = ANT - 2;    // output columns of a pass-A CTA
constexpr int BNT = 128;       // threads of a pass-B CTA: four halo columns on each side
constexpr int BW = BNT - 8;    // output columns of a pass-B CTA
#ifndef LBM_TP_AMIN
#define LBM_TP_AMIN 4
#endif
#ifndef LBM_TP_BMIN
#define LBM_TP_BMIN 5
#endif
#ifndef LBM_TP_AND
#define LBM_TP_AND 4
#endif
constexpr int AMIN = LBM_TP_AMIN;  // resident pass-A CTAs per SM the registers are sized for
constexpr int BMIN = LBM_TP_BMIN;  // resident pass-B CTAs per SM the registers are sized for
constexpr int AND = LBM_TP_AND;    // pass A: rows whose loads are in flight ahead of the row in use
constexpr int ANS = AND + 2;       // pass A: staging slots (the extra one is read two steps
                                   // before its next fill, with a barrier between)
constexpr int BPF = 3;             // pass B: rows whose loads are in flight ahead of the row in
                                   // use (the three register sets Lc, L1, L2 below)

struct PassASmem {
  float4 pad_lo;         // neighbour reads of thread 0 below the first ring slot
  float psi[4][ANT];     // psi - psi_r of rows r-3 .. r
  float4 pad_hi;         // neighbour reads of the last thread above the last slot
  // Loads staged by cp.async, each thread in its own column slots: the nine pulled
  // populations (32-bit words holding them) and T of a row, and the row's Zou-He unknowns
  // (bits 0-8) and, with 16-bit storage, which half of each word holds the population
  // (bits 16-24).
  uint32_t pf[ANS][10][ANT];
  unsigned pfu[ANS][ANT];
};

// pulled populations of one row at the thread's column, with T and the Zou-He unknowns
struct PulledRow {
  float f[9];
  float T;
  float drho;
  unsigned unk;
};

// 4-byte asynchronous copy global -> shared (cp.async, completion by commit groups)
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// wait until at most N of this thread's most recent commit groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Staging of one stored population: the 4-byte word that holds element idx, and the value
// of population i from that word, converted exactly as the storage's load does.
template <class ST>
struct Staged;
template <>
struct Staged<StoreF32> {
  static __device__ __forceinline__ const void *src(const float *g, int idx, unsigned &hi) {
    hi = 0u;
    return g + idx;
  }
  static __device__ __forceinline__ float value(uint32_t w, unsigned, int) {
    return __uint_as_float(w);
  }
};
template <>
struct Staged<StoreF16> {
  // the word of an element pair: in bounds, the population arrays have an even length
  static __device__ __forceinline__ const void *src(const __half *g, int idx, unsigned &hi) {
    hi = (unsigned)idx & 1u;
    return g + (idx & ~1);
  }
  static __device__ __forceinline__ float value(uint32_t w, unsigned hi, int i) {
    return wlat(i) * __half2float(__ushort_as_half((unsigned short)(hi ? w >> 16 : w)));
  }
};
template <>
struct Staged<StoreBF16> {
  static __device__ __forceinline__ const void *src(const __nv_bfloat16 *g, int idx,
                                                    unsigned &hi) {
    hi = (unsigned)idx & 1u;
    return g + (idx & ~1);
  }
  static __device__ __forceinline__ float value(uint32_t w, unsigned hi, int i) {
    return wlat(i) * __bfloat162float(__ushort_as_bfloat16((unsigned short)(hi ? w >> 16 : w)));
  }
};

// Element indices of the populations that node (x, y) pulls (Eq. 12), with half-way
// bounce-back from the node's own opposite population on links from solid rows and the
// Zou-He unknowns (links from beyond an open end) flagged in `unknown`: the index form of
// pull_load.
__device__ __forceinline__ void pull_index(const DevParams &p, int x, int y, int (&idx)[9],
                                           unsigned &unknown) {
  const int c = y * p.pitch + x;
  unknown = 0u;
  idx[0] = c;
#pragma unroll
  for (int i = 1; i < 9; i++) {
    int xo, yo;
    const int k = classify(p, x, y, -ex(i), -ey(i), xo, yo);
    if (k == NB_FLUID) {
      idx[i] = i * (int)p.plane + yo * p.pitch + xo;
    } else {
      idx[i] = opp(i) * (int)p.plane + c;
      if (k == NB_INLET || k == NB_OUTLET) unknown |= 1u << i;
    }
  }
}

// Pass A on one tile: output columns [X0, X0 + W), rows [Y0, ye).  Thread t owns column
// X0 - 1 + t.  Per row step j (row r = Y0 - 1 + j):
//   - the loads of row r + AND are issued into the staging slots (cp.async), so that a
//     row's loads have AND row steps of arithmetic to land in;
//   - S0 finishes row r (staged AND steps ago): Zou-He fix-up, density, psi into the
//     ring;  __syncthreads;
//   - S1 collides row r - 1 with the psi of rows r - 2 .. r and stores it.
// One barrier per step orders S0's ring write before S1's reads of the same step; the
// next step's write goes to the slot of row r + 1, which no read of this step touches.
template <bool YW, bool XO, bool TH, bool MP, class ST>
__device__ __forceinline__ void sc_tile(const DevParams &p, const typename ST::T *__restrict__ gs,
                                        typename ST::T *__restrict__ gout,
                                        const float *__restrict__ Tin, float *__restrict__ rho_o,
                                        float *__restrict__ ux_o, float *__restrict__ uy_o,
                                        unsigned *status, const StepScalars &sc, int X0, int W,
                                        int Y0, int ye, PassASmem &S) {
  const int t = threadIdx.x;
  const int c = X0 - 1 + t;
  const int xe = min(X0 + W, p.nx);
  // ghosts beyond an open end load their clamped column and never use it: the boundary
  // column's thread writes their psi slot (zero gradient of psi at the open ends)
  const bool ghost = XO && (c < 0 || c >= p.nx);
  const int cx = XO ? min(max(c, 0), p.nx - 1) : modi(c, p.nx);
  const bool outc = c >= X0 && c < xe;
  const bool mir = XO && c == p.nx - 1 && t + 1 < ANT;
  const bool min0 = XO && c == 0 && t >= 1;
  // the CTA holds a column of an open end: only such CTAs have Zou-He unknowns to fix
  const bool xb = XO && (X0 - 1 <= 0 || X0 - 2 + ANT >= p.nx - 1);
  int poff[9];
  unsigned unk_edge = 0u;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    poff[i] = i * (int)p.plane - ey(i) * p.pitch - ex(i);
    if (!XO) {
      if (cx == 0 && ex(i) == 1) poff[i] += p.nx;
      if (cx == p.nx - 1 && ex(i) == -1) poff[i] -= p.nx;
    } else {
      if (cx == 0 && ex(i) == 1) unk_edge |= 1u << i;
      if (cx == p.nx - 1 && ex(i) == -1) unk_edge |= 1u << i;
    }
  }
  const unsigned uny = (unsigned)p.ny;
  const int HR = ye - Y0;
  const int J = HR + 2;  // S0 rows Y0 - 1 .. ye, S1 rows Y0 .. ye - 1

  unsigned st = 0;
  float chk = 0.0f, drho_min = 0.0f, drho_max = 0.0f, dT_min = 0.0f;

  // Issue the loads of the row of step jj (row Y0 - 1 + jj) into its staging slot: one
  // commit group per step, empty on a solid row or past the chunk, so that the group count
  // stays uniform.
  auto issue = [&](const int jj) {
    const int r = Y0 - 1 + jj;
    if (jj < J && !(YW && (unsigned)r >= uny)) {
      const int sl = jj % ANS;
      const int ry = YW ? r : modi(r, p.ny);
      const int own = ry * p.pitch + cx;
      int idx[9];
      unsigned unk;
      if ((unsigned)(ry - 1) < (unsigned)(p.ny - 2)) {  // 0 < ry < ny - 1
#pragma unroll
        for (int i = 0; i < 9; i++) idx[i] = own + poff[i];
        unk = unk_edge;
      } else {
        pull_index(p, cx, ry, idx, unk);
      }
      if (ghost) unk = 0u;
#pragma unroll
      for (int i = 0; i < 9; i++) {
        unsigned hi;
        cp_async4(&S.pf[sl][i][t], Staged<ST>::src(gs, idx[i], hi));
        unk |= hi << (16 + i);
      }
      cp_async4(&S.pf[sl][9][t], Tin + own);
      S.pfu[sl][t] = unk;
    }
    cp_async_commit();
  };

  float *const ring = &S.psi[0][0];
  // one step; Pc receives row r, Pa holds row r - 1
  auto step = [&](const int j, PulledRow &Pc, PulledRow &Pa) {
    const int r = Y0 - 1 + j;
    issue(j + AND);
    cp_async_wait<AND>();  // the group of row r has landed
    // ---------------- S0: row r ----------------
    {
      const int sl = 4 * ((j & 3) * ANT + t);
      if (YW && (unsigned)r >= uny) {
        F1(ring, sl) = 0.0f;
        Pc.drho = 0.0f;
        Pc.T = 0.0f;
      } else {
        const int ps = j % ANS;
        const unsigned u = S.pfu[ps][t];
#pragma unroll
        for (int i = 0; i < 9; i++) Pc.f[i] = Staged<ST>::value(S.pf[ps][i][t], (u >> (16 + i)) & 1u, i);
        Pc.T = __uint_as_float(S.pf[ps][9][t]);
        Pc.unk = u & 0x1ffu;
        if (xb) pull_fix(p, cx, sc, Pc.f, Pc.unk);
        const float drho = sum9(Pc.f);
        Pc.drho = drho;
        float dpsi = 0.0f;
        unsigned st_psi = 0u;
        if (MP) dpsi = pseudopotential_dev(p, drho, Pc.T, st_psi);
        if (!ghost) {
          st |= st_psi;  // a ghost's populations include unfixed placeholders
          drho_min = fminf(drho_min, drho);
          drho_max = fmaxf(drho_max, drho);
          dT_min = fminf(dT_min, Pc.T);
          chk += drho;
          F1(ring, sl) = dpsi;
        }
        if (mir) F1(ring, sl + 4) = dpsi;
        if (min0) F1(ring, sl - 4) = dpsi;
      }
    }
    __syncthreads();
    // ---------------- S1: row q = r - 1 ----------------
    const int q = r - 1;
    if (j >= 2) {  // q in [Y0, ye): always a fluid row
      const int sm = 4 * (((j - 2) & 3) * ANT + t), s0 = 4 * (((j - 1) & 3) * ANT + t),
                sp = 4 * ((j & 3) * ANT + t);
      Force F{0.0f, 0.0f, 0.0f};
      if (MP) {
        float dn[9];
        dn[0] = 0.0f;
        dn[1] = F1(ring, s0 + 4);
        dn[2] = F1(ring, sp);
        dn[3] = F1(ring, s0 - 4);
        dn[4] = F1(ring, sm);
        dn[5] = F1(ring, sp + 4);
        dn[6] = F1(ring, sp - 4);
        dn[7] = F1(ring, sm - 4);
        dn[8] = F1(ring, sm + 4);
        const float dpc = F1(ring, s0);
        const bool sdn = YW && q == 0;
        const bool sup = YW && q == p.ny - 1;
        if (!sdn && !sup) {
          // no wall neighbour: F = -G psi sum w dpsi e (Eq. 9), x and y pairwise
          const float2 d5786 = P2::sub(make_float2(dn[5], dn[8]), make_float2(dn[7], dn[6]));
          const float2 d1324 = P2::sub(make_float2(dn[1], dn[2]), make_float2(dn[3], dn[4]));
          const float d57 = d5786.x, d86 = d5786.y;
          const float2 Q = P2::fma(make_float2(0.25f, 0.25f), make_float2(d57 + d86, d57 - d86),
                                   d1324);
          const float gpsi = fmaf(p.G3, dpc, p.G3r);  // -G psi / 3
          const float2 Fq = P2::mul(make_float2(gpsi, gpsi), Q);
          F.Fx = Fq.x;
          F.Fy = Fq.y;
          F.fm2 = fmaf(Q.x, Q.x, Q.y * Q.y);
        } else {
          unsigned solid_mask = 0u;
          if (sup) solid_mask |= (1u << 2) | (1u << 5) | (1u << 6);
          if (sdn) solid_mask |= (1u << 4) | (1u << 7) | (1u << 8);
          float psiw = 0.0f;
          if (p.rho_w > 0.0f) {
            unsigned st_unused = 0;
            psiw = pseudopotential(p, p.rho_w, p.T_ref + Pa.T, st_unused);
          }
          F = interaction_force(p, dpc, dn, solid_mask, psiw);
        }
      }
      if (p.has_g) {
        const float rho_v = p.drho_ref_g + Pa.drho;  // rho - rho_v of Eq. 15
        F.Fx += rho_v * p.gx * sc.gcos;
        F.Fy += rho_v * p.gy * sc.gcos;
      }
      float gn[9], rr, ux, uy;
      collide(p, Pa.f, Pa.drho, F.Fx, F.Fy, F.fm2, gn, rr, ux, uy);
      if (outc) {
        chk += ux + uy;
        const int o = q * p.pitch + c;
#pragma unroll
        for (int i = 0; i < 9; i++) gout[i * p.plane + o] = ST::pack(gn[i], i);
        if (TH) {
          rho_o[o] = rr;
          ux_o[o] = ux;
          uy_o[o] = uy;
        }
      }
    }
  };

#pragma unroll
  for (int k = 0; k < AND; k++) issue(k);
  PulledRow P0, P1;
#pragma unroll 1
  for (int j = 0; j < J; j += 2) {
    // two steps per iteration, so that the two row buffers swap roles by renaming
    // (every thread takes the same branch: j is uniform)
    step(j, P0, P1);
    if (j + 1 < J) step(j + 1, P1, P0);
  }
  cp_async_wait<0>();  // no copy outlives the CTA
  if (!isfinite(chk)) st |= ST_NAN;
  if (!(p.rho_ref + drho_min > 0.0f)) st |= ST_RHO_NONPOS;
  if (!(p.eos_b * (p.rho_ref + drho_max) < 1.0f)) st |= ST_EOS_POLE;
  if (!(p.T_ref + dT_min > 0.0f)) st |= ST_T_NONPOS;
  set_status(status, st);
}

template <bool YW, bool XO, bool TH, bool MP, class ST>
__global__ void __launch_bounds__(ANT, AMIN)
    k_stream_collide(DevParams p, const typename ST::T *__restrict__ gs,
                     typename ST::T *__restrict__ gout, const float *__restrict__ Tin,
                     float *__restrict__ rho_o, float *__restrict__ ux_o,
                     float *__restrict__ uy_o, unsigned *status,
                     const StepScalars *__restrict__ sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassASmem &S = *reinterpret_cast<PassASmem *>(smem_raw);
  __shared__ StepScalars ssc;
  const int X0 = (int)(((long long)blockIdx.x * p.nx) / gridDim.x);
  const int X1 = (int)(((long long)(blockIdx.x + 1) * p.nx) / gridDim.x);
  const int Y0 = (int)(((long long)blockIdx.y * p.ny) / gridDim.y);
  const int ye = (int)(((long long)(blockIdx.y + 1) * p.ny) / gridDim.y);
  if (threadIdx.x == 0) ssc = *sc;
  __syncthreads();
  sc_tile<YW, XO, TH, MP, ST>(p, gs, gout, Tin, rho_o, ux_o, uy_o, status, ssc, X0, X1 - X0, Y0,
                              ye, S);
}

struct PassBSmem {
  float4 pad_lo;
  float2 u[4][BNT];      // velocity, rows r-3 .. r
  float T[4][BNT];       // T - T_ref, rows r-3 .. r
  float T2[4][BNT], T3[4][BNT], T4[4][BNT];  // RK stage fields
  // own-column values of rows r-8 .. r-2: (ux/3, uy/3, cl, E1), (E2, Tb) and the RK4 sum
  float4 o1[8][BNT];
  float2 o2[8][BNT];
  float oacc[8][BNT];
  float4 pad_hi;
};

// Pass B on one tile: output columns [X0, X0 + W), rows [Y0, ye).  Thread t owns column
// X0 - 4 + t.  Per row step j (row r = Y0 - 4 + j) the stages trail by two rows:
//   L  row r    : T, rho and u of time t (written by pass A) into the rings, with the
//                 energy-equation ghosts of walls and open ends
//   S2 row r-2  : div u, the node's coefficients of K(T) (Eq. 16) and h1 (Eq. 18)
//   S3 row r-4  : h2      S4 row r-6 : h3      S5 row r-8 : h4 and Eq. 17, T stored
// The stages are those of the fused kernel's energy part, with the same ghost rules:
// walls hold the wall temperature (isothermal columns) or copy the fluid node across the
// wall (adiabatic columns, periodic x only); the inlet ghost holds T_inlet and the inlet
// velocity (with a pressure inlet the velocity of column 0); the outlet ghost copies
// column nx - 1.  Ghosts of T and u load their clamped column, which is that copy; the
// outlet ghost's stage fields are written by the thread of column nx - 1.
template <bool YW, bool XO>
__device__ __forceinline__ void rk_tile(const DevParams &p, const float *__restrict__ Tin,
                                        float *__restrict__ Tout, const float *__restrict__ rho_in,
                                        const float *__restrict__ ux_in,
                                        const float *__restrict__ uy_in, unsigned *status,
                                        const StepScalars &sc, int X0, int W, int Y0, int ye,
                                        PassBSmem &S) {
  constexpr int NC = BNT;
  const int t = threadIdx.x;
  const int c = X0 - 4 + t;
  const int xe = min(X0 + W, p.nx);
  const bool gin = XO && c < 0, gout = XO && c >= p.nx;
  const int cx = XO ? min(max(c, 0), p.nx - 1) : modi(c, p.nx);
  const bool outc = c >= X0 && c < xe;
  const bool mir = XO && c == p.nx - 1 && t + 1 < NC;  // writes the outlet ghost's stage slots
  const bool adb = YW && !XO && p.adiabatic && wall_adiabatic(p, cx, false);
  const bool adt = YW && !XO && p.adiabatic && wall_adiabatic(p, cx, true);
  const bool wT = !gout;  // the outlet ghost's stage slots come from column nx - 1
  const unsigned uny = (unsigned)p.ny;
  const int HR = ye - Y0;
  const int J = HR + 12;
#define TWALL wall_T_dev(p, cx)
#define TWALL_TOP wall_T_top_dev(p, cx)

  unsigned st = 0;
  float chk = 0.0f, dT_min = 0.0f;
  float rho1 = 0.0f, rho2 = 0.0f;  // density of rows r - 1 and r - 2

  // L's loads run BPF row steps ahead of their use: T, rho and u of rows r .. r + BPF
  // (Lc is row r; La is the row just issued)
  struct Loaded {
    float T, rho, ux, uy;
  };
  auto load = [&](const int jj, Loaded &o) {
    const int r = Y0 - 4 + jj;
    o = Loaded{0.0f, 0.0f, 0.0f, 0.0f};
    if (jj < HR + 8 && !(YW && (unsigned)r >= uny)) {
      const int own = (YW ? r : modi(r, p.ny)) * p.pitch + cx;
      o.T = __ldg(Tin + own);
      o.rho = __ldg(rho_in + own);
      o.ux = __ldg(ux_in + own);
      o.uy = __ldg(uy_in + own);
    }
  };
  Loaded Lc, L1, L2;  // rows r, r + 1, r + 2 at the start of step j
  load(0, Lc);
  load(1, L1);
  load(2, L2);

  // float byte offset of ring row (r - k) at this thread's column (R4, R8 below), rotated
  // by one position per row step
  int q4[4], q8[8];
#pragma unroll
  for (int d = 0; d < 4; d++) q4[d] = 4 * (d * NC + t);
#pragma unroll
  for (int d = 0; d < 8; d++) q8[d] = 4 * (d * NC + t);

  auto row_step = [&](const int j) {
    const int r = Y0 - 4 + j;
#define R4(k) q4[(4 - ((k) & 3)) & 3]
#define R8(k) q8[(8 - ((k) & 7)) & 7]
    float2 *const ring_u = &S.u[0][0];
    float *const ring_T = &S.T[0][0];
    float *const ring_T2 = &S.T2[0][0];
    float *const ring_T3 = &S.T3[0][0];
    float *const ring_T4 = &S.T4[0][0];
    float4 *const ring_o1 = &S.o1[0][0];
    float2 *const ring_o2 = &S.o2[0][0];
    float *const ring_acc = &S.oacc[0][0];

    // ---------------- L loads: row r + BPF ----------------
    const bool l_row = j < HR + 8;
    const bool r_solid = YW && (unsigned)r >= uny;
    Loaded La;
    load(j + BPF, La);
    const float Tn = Lc.T, rn = Lc.rho, uxn = Lc.ux, uyn = Lc.uy;

    // ---------------- S2: row r-2 (div u, h1) ----------------
    {
      const int q = r - 2;
      if ((unsigned)(j - 3) < (unsigned)(HR + 6)) {
        const int sl = R4(2);
        if (YW && (unsigned)q >= uny) {
          F1(ring_T2, sl) = q < 0 ? TWALL : (adt ? F1(ring_T2, R4(3)) : TWALL_TOP);
        } else {
          float2 um[3], u0[3], up[3];
          ring_row2<1>(ring_u, R4(3), um);
          ring_row2<1>(ring_u, R4(2), u0);
          ring_row2<1>(ring_u, R4(1), up);
          float tm[3], t0[3], tp[3];
          ring_row<1>(ring_T, R4(3), tm);
          ring_row<1>(ring_T, R4(2), t0);
          ring_row<1>(ring_T, R4(1), tp);
          const float2 a1 = u0[2], a3 = u0[0];
          const float2 a2 = up[1], a4 = um[1];
          const float2 a5 = up[2], a6 = up[0];
          const float2 a7 = um[0], a8 = um[2];
          // 3 div u = 9 sum w_i u(x+e_i).e_i; the 1/3 is folded into the coefficients
          const float2 d57 = P2::sub(a5, a7), d86 = P2::sub(a8, a6);
          const float divu3 = ((a1.x - a3.x) + (a2.y - a4.y)) +
                              0.25f * ((d57.x + d86.x) + (d57.y - d86.y));
          // energy coefficients of the node (see rk_rate): E1 / (3 div u), E2 / (3 div u), cl
          const float rho = rho2;
          const float br = p.eos_b * rho;
          const float z = __fdividef(p.akap1_cv3 * rho, fmaf(br, 2.0f - br, 1.0f));
          const float cfx = __fdividef(p.RTc_cv3, 1.0f - br) - p.kappa_r * z;
          const float cl = p.lam23_cv * __fdividef(1.0f, rho);
          const float2 E = P2::mul(make_float2(cfx, z), make_float2(divu3, divu3));
          const float2 us = P2::mul(u0[1], make_float2(1.0f / 3.0f, 1.0f / 3.0f));
          const float Tb = t0[1];
          const float h1 = rk_rate<1>(p, tm, t0, tp, 0, us.x, us.y, cl, E.x, E.y);
          const float v = gin ? p.T_inlet_dev : Tb + 0.5f * h1;
          const int o = R8(2);
          F4(ring_o1, o) = make_float4(us.x, us.y, cl, E.x);
          F2(ring_o2, o) = make_float2(E.y, Tb);
          F1(ring_acc, o) = h1;
          if (wT) F1(ring_T2, sl) = v;
          if (mir) F1(ring_T2, sl + 4) = v;
          if (adb && q == 0) F1(ring_T2, R4(3)) = v;
        }
      }
    }
    // ---------------- S3: row r-4 (h2) and S4: row r-6 (h3) ----------------
    // T2 -> T3 with the half step, T3 -> T4 with the full step
    auto mid_stage = [&](const int q, const bool active, const int sl, const int below,
                         const int above, const int o, float *const src, float *const dst,
                         const bool full) {
      if (!active) return;
      if (YW && (unsigned)q >= uny) {
        F1(dst, sl) = q < 0 ? TWALL : (adt ? F1(dst, below) : TWALL_TOP);
      } else {
        float sm[3], s0[3], sp[3];
        ring_row<1>(src, below, sm);
        ring_row<1>(src, sl, s0);
        ring_row<1>(src, above, sp);
        const float4 w1 = F4(ring_o1, o);
        const float2 w2 = F2(ring_o2, o);
        const float h = rk_rate<1>(p, sm, s0, sp, 0, w1.x, w1.y, w1.z, w1.w, w2.x);
        const float v = gin ? p.T_inlet_dev : (full ? w2.y + h : w2.y + 0.5f * h);
        F1(ring_acc, o) += 2.0f * h;
        if (wT) F1(dst, sl) = v;
        if (mir) F1(dst, sl + 4) = v;
        if (adb && q == 0) F1(dst, below) = v;
      }
    };
    mid_stage(r - 4, (unsigned)(j - 6) < (unsigned)(HR + 4), R4(4), R4(5), R4(3), R8(4), ring_T2,
              ring_T3, false);
    mid_stage(r - 6, (unsigned)(j - 9) < (unsigned)(HR + 2), R4(6), R4(7), R4(5), R8(6), ring_T3,
              ring_T4, true);
    // ---------------- S5: row r-8 (h4, new temperature) ----------------
    {
      const int q = r - 8;
      if ((unsigned)(j - 12) < (unsigned)HR) {
        float sm[3], s0[3], sp[3];
        ring_row<1>(ring_T4, R4(9), sm);
        ring_row<1>(ring_T4, R4(8), s0);
        ring_row<1>(ring_T4, R4(7), sp);
        const int o = R8(8);
        const float4 w1 = F4(ring_o1, o);
        const float2 w2 = F2(ring_o2, o);
        const float h4 = rk_rate<1>(p, sm, s0, sp, 0, w1.x, w1.y, w1.z, w1.w, w2.x);
        const float Tnew = w2.y + (F1(ring_acc, o) + h4) * (1.0f / 6.0f);
        if (outc) {
          chk += Tnew;
          dT_min = fminf(dT_min, Tnew);
          Tout[q * p.pitch + c] = Tnew;
        }
      }
    }

    // ---------------- L finish: row r ----------------
    if (l_row) {
      const int sl = R4(0);
      if (r_solid) {
        F1(ring_T, sl) = r < 0 ? TWALL : (adt ? F1(ring_T, R4(1)) : TWALL_TOP);
        F2(ring_u, sl) = make_float2(0.0f, 0.0f);
      } else {
        // the velocity inlet's ghost holds the inlet velocity and T_inlet; every other
        // ghost holds its clamped column (a copy of the boundary column)
        F1(ring_T, sl) = gin ? p.T_inlet_dev : Tn;
        F2(ring_u, sl) = gin && !p.p_inlet ? make_float2(sc.u_in, 0.0f) : make_float2(uxn, uyn);
        if (adb && r == 0) F1(ring_T, R4(1)) = Tn;
      }
    }
    rho2 = rho1;
    rho1 = rn;
    Lc = L1;
    L1 = L2;
    L2 = La;
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
#pragma unroll 1
  for (int j = 0; j < J; j += 2) {
    row_step(j);
    __syncthreads();
    row_step(j + 1);  // a step past J runs no stage: every stage range ends by J
    __syncthreads();
  }
  if (!isfinite(chk)) st |= ST_NAN;
  if (!(p.T_ref + dT_min > 0.0f)) st |= ST_T_NONPOS;
  set_status(status, st);
#undef TWALL
#undef TWALL_TOP
}

template <bool YW, bool XO>
__global__ void __launch_bounds__(BNT, BMIN)
    k_energy_rk4(DevParams p, const float *__restrict__ Tin, float *__restrict__ Tout,
                 const float *__restrict__ rho_in, const float *__restrict__ ux_in,
                 const float *__restrict__ uy_in, unsigned *status,
                 const StepScalars *__restrict__ sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassBSmem &S = *reinterpret_cast<PassBSmem *>(smem_raw);
  __shared__ StepScalars ssc;
  const int X0 = (int)(((long long)blockIdx.x * p.nx) / gridDim.x);
  const int X1 = (int)(((long long)(blockIdx.x + 1) * p.nx) / gridDim.x);
  const int Y0 = (int)(((long long)blockIdx.y * p.ny) / gridDim.y);
  const int ye = (int)(((long long)(blockIdx.y + 1) * p.ny) / gridDim.y);
  if (threadIdx.x == 0) ssc = *sc;
  __syncthreads();
  rk_tile<YW, XO>(p, Tin, Tout, rho_in, ux_in, uy_in, status, ssc, X0, X1 - X0, Y0, ye, S);
}

template <class ST>
using PassAFn = void (*)(DevParams, const typename ST::T *, typename ST::T *, const float *,
                         float *, float *, float *, unsigned *, const StepScalars *);
using PassBFn = void (*)(DevParams, const float *, float *, const float *, const float *,
                         const float *, unsigned *, const StepScalars *);

template <class ST>
PassAFn<ST> pass_a_variant(const DevParams &p) {
#define KA(a, b, c, d) k_stream_collide<a, b, c, d, ST>
  static const PassAFn<ST> table[16] = {
      KA(false, false, false, false), KA(false, false, false, true), KA(false, false, true, false),
      KA(false, false, true, true),   KA(false, true, false, false), KA(false, true, false, true),
      KA(false, true, true, false),   KA(false, true, true, true),   KA(true, false, false, false),
      KA(true, false, false, true),   KA(true, false, true, false),  KA(true, false, true, true),
      KA(true, true, false, false),   KA(true, true, false, true),   KA(true, true, true, false),
      KA(true, true, true, true)};
#undef KA
  const int k = (p.y_walls ? 8 : 0) | (p.x_open ? 4 : 0) | (p.thermal ? 2 : 0) |
                (p.multiphase ? 1 : 0);
  return table[k];
}

PassBFn pass_b_variant(const DevParams &p) {
  static const PassBFn table[4] = {k_energy_rk4<false, false>, k_energy_rk4<false, true>,
                                   k_energy_rk4<true, false>, k_energy_rk4<true, true>};
  return table[(p.y_walls ? 2 : 0) | (p.x_open ? 1 : 0)];
}

template <class ST>
cudaError_t occupancy_a(const DevParams &p, int *occ) {
  const PassAFn<ST> fn = pass_a_variant<ST>(p);
  const int smem = (int)sizeof(PassASmem);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, ANT, smem);
}

cudaError_t occupancy_b(const DevParams &p, int *occ) {
  const PassBFn fn = pass_b_variant(p);
  const int smem = (int)sizeof(PassBSmem);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, BNT, smem);
}

// Row-chunk height of one pass: with `strips` strips of the lattice and `slots` resident
// CTAs, the height whose launch takes the fewest row steps per SM slot, (H + extra) x
// waves, where extra is the pass's fill of halo and trailing stages (ties keep the
// taller chunk).
int chunk_height(int ny, int strips, long long slots, int extra) {
  int best = ny;
  long long best_cost = -1;
  const long long max_chunks = std::min<long long>(ny, std::max<long long>(1, 4 * slots / strips));
  for (long long ch = 1; ch <= max_chunks; ch++) {
    const int h = (int)((ny + ch - 1) / ch);
    const long long tiles = (long long)strips * ((ny + h - 1) / h);
    const long long waves = (tiles + slots - 1) / slots;
    const long long cost = (h + extra) * waves;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = h;
    }
  }
  return best;
}

}  // namespace

int twopass_width_a() { return AW; }
int twopass_width_b() { return BW; }

TwoPassTiling twopass_tiling(const DevParams &p, int storage, int device) {
  TwoPassTiling tl{0, 0};
  int sms = 0, occa = 0, occb = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return tl;
  cudaError_t e = storage == STORAGE_BF16  ? occupancy_a<StoreBF16>(p, &occa)
                  : storage == STORAGE_F16 ? occupancy_a<StoreF16>(p, &occa)
                                           : occupancy_a<StoreF32>(p, &occa);
  if (e != cudaSuccess || occa < 1) return tl;
  if (occupancy_b(p, &occb) != cudaSuccess || occb < 1) return tl;
  tl.Ha = chunk_height(p.ny, (p.nx + AW - 1) / AW, (long long)sms * occa, 2);
  tl.Hb = chunk_height(p.ny, (p.nx + BW - 1) / BW, (long long)sms * occb, 12);
  return tl;
}

cudaError_t launch_stream_collide(const DevParams &p, int storage, const void *gs, void *gout,
                                  const float *Tin, float *rho, float *ux, float *uy,
                                  unsigned *status, const StepScalars *sc, int Ha,
                                  cudaStream_t s) {
  if (Ha < 1) return cudaErrorInvalidValue;
  const dim3 grid((p.nx + AW - 1) / AW, (p.ny + Ha - 1) / Ha);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  switch (storage) {
    case STORAGE_BF16:
      pass_a_variant<StoreBF16>(p)<<<grid, ANT, sizeof(PassASmem), s>>>(
          p, static_cast<const __nv_bfloat16 *>(gs), static_cast<__nv_bfloat16 *>(gout), Tin,
          rho, ux, uy, status, sc);
      break;
    case STORAGE_F16:
      pass_a_variant<StoreF16>(p)<<<grid, ANT, sizeof(PassASmem), s>>>(p, static_cast<const __half *>(gs),
                                                       static_cast<__half *>(gout), Tin, rho,
                                                       ux, uy, status, sc);
      break;
    default:
      pass_a_variant<StoreF32>(p)<<<grid, ANT, sizeof(PassASmem), s>>>(p, static_cast<const float *>(gs),
                                                       static_cast<float *>(gout), Tin, rho, ux,
                                                       uy, status, sc);
  }
  return cudaGetLastError();
}

cudaError_t launch_energy_rk4(const DevParams &p, const float *Tin, float *Tout, const float *rho,
                              const float *ux, const float *uy, unsigned *status,
                              const StepScalars *sc, int Hb, cudaStream_t s) {
  if (Hb < 1) return cudaErrorInvalidValue;
  const dim3 grid((p.nx + BW - 1) / BW, (p.ny + Hb - 1) / Hb);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  pass_b_variant(p)<<<grid, BNT, sizeof(PassBSmem), s>>>(p, Tin, Tout, rho, ux, uy, status, sc);
  return cudaGetLastError();
}

}  // namespace lbm
