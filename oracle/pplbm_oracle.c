/*
 * Plain FP64 CPU oracle of the D2Q9 pseudopotential MRT lattice Boltzmann
 * update with the finite-difference energy equation (Zhao, Xu & Zhang,
 * arXiv:1803.01756, Section 2).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and
 * the CPU-baseline leg of the benchmark, never by the product path.  It shares
 * no code with the CUDA path.  Written to be read against the paper: one
 * whole-grid loop nest per stage, no fusion, no blocking.
 *
 * Readings taken where the paper is silent or garbled (each also marked at the
 * code that takes it):
 *  - Eq. 5 is read as tau_nu = tau_g + clamp((rho-rho_g)/(rho_l-rho_g),0,1)(tau_l-tau_g).
 *  - Eq. 6 m^eq is read as M f^eq of the second-order equilibrium (quadratic
 *    moments carry rho |u|^2, i.e. |j|^2/rho).
 *  - Eq. 8: the theta term of the third entry (epsilon) takes a minus sign, and
 *    the last entry is u_x F_y + u_y F_x (the symmetric form that M S of Guo's
 *    forcing gives).
 *  - Eq. 10: a negative square-root argument gives psi = 0 and a status bit.
 *  - Eq. 14: s = 1 on solid sites (the adhesion sums over wall neighbours); the
 *    fluid-fluid sum of Eq. 9 runs over fluid neighbours only; psi(rho_w) is the
 *    local psi when rho_w <= 0.
 *  - Eq. 17: classical weights (h1 + 2 h2 + 2 h3 + h4)/6, the weights of the
 *    fourth-order scheme whose stages Eq. 18 defines.
 *  - Open ends: zero-gradient psi; Zou-He velocity inlet and density outlet
 *    applied, without force, to the populations that enter from outside the x
 *    range through fluid rows; wall-row links are bounced back first.
 *  - Energy-equation ghosts: wall rows hold the wall temperature (linear in x
 *    between the two given end values, the top wall optionally with its own
 *    values) and zero velocity; on adiabatic wall columns (Section 3.2: outside a
 *    wall's isothermal window) the ghost copies the fluid node across the wall;
 *    the inlet ghost holds T_inlet and the inlet velocity; the outlet ghost copies
 *    the last column.
 *  - Pressure inlet (Section 3.3): the inlet pressure p0 (1 + a sin(2 pi t/P)) is
 *    imposed through the density whose Peng-Robinson pressure at T_inlet equals it,
 *    taken on the vapour branch (below the first maximum of P(rho)); p0 is the
 *    pressure of the outlet density at T_inlet.  Its energy-equation ghost copies the
 *    velocity of the inlet column.
 *  - Time: the populations f^t carry the inlet velocity u_amp sin(2 pi t/P) and
 *    the body force of step t is multiplied by cos(g_omega t).
 */
#include "pplbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 discrete velocities, Eq. 2 */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* D2Q9 lattice weights (equilibrium and the isotropic FD stencils) */
static const double WLAT[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                               1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* interaction weights of Eq. 9: w(1) = 1/3, w(2) = 1/12 */
static const double WPSI[9] = {0.0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 1.0 / 3,
                               1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12};

/* transform matrix of Eq. 6 (rows: rho, e, epsilon, jx, qx, jy, qy, pxx, pxy) */
static const int MM[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

static const double PI = 3.14159265358979323846;

struct orc_lattice {
  int nx, ny;
  orc_params p;
  double Tc;
  long t;
  unsigned status;
  double *f;  /* [9][ny][nx] pre-collision populations at time t */
  double *T;  /* [ny][nx] absolute temperature at time t */
  /* whole-grid stage arrays */
  double *rho, *psi, *Fx, *Fy, *Fm2psi2, *ux, *uy;
  double *fs, *fn;           /* post-collision, next populations */
  double *Tk, *h, *acc, *Tn; /* Runge-Kutta stage field, stage slope, sum, result */
  double *divu;
};

/* ------------------------------------------------------------------ */
/* Peng-Robinson equation of state, Eq. 11                             */
/* ------------------------------------------------------------------ */

/* a = 0.45724 R^2 Tc^2 / Pc and b = 0.0778 R Tc / Pc give Tc = 0.0778 a / (0.45724 b R) */
double orc_critical_temperature(const orc_params *p) {
  return 0.0778 * p->eos_a / (0.45724 * p->eos_b * p->eos_R);
}

static double pr_kappa(double omega) {
  return 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
}

/* varphi(T) = [1 + kappa (1 - sqrt(T/Tc))]^2 */
static double pr_varphi(const orc_params *p, double T) {
  double Tc = orc_critical_temperature(p);
  double r = 1.0 + pr_kappa(p->eos_omega) * (1.0 - sqrt(T / Tc));
  return r * r;
}

/* d varphi / dT = -kappa [1 + kappa (1 - sqrt(T/Tc))] / sqrt(T Tc) */
static double pr_dvarphi_dT(const orc_params *p, double T) {
  double Tc = orc_critical_temperature(p);
  double k = pr_kappa(p->eos_omega);
  double r = 1.0 + k * (1.0 - sqrt(T / Tc));
  return -k * r / sqrt(T * Tc);
}

double orc_eos_pressure(const orc_params *p, double rho, double T) {
  double a = p->eos_a, b = p->eos_b, R = p->eos_R;
  return rho * R * T / (1.0 - b * rho) -
         a * pr_varphi(p, T) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

/* (dP/dT) at constant rho, the coefficient in the last term of Eq. 16 */
double orc_eos_dpdt(const orc_params *p, double rho, double T) {
  double a = p->eos_a, b = p->eos_b, R = p->eos_R;
  return rho * R / (1.0 - b * rho) -
         a * pr_dvarphi_dT(p, T) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

/* Eq. 10 with c = 1, cs^2 = 1/3 */
double orc_psi(const orc_params *p, double rho, double T, int *neg) {
  double arg = 2.0 * (orc_eos_pressure(p, rho, T) - rho / 3.0) / p->G;
  if (neg) *neg = 0;
  if (!(arg >= 0.0)) {
    if (neg) *neg = 1;
    return 0.0;
  }
  return sqrt(arg);
}

/* ------------------------------------------------------------------ */
/* Moment space, Eqs. 6-8                                              */
/* ------------------------------------------------------------------ */

void orc_moment_matrix(int M[81]) {
  for (int r = 0; r < 9; r++)
    for (int c = 0; c < 9; c++) M[r * 9 + c] = MM[r][c];
}

void orc_feq(double rho, double ux, double uy, double feq[9]) {
  double uu = ux * ux + uy * uy;
  for (int i = 0; i < 9; i++) {
    double eu = EX[i] * ux + EY[i] * uy;
    feq[i] = WLAT[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
  }
}

/* Eq. 6 m^eq with j = rho u; quadratic entries read as |j|^2 / rho */
void orc_meq(double rho, double ux, double uy, double meq[9]) {
  double jx = rho * ux, jy = rho * uy;
  double jj = (jx * jx + jy * jy) / rho;
  meq[0] = rho;
  meq[1] = -2.0 * rho + 3.0 * jj;
  meq[2] = rho - 3.0 * jj;
  meq[3] = jx;
  meq[4] = -jx;
  meq[5] = jy;
  meq[6] = -jy;
  meq[7] = (jx * jx - jy * jy) / rho;
  meq[8] = jx * jy / rho;
}

/* Eq. 8, Li's improved forcing in moment space; Fm2_over_psi2 = |F_m|^2 / psi^2 */
void orc_forcing_moments(double ux, double uy, double Fx, double Fy, double Fm2_over_psi2,
                         double theta, double s_e, double s_zeta, double S[9]) {
  double tau_e = 1.0 / s_e, tau_z = 1.0 / s_zeta;
  double uF = ux * Fx + uy * Fy;
  S[0] = 0.0;
  S[1] = 6.0 * uF + 12.0 * theta * Fm2_over_psi2 / (tau_e - 0.5);
  S[2] = -6.0 * uF - 12.0 * theta * Fm2_over_psi2 / (tau_z - 0.5); /* sign: see header */
  S[3] = Fx;
  S[4] = -Fx;
  S[5] = Fy;
  S[6] = -Fy;
  S[7] = 2.0 * (ux * Fx - uy * Fy);
  S[8] = ux * Fy + uy * Fx; /* symmetric form: see header */
}

/* Eq. 5 read with the denominator (rho_l - rho_g), fraction clamped to [0, 1] */
static double tau_nu(const orc_params *p, double rho) {
  double frac = (p->rho_l != p->rho_g) ? (rho - p->rho_g) / (p->rho_l - p->rho_g) : 0.0;
  if (frac < 0.0) frac = 0.0;
  if (frac > 1.0) frac = 1.0;
  return p->tau_g + frac * (p->tau_l - p->tau_g);
}

/* Eq. 7 on one node followed by f* = M^-1 m* (M^-1 = M^T D^-1, D = diag(M M^T)) */
void orc_collide_node(const orc_params *p, const double f[9], double Fx, double Fy,
                      double Fm2_over_psi2, double fstar[9]) {
  double m[9], meq[9], S[9], ms[9], Lam[9], D[9];
  double rho = 0.0, jx = 0.0, jy = 0.0;
  for (int r = 0; r < 9; r++) {
    m[r] = 0.0;
    for (int c = 0; c < 9; c++) m[r] += MM[r][c] * f[c];
  }
  for (int i = 0; i < 9; i++) {
    rho += f[i];
    jx += EX[i] * f[i];
    jy += EY[i] * f[i];
  }
  /* Eq. 13 */
  double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
  orc_meq(rho, ux, uy, meq);
  orc_forcing_moments(ux, uy, Fx, Fy, Fm2_over_psi2, p->theta, p->s_e, p->s_zeta, S);
  /* Eq. 3; s0, s3, s5 act on conserved or exactly forced moments and are set to 1 */
  double snu = 1.0 / tau_nu(p, rho);
  Lam[0] = 1.0; Lam[1] = p->s_e; Lam[2] = p->s_zeta; Lam[3] = 1.0; Lam[4] = p->s_q;
  Lam[5] = 1.0; Lam[6] = p->s_q; Lam[7] = snu; Lam[8] = snu;
  for (int r = 0; r < 9; r++)
    ms[r] = m[r] - Lam[r] * (m[r] - meq[r]) + (1.0 - 0.5 * Lam[r]) * S[r];
  for (int r = 0; r < 9; r++) {
    D[r] = 0.0;
    for (int c = 0; c < 9; c++) D[r] += (double)(MM[r][c] * MM[r][c]);
  }
  for (int c = 0; c < 9; c++) {
    fstar[c] = 0.0;
    for (int r = 0; r < 9; r++) fstar[c] += MM[r][c] * ms[r] / D[r];
  }
}

/* ------------------------------------------------------------------ */
/* Finite-difference stencils of Eq. 16 (isotropic nine-point forms)   */
/*   grad phi = 3 sum_i w_i phi(x+e_i) e_i                             */
/*   lap  phi = 6 sum_i w_i (phi(x+e_i) - phi(x))                      */
/* ------------------------------------------------------------------ */

static int wrap(int v, int n) { return ((v % n) + n) % n; }

void orc_grad_periodic(int nx, int ny, const double *phi, double *gx, double *gy) {
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      double sx = 0.0, sy = 0.0;
      for (int i = 1; i < 9; i++) {
        double v = phi[wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx)];
        sx += WLAT[i] * v * EX[i];
        sy += WLAT[i] * v * EY[i];
      }
      gx[y * nx + x] = 3.0 * sx;
      gy[y * nx + x] = 3.0 * sy;
    }
}

void orc_lap_periodic(int nx, int ny, const double *phi, double *lap) {
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      double s = 0.0, c = phi[y * nx + x];
      for (int i = 1; i < 9; i++)
        s += WLAT[i] * (phi[wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx)] - c);
      lap[y * nx + x] = 6.0 * s;
    }
}

/* ------------------------------------------------------------------ */
/* Lattice geometry                                                    */
/* ------------------------------------------------------------------ */

enum { NB_FLUID = 0, NB_SOLID = 1, NB_INLET = 2, NB_OUTLET = 3 };

/* Classify site (x+dx, y+dy) seen from a fluid node.  Wall rows are tested
   first.  For fluid, inlet-ghost and outlet-ghost sites (*xo, *yo) is the
   fluid node that supplies a copied value (wrapped, or clamped at open ends);
   for a wall site, *xo is its column (the periodic image when x is periodic,
   clamped at open ends) and *yo the fluid row next to the wall. */
static int classify(const orc_lattice *L, int x, int y, int dx, int dy, int *xo, int *yo) {
  int xs = x + dx, ys = y + dy;
  if (L->p.y_bc == ORC_Y_WALLS) {
    if (ys < 0 || ys >= L->ny) {
      if (L->p.x_bc == ORC_X_PERIODIC)
        *xo = wrap(xs, L->nx);
      else
        *xo = xs < 0 ? 0 : (xs >= L->nx ? L->nx - 1 : xs);
      *yo = ys < 0 ? 0 : L->ny - 1;
      return NB_SOLID;
    }
  } else {
    ys = wrap(ys, L->ny);
  }
  *yo = ys;
  if (L->p.x_bc == ORC_X_PERIODIC) {
    *xo = wrap(xs, L->nx);
    return NB_FLUID;
  }
  if (xs < 0) { *xo = 0; return NB_INLET; }
  if (xs >= L->nx) { *xo = L->nx - 1; return NB_OUTLET; }
  *xo = xs;
  return NB_FLUID;
}

/* first density where dP/drho = 0 at temperature T (the vapour spinodal), or the
   pole region when the isotherm is monotone */
static double vapour_branch_end(const orc_params *p, double T) {
  double h = 1e-7, rmax = 0.999 / p->eos_b, step = 1e-3;
  double prev = 1e-6;
  for (double r = 1e-6 + step; r < rmax; r += step) {
    double d = orc_eos_pressure(p, r + h, T) - orc_eos_pressure(p, r - h, T);
    if (d <= 0.0) {
      double lo = prev, hi = r;
      for (int it = 0; it < 100; it++) {
        double mid = 0.5 * (lo + hi);
        double dm = orc_eos_pressure(p, mid + h, T) - orc_eos_pressure(p, mid - h, T);
        if (dm > 0.0) lo = mid; else hi = mid;
      }
      return lo;
    }
    prev = r;
  }
  return rmax;
}

double orc_inlet_density(const orc_params *p, long t) {
  double T = orc_critical_temperature(p) * p->T_inlet;
  double p0 = orc_eos_pressure(p, p->rho_out, T);
  double s = p->u_period == 0.0 ? 1.0 : sin(2.0 * PI * (double)t / p->u_period);
  double target = p0 * (1.0 + p->p_amp_frac * s);
  double lo = 0.0, hi = vapour_branch_end(p, T);
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    if (orc_eos_pressure(p, mid, T) < target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

static double inlet_velocity(const orc_lattice *L, long t) {
  if (L->p.u_period == 0.0) return L->p.u_amp;
  return L->p.u_amp * sin(2.0 * PI * (double)t / L->p.u_period);
}

/* wall temperature, linear between the end values along x (units of Tc -> absolute);
   the top wall has its own profile when one of its end values is set */
static double wall_temperature(const orc_lattice *L, int x, int top) {
  double s = L->nx > 1 ? (double)x / (double)(L->nx - 1) : 0.0;
  double a = L->p.T_wall_left, b = L->p.T_wall_right;
  if (top && (L->p.T_top_left != 0.0 || L->p.T_top_right != 0.0)) {
    a = L->p.T_top_left;
    b = L->p.T_top_right;
  }
  return L->Tc * (a + s * (b - a));
}

/* 1 when column x of the top (or bottom) wall is adiabatic: outside the wall's
   isothermal window [x0, x1); an empty window (x1 <= x0) makes the whole wall isothermal */
static int wall_adiabatic(const orc_lattice *L, int x, int top) {
  int x0 = top ? L->p.top_iso_x0 : L->p.bot_iso_x0;
  int x1 = top ? L->p.top_iso_x1 : L->p.bot_iso_x1;
  if (x1 <= x0) return 0;
  return x < x0 || x >= x1;
}

/* ------------------------------------------------------------------ */
/* Streaming boundaries                                                */
/* ------------------------------------------------------------------ */

/* Zou-He on the open columns of population set g (whole grid, time t).
   unknown[i] marks the populations that entered from outside the x range
   through fluid rows; those are the only ones replaced. */
static void zou_he_column(orc_lattice *L, double *g, int x, long t) {
  int N = L->nx * L->ny;
  for (int y = 0; y < L->ny; y++) {
    int id = y * L->nx + x;
    double f[9];
    int unknown[9] = {0};
    for (int i = 0; i < 9; i++) f[i] = g[i * N + id];
    for (int i = 1; i < 9; i++) {
      int xo, yo;
      int k = classify(L, x, y, -EX[i], -EY[i], &xo, &yo);
      if ((k == NB_INLET && x == 0) || (k == NB_OUTLET && x == L->nx - 1)) unknown[i] = 1;
    }
    if (x == 0) {
      double U, rb;
      if (L->p.x_bc == ORC_X_PRESSURE_INLET) {
        /* density given: velocity from the known populations */
        rb = orc_inlet_density(&L->p, t);
        U = 1.0 - (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / rb;
      } else {
        U = inlet_velocity(L, t);
        rb = (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / (1.0 - U);
      }
      if (unknown[1]) f[1] = f[3] + (2.0 / 3.0) * rb * U;
      if (unknown[5]) f[5] = f[7] - 0.5 * (f[2] - f[4]) + rb * U / 6.0;
      if (unknown[8]) f[8] = f[6] + 0.5 * (f[2] - f[4]) + rb * U / 6.0;
    } else {
      double ro = L->p.rho_out;
      double U = -1.0 + (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) / ro;
      if (unknown[3]) f[3] = f[1] - (2.0 / 3.0) * ro * U;
      if (unknown[7]) f[7] = f[5] + 0.5 * (f[2] - f[4]) - ro * U / 6.0;
      if (unknown[6]) f[6] = f[8] - 0.5 * (f[2] - f[4]) - ro * U / 6.0;
    }
    for (int i = 0; i < 9; i++) g[i * N + id] = f[i];
  }
}

static void apply_open_boundaries(orc_lattice *L, double *g, long t) {
  if (L->p.x_bc == ORC_X_PERIODIC) return;
  zou_he_column(L, g, 0, t);
  zou_he_column(L, g, L->nx - 1, t);
}

/* Eq. 12 written per destination: f_i(x) = f*_i(x - e_i); sources in a wall row
   give the half-way bounce-back f_i(x) = f*_opp(i)(x).  Sources beyond an open
   end are left for the Zou-He rule (filled with the bounce-back value first). */
static void stream(orc_lattice *L) {
  int N = L->nx * L->ny;
  for (int i = 0; i < 9; i++)
    for (int y = 0; y < L->ny; y++)
      for (int x = 0; x < L->nx; x++) {
        int xo, yo, id = y * L->nx + x;
        int k = classify(L, x, y, -EX[i], -EY[i], &xo, &yo);
        if (i == 0)
          L->fn[id] = L->fs[id];
        else if (k == NB_FLUID)
          L->fn[i * N + id] = L->fs[i * N + yo * L->nx + xo];
        else
          L->fn[i * N + id] = L->fs[OPP[i] * N + id];
      }
  apply_open_boundaries(L, L->fn, L->t + 1);
}

/* ------------------------------------------------------------------ */
/* Macroscopic stages at time t: Eq. 13, Eq. 10-11, Eq. 9, 14, 15      */
/* ------------------------------------------------------------------ */

static void check(orc_lattice *L, double v, unsigned bit) {
  if (v != v) L->status |= ORC_ST_NAN;
  (void)bit;
}

static void macroscopic(orc_lattice *L) {
  int nx = L->nx, ny = L->ny, N = nx * ny;
  const orc_params *p = &L->p;
  /* density, Eq. 13 */
  for (int id = 0; id < N; id++) {
    double s = 0.0;
    for (int i = 0; i < 9; i++) s += L->f[i * N + id];
    L->rho[id] = s;
    if (!(s > 0.0)) L->status |= ORC_ST_RHO_NONPOS;
    if (p->eos_b * s >= 1.0) L->status |= ORC_ST_EOS_POLE;
    check(L, s, 0);
  }
  /* pseudopotential, Eqs. 10-11 */
  for (int id = 0; id < N; id++) {
    int neg = 0;
    if (!(L->T[id] > 0.0)) L->status |= ORC_ST_T_NONPOS;
    L->psi[id] = p->multiphase ? orc_psi(p, L->rho[id], L->T[id], &neg) : 0.0;
    if (neg) L->status |= ORC_ST_PSI_NEG;
  }
  /* forces, Eqs. 9, 14, 15 */
  double gcos = cos(p->g_omega * (double)L->t);
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      int id = y * nx + x;
      double sfx = 0.0, sfy = 0.0, swx = 0.0, swy = 0.0;
      for (int i = 1; i < 9; i++) {
        int xo, yo;
        int k = classify(L, x, y, EX[i], EY[i], &xo, &yo);
        if (k == NB_SOLID) {
          swx += WPSI[i] * EX[i];
          swy += WPSI[i] * EY[i];
        } else {
          double pn = L->psi[yo * nx + xo];
          sfx += WPSI[i] * pn * EX[i];
          sfy += WPSI[i] * pn * EY[i];
        }
      }
      double Fx = 0.0, Fy = 0.0, Fm2 = 0.0;
      if (p->multiphase) {
        double ps = L->psi[id];
        double Fmx = -p->G * ps * sfx, Fmy = -p->G * ps * sfy;
        double psw = p->rho_w > 0.0 ? orc_psi(p, p->rho_w, L->T[id], NULL) : ps;
        double Fax = -p->Gw * ps * psw * swx, Fay = -p->Gw * ps * psw * swy;
        Fx = Fmx + Fax;
        Fy = Fmy + Fay;
        Fm2 = ps > 0.0 ? (Fmx * Fmx + Fmy * Fmy) / (ps * ps) : 0.0;
      }
      Fx += (L->rho[id] - p->rho_g) * p->gx * gcos;
      Fy += (L->rho[id] - p->rho_g) * p->gy * gcos;
      L->Fx[id] = Fx;
      L->Fy[id] = Fy;
      L->Fm2psi2[id] = Fm2;
    }
  /* velocity, Eq. 13 */
  for (int id = 0; id < N; id++) {
    double jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; i++) {
      jx += EX[i] * L->f[i * N + id];
      jy += EY[i] * L->f[i * N + id];
    }
    L->ux[id] = (jx + 0.5 * L->Fx[id]) / L->rho[id];
    L->uy[id] = (jy + 0.5 * L->Fy[id]) / L->rho[id];
    check(L, L->ux[id] + L->uy[id], 0);
  }
}

/* ------------------------------------------------------------------ */
/* Energy equation, Eqs. 16-18                                         */
/* ------------------------------------------------------------------ */

static double ghost_T(const orc_lattice *L, const double *Tf, int x, int y, int i) {
  int xo, yo;
  int k = classify(L, x, y, EX[i], EY[i], &xo, &yo);
  if (k == NB_SOLID) {
    /* isothermal: the wall temperature; adiabatic: the fluid node across the wall
       (the ghost mirrors the first fluid row, so the normal gradient vanishes) */
    int top = y + EY[i] >= L->ny;
    if (wall_adiabatic(L, xo, top)) return Tf[(top ? L->ny - 1 : 0) * L->nx + xo];
    return wall_temperature(L, xo, top);
  }
  if (k == NB_INLET) return L->Tc * L->p.T_inlet;
  return Tf[yo * L->nx + xo]; /* fluid, or outlet copy */
}

static void ghost_u(const orc_lattice *L, const double *ux, const double *uy, int x, int y,
                    int i, double *vx, double *vy) {
  int xo, yo;
  int k = classify(L, x, y, EX[i], EY[i], &xo, &yo);
  if (k == NB_SOLID) { *vx = 0.0; *vy = 0.0; return; }
  if (k == NB_INLET && L->p.x_bc == ORC_X_INLET_OUTLET) {
    *vx = inlet_velocity(L, L->t);
    *vy = 0.0;
    return;
  }
  *vx = ux[yo * L->nx + xo];
  *vy = uy[yo * L->nx + xo];
}

/* K(T) = -u.grad T + lambda lap T / (rho Cv) - T (dP/dT)_rho div u / (rho Cv) */
static void energy_rhs(orc_lattice *L, const double *rho, const double *ux, const double *uy,
                       const double *divu, const double *Tf, double *K) {
  const orc_params *p = &L->p;
  for (int y = 0; y < L->ny; y++)
    for (int x = 0; x < L->nx; x++) {
      int id = y * L->nx + x;
      double c = Tf[id], gx = 0.0, gy = 0.0, lap = 0.0;
      for (int i = 1; i < 9; i++) {
        double v = ghost_T(L, Tf, x, y, i);
        gx += WLAT[i] * v * EX[i];
        gy += WLAT[i] * v * EY[i];
        lap += WLAT[i] * (v - c);
      }
      gx *= 3.0;
      gy *= 3.0;
      lap *= 6.0;
      double rcv = rho[id] * p->Cv;
      K[id] = -(ux[id] * gx + uy[id] * gy) + p->lambda * lap / rcv -
              c * orc_eos_dpdt(p, rho[id], c) * divu[id] / rcv;
    }
}

static void divergence(orc_lattice *L, const double *ux, const double *uy, double *divu) {
  for (int y = 0; y < L->ny; y++)
    for (int x = 0; x < L->nx; x++) {
      double s = 0.0;
      for (int i = 1; i < 9; i++) {
        double vx, vy;
        ghost_u(L, ux, uy, x, y, i, &vx, &vy);
        s += WLAT[i] * (vx * EX[i] + vy * EY[i]);
      }
      divu[y * L->nx + x] = 3.0 * s;
    }
}

int orc_energy_rhs(orc_lattice *L, const double *rho, const double *ux, const double *uy,
                   const double *T, double *K) {
  divergence(L, ux, uy, L->divu);
  energy_rhs(L, rho, ux, uy, L->divu, T, K);
  return 0;
}

/* classical fourth-order Runge-Kutta with rho, u frozen at time t */
static void advance_temperature(orc_lattice *L) {
  int N = L->nx * L->ny;
  static const double stage_c[4] = {0.0, 0.5, 0.5, 1.0};
  static const double weight[4] = {1.0, 2.0, 2.0, 1.0};
  divergence(L, L->ux, L->uy, L->divu);
  for (int id = 0; id < N; id++) { L->acc[id] = 0.0; L->h[id] = 0.0; }
  for (int s = 0; s < 4; s++) {
    for (int id = 0; id < N; id++) L->Tk[id] = L->T[id] + stage_c[s] * L->h[id];
    energy_rhs(L, L->rho, L->ux, L->uy, L->divu, L->Tk, L->h);
    for (int id = 0; id < N; id++) L->acc[id] += weight[s] * L->h[id];
  }
  for (int id = 0; id < N; id++) {
    L->Tn[id] = L->T[id] + L->acc[id] / 6.0;
    check(L, L->Tn[id], 0);
  }
}

/* ------------------------------------------------------------------ */
/* Lattice life cycle and the time step                                */
/* ------------------------------------------------------------------ */

orc_lattice *orc_create(int nx, int ny, const orc_params *p) {
  if (nx < 1 || ny < 1) return NULL;
  if (p->x_bc != ORC_X_PERIODIC && nx < 2) return NULL;
  orc_lattice *L = (orc_lattice *)calloc(1, sizeof(orc_lattice));
  size_t N = (size_t)nx * ny;
  L->nx = nx;
  L->ny = ny;
  L->p = *p;
  L->Tc = orc_critical_temperature(p);
  L->f = calloc(9 * N, sizeof(double));
  L->fs = calloc(9 * N, sizeof(double));
  L->fn = calloc(9 * N, sizeof(double));
  double **arr[] = {&L->T, &L->rho, &L->psi, &L->Fx, &L->Fy, &L->Fm2psi2, &L->ux,
                    &L->uy, &L->Tk, &L->h, &L->acc, &L->Tn, &L->divu};
  for (size_t k = 0; k < sizeof(arr) / sizeof(arr[0]); k++) *arr[k] = calloc(N, sizeof(double));
  for (size_t id = 0; id < N; id++) L->T[id] = p->T0 * L->Tc;
  return L;
}

void orc_destroy(orc_lattice *L) {
  if (!L) return;
  double *arr[] = {L->f, L->fs, L->fn, L->T, L->rho, L->psi, L->Fx, L->Fy, L->Fm2psi2,
                   L->ux, L->uy, L->Tk, L->h, L->acc, L->Tn, L->divu};
  for (size_t k = 0; k < sizeof(arr) / sizeof(arr[0]); k++) free(arr[k]);
  free(L);
}

int orc_set_fields(orc_lattice *L, const double *rho0, const double *T) {
  int N = L->nx * L->ny;
  for (int id = 0; id < N; id++) {
    double feq[9];
    orc_feq(rho0[id], 0.0, 0.0, feq);
    for (int i = 0; i < 9; i++) L->f[i * N + id] = feq[i];
    L->T[id] = T ? T[id] : L->p.T0 * L->Tc;
  }
  apply_open_boundaries(L, L->f, L->t);
  return 0;
}

int orc_step(orc_lattice *L, long nsteps) {
  int N = L->nx * L->ny;
  for (long n = 0; n < nsteps; n++) {
    macroscopic(L);
    for (int id = 0; id < N; id++) {
      double f[9], fs[9];
      for (int i = 0; i < 9; i++) f[i] = L->f[i * N + id];
      orc_collide_node(&L->p, f, L->Fx[id], L->Fy[id], L->Fm2psi2[id], fs);
      for (int i = 0; i < 9; i++) L->fs[i * N + id] = fs[i];
    }
    stream(L);
    if (L->p.thermal) {
      advance_temperature(L);
      double *tmp = L->T; L->T = L->Tn; L->Tn = tmp;
    }
    double *tmp = L->f; L->f = L->fn; L->fn = tmp;
    L->t += 1;
  }
  return (int)L->status;
}

int orc_fields(orc_lattice *L, double *rho, double *ux, double *uy, double *T) {
  int N = L->nx * L->ny;
  macroscopic(L);
  for (int id = 0; id < N; id++) {
    if (rho) rho[id] = L->rho[id];
    if (ux) ux[id] = L->ux[id];
    if (uy) uy[id] = L->uy[id];
    if (T) T[id] = L->T[id];
  }
  return 0;
}

int orc_populations(orc_lattice *L, double *f) {
  memcpy(f, L->f, sizeof(double) * 9 * (size_t)L->nx * L->ny);
  return 0;
}

int orc_set_populations(orc_lattice *L, const double *f) {
  memcpy(L->f, f, sizeof(double) * 9 * (size_t)L->nx * L->ny);
  return 0;
}

void orc_mass_heat(orc_lattice *L, double *mass, double *heat) {
  int N = L->nx * L->ny;
  double m = 0.0, h = 0.0;
  for (int id = 0; id < N; id++) {
    double r = 0.0;
    for (int i = 0; i < 9; i++) r += L->f[i * N + id];
    m += r;
    h += r * L->p.Cv * L->T[id];
  }
  *mass = m;
  *heat = h;
}

long orc_time(const orc_lattice *L) { return L->t; }
unsigned orc_status(const orc_lattice *L) { return L->status; }
