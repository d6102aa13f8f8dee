/*
 * Plain FP64 CPU oracle of the D2Q9 pseudopotential MRT lattice Boltzmann
 * update with the finite-difference energy equation (Zhao, Xu & Zhang,
 * arXiv:1803.01756, Section 2, Eqs. 1-18).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Every stage is one loop nest over the whole grid writing a whole-grid array,
 * in the order of the paper's flow of Section 2 (density -> pseudopotential ->
 * forces -> velocity -> moment-space collision -> streaming with boundaries ->
 * Runge-Kutta temperature update).  Readings of passages that are silent or
 * garbled are stated beside the code that takes them.
 */
#ifndef PPLBM_ORACLE_H
#define PPLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* x boundary modes */
#define ORC_X_PERIODIC 0
#define ORC_X_INLET_OUTLET 1 /* Zou-He velocity inlet at x=0, density outlet at x=nx-1 */
#define ORC_X_PRESSURE_INLET 2 /* Zou-He pressure inlet at x=0, density outlet at x=nx-1 */
/* y boundary modes */
#define ORC_Y_PERIODIC 0
#define ORC_Y_WALLS 1        /* half-way bounce-back walls below y=0 and above y=ny-1 */

/* status bits */
#define ORC_ST_NAN 1u
#define ORC_ST_PSI_NEG 2u    /* argument of the square root of Eq. 10 negative */
#define ORC_ST_RHO_NONPOS 4u
#define ORC_ST_EOS_POLE 8u   /* b*rho >= 1 in Eq. 11 */
#define ORC_ST_T_NONPOS 16u

typedef struct orc_params {
  double eos_a, eos_b, eos_R, eos_omega; /* Peng-Robinson, Eq. 11 */
  double G;                              /* fluid-fluid strength, Eq. 9 */
  double Gw;                             /* fluid-wall strength, Eq. 14 */
  double rho_w;                          /* Eq. 14 psi(rho_w); <= 0 means the local psi */
  double theta;                          /* Eq. 8 constant */
  double tau_g, tau_l, rho_g, rho_l;     /* Eq. 5 (rho_g also the rho_v of Eq. 15) */
  double s_e, s_zeta, s_q;               /* Eq. 3 rates s1 = s2 (read as s_e, s_zeta), s4 = s6 */
  double Cv, lambda;                     /* Eq. 16 */
  double gx, gy, g_omega;                /* Eq. 15 body force, times cos(g_omega t) */
  double T0, T_wall_left, T_wall_right, T_inlet; /* in units of Tc */
  int x_bc, y_bc;
  double u_amp, u_period;                /* inlet u = u_amp sin(2 pi t / u_period) */
  double rho_out;                        /* outlet density */
  int thermal;                           /* 1: advance T by Eqs. 16-18 */
  int multiphase;                        /* 1: pseudopotential forces of Eqs. 9, 14 */
  double p_amp_frac;                     /* pressure inlet: p = p0 (1 + p_amp_frac sin(2 pi t/u_period)) */
  /* Section 3.2 walls: the top wall's temperature profile (units of Tc, linear in x;
     both 0 means the profile of T_wall_left/right) and, per wall, the columns
     [x0, x1) that are isothermal; the rest of that wall is adiabatic (zero normal
     gradient of T: the energy-equation ghost copies the fluid node across the wall).
     x1 <= x0: the whole wall is isothermal. */
  double T_top_left, T_top_right;
  int top_iso_x0, top_iso_x1;
  int bot_iso_x0, bot_iso_x1;
} orc_params;

typedef struct orc_lattice orc_lattice;

/* ---- pure functions (for pins) ---- */
double orc_critical_temperature(const orc_params *p);
double orc_eos_pressure(const orc_params *p, double rho, double T);
double orc_eos_dpdt(const orc_params *p, double rho, double T);
/* psi of Eq. 10; sets *neg when the square-root argument is negative (then psi = 0) */
double orc_psi(const orc_params *p, double rho, double T, int *neg);
/* the 9x9 integer matrix of Eq. 6, row-major */
void orc_moment_matrix(int M[81]);
/* second-order D2Q9 equilibrium */
void orc_feq(double rho, double ux, double uy, double feq[9]);
/* m^eq of Eq. 6 as a function of rho and u (reading: compressible form M f^eq) */
void orc_meq(double rho, double ux, double uy, double meq[9]);
/* S-bar of Eq. 8 */
void orc_forcing_moments(double ux, double uy, double Fx, double Fy,
                         double Fm2_over_psi2, double theta, double s_e,
                         double s_zeta, double S[9]);
/* one collision of Eq. 7 on a single node: f (in) -> fstar (out) */
void orc_collide_node(const orc_params *p, const double f[9], double Fx, double Fy,
                      double Fm2_over_psi2, double fstar[9]);

/* isotropic finite-difference stencils used by Eq. 16 on a whole periodic grid */
void orc_grad_periodic(int nx, int ny, const double *phi, double *gx, double *gy);
void orc_lap_periodic(int nx, int ny, const double *phi, double *lap);

/* inlet density of the pressure inlet at time t: the vapour-branch root of
   P_EOS(rho, T_inlet) = p0 (1 + p_amp_frac sin(2 pi t / u_period)), p0 = P_EOS(rho_out, T_inlet) */
double orc_inlet_density(const orc_params *p, long t);

/* ---- lattice ---- */
orc_lattice *orc_create(int nx, int ny, const orc_params *p);
void orc_destroy(orc_lattice *L);
/* rho0 [ny*nx]; T (absolute) [ny*nx] or NULL for uniform T0*Tc.  Sets f = f^eq(rho0, 0)
   and applies the open-boundary rules at time 0. */
int orc_set_fields(orc_lattice *L, const double *rho0, const double *T);
int orc_step(orc_lattice *L, long nsteps);
/* fields at the current time t: rho, u (Eq. 13 with the force of time t), T */
int orc_fields(orc_lattice *L, double *rho, double *ux, double *uy, double *T);
/* raw pre-collision populations [9][ny][nx] at time t */
int orc_populations(orc_lattice *L, double *f);
int orc_set_populations(orc_lattice *L, const double *f);
/* FP64 sum of rho and of rho*Cv*T */
void orc_mass_heat(orc_lattice *L, double *mass, double *heat);
long orc_time(const orc_lattice *L);
unsigned orc_status(const orc_lattice *L);
/* K(T) of Eq. 16 for given whole-grid rho, u, T (ghost rules of the lattice at its
   current time); used by the energy-equation pins */
int orc_energy_rhs(orc_lattice *L, const double *rho, const double *ux, const double *uy,
                   const double *T, double *K);

#ifdef __cplusplus
}
#endif
#endif
