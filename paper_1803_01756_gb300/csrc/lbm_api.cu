// Host runtime and C ABI (include/lbm.h).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_handle.h"

using lbm::DevParams;
using lbm::StepScalars;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr uint32_t kStateMagic = 0x534d424cu;  // "LBMS"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
  uint32_t magic, version;
  int32_t nx, ny, pitch, storage;
  int64_t t;
  int64_t reserved[4];
};

using namespace lbm_host;
const char *kKernelNames[KN_COUNT] = {"k_density_psi", "k_collide", "k_energy", "k_fused_step",
                                       "k_stream_collide", "k_energy_rk4"};


}  // namespace

namespace lbm_host {

int cuda_fail(cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  if (e == cudaErrorMemoryAllocation) return LBM_ERR_OOM;
  return LBM_ERR_CUDA;
}

}  // namespace lbm_host

namespace {

double critical_temperature(const lbm_params_t &p) {
  return 0.0778 * p.eos_a / (0.45724 * p.eos_b * p.eos_R);
}

bool valid_rate(double s) { return s > 0.0 && s < 2.0; }

// Lattice columns per thread of the fused kernel for an nx x ny lattice.
int default_cpt(int nx, int ny) {
  (void)nx;
  (void)ny;
  return 1;
}

int validate(int nx, int ny, const lbm_params_t &p) {
  if (nx < 1 || ny < 1) return LBM_ERR_ARG;
  if (nx > (1 << 20) || ny > (1 << 20)) return LBM_ERR_ARG;
  if (p.x_bc != LBM_X_PERIODIC && p.x_bc != LBM_X_INLET_OUTLET && p.x_bc != LBM_X_PRESSURE_INLET)
    return LBM_ERR_ARG;
  if (p.y_bc != LBM_Y_PERIODIC && p.y_bc != LBM_Y_WALLS) return LBM_ERR_ARG;
  if (p.x_bc != LBM_X_PERIODIC && (nx < 2 || !(p.rho_out > 0.0))) return LBM_ERR_ARG;
  if (p.x_bc == LBM_X_PRESSURE_INLET && !(std::fabs(p.p_amp_frac) < 1.0)) return LBM_ERR_ARG;
  if (!(p.eos_a > 0.0) || !(p.eos_b > 0.0) || !(p.eos_R > 0.0)) return LBM_ERR_ARG;
  if (p.multiphase && !(p.G != 0.0)) return LBM_ERR_ARG;
  if (p.thermal && !(p.Cv > 0.0)) return LBM_ERR_ARG;
  if (!(p.T0 > 0.0)) return LBM_ERR_ARG;
  if (!(p.tau_g > 0.5) || !(p.tau_l > 0.5)) return LBM_ERR_ARG;
  if (!valid_rate(p.s_e) || !valid_rate(p.s_zeta) || !valid_rate(p.s_q)) return LBM_ERR_ARG;
  if (p.storage != LBM_STORAGE_F32 && p.storage != LBM_STORAGE_BF16 && p.storage != LBM_STORAGE_F16)
    return LBM_ERR_ARG;
  if (p.kernel < LBM_KERNEL_AUTO || p.kernel > LBM_KERNEL_TWOPASS) return LBM_ERR_ARG;
  if (p.u_period < 0.0 || std::fabs(p.u_amp) >= 1.0) return LBM_ERR_ARG;
  // adiabatic wall columns (outside a non-empty isothermal window) only with periodic x
  const bool adia = (p.top_iso_x1 > p.top_iso_x0 && (p.top_iso_x0 > 0 || p.top_iso_x1 < nx)) ||
                    (p.bot_iso_x1 > p.bot_iso_x0 && (p.bot_iso_x0 > 0 || p.bot_iso_x1 < nx));
  if (adia && (p.x_bc != LBM_X_PERIODIC || p.y_bc != LBM_Y_WALLS)) return LBM_ERR_ARG;
  return LBM_OK;
}

DevParams derive(int nx, int ny, int pitch, const lbm_params_t &p, double &Tc, double &T_ref,
                 double &rho_ref) {
  DevParams d{};
  d.nx = nx;
  d.ny = ny;
  d.pitch = pitch;
  d.plane = (long long)ny * pitch;
  d.x_open = p.x_bc != LBM_X_PERIODIC;
  d.p_inlet = p.x_bc == LBM_X_PRESSURE_INLET;
  d.y_walls = p.y_bc == LBM_Y_WALLS;
  d.multiphase = p.multiphase != 0;
  d.thermal = p.thermal != 0;
  Tc = critical_temperature(p);
  T_ref = p.T0 * Tc;
  // deviation reference: given, else the gas density, else the outlet density, else 1
  rho_ref = p.rho_ref > 0.0 ? p.rho_ref
                            : (p.rho_g > 0.0 ? p.rho_g : (p.rho_out > 0.0 ? p.rho_out : 1.0));
  d.rho_ref = (float)rho_ref;
  d.T_ref = (float)T_ref;
  d.Tc = (float)Tc;
  d.inv_Tc = (float)(1.0 / Tc);
  d.eos_a = (float)p.eos_a;
  d.eos_b = (float)p.eos_b;
  d.eos_R = (float)p.eos_R;
  d.kappa = (float)(0.37464 + 1.54226 * p.eos_omega - 0.26992 * p.eos_omega * p.eos_omega);
  d.G = (float)p.G;
  d.Gw = (float)p.Gw;
  d.rho_w = (float)p.rho_w;
  {
    // reference state of the deviation pseudopotential, evaluated in double at the
    // FP32 values of rho_ref and T_ref that the kernels add deviations to
    const double rr = (double)d.rho_ref, Tr = (double)d.T_ref, b = p.eos_b;
    const double kap = (double)d.kappa;
    const double Dr = 1.0 + 2.0 * b * rr - b * b * rr * rr;
    const double sr = std::sqrt(Tr / Tc);
    const double rphi = 1.0 + kap * (1.0 - sr);
    const double P = rr * p.eos_R * Tr / (1.0 - b * rr) - p.eos_a * rphi * rphi * rr * rr / Dr;
    const double psi2 = p.G != 0.0 ? 2.0 * (P - rr / 3.0) / p.G : 0.0;
    const double tG = p.G != 0.0 ? 2.0 / p.G : 0.0;
    d.sr = (float)sr;
    d.rphi_r = (float)rphi;
    d.kappa1 = (float)(1.0 + kap);
    d.psi_r2 = (float)(psi2 > 0.0 ? psi2 : 0.0);
    d.psi_r = (float)std::sqrt(psi2 > 0.0 ? psi2 : 0.0);
    d.ps_RT = (float)(tG * p.eos_R);
    d.ps_R = (float)(tG * p.eos_R * Tr / (1.0 - b * rr));
    d.ps_g = (float)(1.0 + 2.0 * b * rr);
    d.ps_B = (float)(tG * p.eos_a * rphi * rphi / Dr);
    d.ps_phi = (float)(-tG * p.eos_a * kap);
    d.ps_3 = (float)(-tG / 3.0);
    d.G3 = (float)(-p.G / 3.0);
    d.G3r = (float)(-p.G / 3.0 * std::sqrt(psi2 > 0.0 ? psi2 : 0.0));
    d.wall_r = (float)((p.G - p.Gw) * std::sqrt(psi2 > 0.0 ? psi2 : 0.0));
    d.drho_ref_g = (float)(rr - p.rho_g);
  }
  d.c_theta_e = (float)(12.0 * p.theta * p.s_e * p.G * p.G);
  d.c_theta_z = (float)(12.0 * p.theta * p.s_zeta * p.G * p.G);
  {
    const double se = p.s_e, sz = p.s_zeta, sq = p.s_q;
    const double cte = 12.0 * p.theta * se * p.G * p.G, ctz = 12.0 * p.theta * sz * p.G * p.G;
    const double k1[5] = {(1.0 - se) / 36.0, -2.0 * se / 36.0, 3.0 * se / 36.0,
                          (1.0 - 0.5 * se) * 6.0 / 36.0, cte / 36.0 / 9.0};
    const double k2[5] = {(1.0 - sz) / 36.0, sz / 36.0, -3.0 * sz / 36.0,
                          -(1.0 - 0.5 * sz) * 6.0 / 36.0, -ctz / 36.0 / 9.0};
    const double kq[3] = {(1.0 - sq) / 12.0, -sq / 12.0, -(1.0 - 0.5 * sq) / 12.0};
    for (int i = 0; i < 5; i++) {
      d.k1[i] = (float)k1[i];
      d.k2[i] = (float)k2[i];
    }
    for (int i = 0; i < 3; i++) d.kq[i] = (float)kq[i];
  }
  d.s_e = (float)p.s_e;
  d.s_z = (float)p.s_zeta;
  d.s_q = (float)p.s_q;
  d.tau_g = (float)p.tau_g;
  d.dtau = (float)(p.tau_l - p.tau_g);
  d.rho_g = (float)p.rho_g;
  d.inv_drho = p.rho_l != p.rho_g ? (float)(1.0 / (p.rho_l - p.rho_g)) : 0.0f;
  d.tau_const = p.tau_g == p.tau_l || p.rho_l == p.rho_g;
  d.s_nu_const = (float)(1.0 / p.tau_g);
  {
    const double sn = 1.0 / p.tau_g;
    d.kn[0] = (float)(0.25 * (1.0 - sn));
    d.kn[1] = (float)(0.25 * sn);
    d.kn[2] = (float)(0.25 * (2.0 - sn));
    d.kn[3] = (float)(0.25 * (1.0 - 0.5 * sn));
  }
  d.gx = (float)p.gx;
  d.gy = (float)p.gy;
  d.has_g = p.gx != 0.0 || p.gy != 0.0;
  d.Cv = (float)p.Cv;
  d.lambda = (float)p.lambda;
  d.lam_cv = p.Cv > 0.0 ? (float)(p.lambda / p.Cv) : 0.0f;
  d.R_cv = p.Cv > 0.0 ? (float)(p.eos_R / p.Cv) : 0.0f;
  d.akap_cv = p.Cv > 0.0 ? (float)(p.eos_a * (0.37464 + 1.54226 * p.eos_omega -
                                             0.26992 * p.eos_omega * p.eos_omega) / p.Cv)
                         : 0.0f;
  {
    const double kap = 0.37464 + 1.54226 * p.eos_omega - 0.26992 * p.eos_omega * p.eos_omega;
    const double akap = p.eos_a * kap;
    d.lam23_cv = p.Cv > 0.0 ? (float)(2.0 * p.lambda / (3.0 * p.Cv)) : 0.0f;
    d.RTc_cv3 = p.Cv > 0.0 ? (float)(p.eos_R * Tc / (3.0 * p.Cv)) : 0.0f;
    d.akap1_cv3 = p.Cv > 0.0 ? (float)(akap * (1.0 + kap) / (3.0 * p.Cv)) : 0.0f;
    d.kappa_r = (float)(kap / (1.0 + kap));
    d.xr = (float)((double)d.T_ref / Tc);
  }
  d.tw0 = (float)(Tc * p.T_wall_left - T_ref);
  d.tw_slope = nx > 1 ? (float)(Tc * (p.T_wall_right - p.T_wall_left) / (nx - 1)) : 0.0f;
  {
    const bool own = p.T_top_left != 0.0 || p.T_top_right != 0.0;
    const double a = own ? p.T_top_left : p.T_wall_left, b = own ? p.T_top_right : p.T_wall_right;
    d.tw0_top = (float)(Tc * a - T_ref);
    d.tw_slope_top = nx > 1 ? (float)(Tc * (b - a) / (nx - 1)) : 0.0f;
  }
  d.top_iso_x0 = p.top_iso_x0;
  d.top_iso_x1 = p.top_iso_x1;
  d.bot_iso_x0 = p.bot_iso_x0;
  d.bot_iso_x1 = p.bot_iso_x1;
  d.adiabatic = p.y_bc == LBM_Y_WALLS &&
                ((p.top_iso_x1 > p.top_iso_x0 && (p.top_iso_x0 > 0 || p.top_iso_x1 < nx)) ||
                 (p.bot_iso_x1 > p.bot_iso_x0 && (p.bot_iso_x0 > 0 || p.bot_iso_x1 < nx)));
  d.T_inlet_dev = (float)(Tc * p.T_inlet - T_ref);
  d.rho_out = (float)p.rho_out;
  return d;
}

// Peng-Robinson pressure of Eq. 11 (host, double)
double host_pressure(const lbm_params_t &p, double Tc, double rho, double T) {
  const double k = 0.37464 + 1.54226 * p.eos_omega - 0.26992 * p.eos_omega * p.eos_omega;
  const double r = 1.0 + k * (1.0 - std::sqrt(T / Tc));
  const double br = p.eos_b * rho;
  return rho * p.eos_R * T / (1.0 - br) - p.eos_a * r * r * rho * rho / (1.0 + 2.0 * br - br * br);
}

// Real roots of the polynomial c[0] + c[1] x + ... + c[deg] x^deg in [lo, hi], in
// increasing order.  The roots of the derivative (found the same way, down to degree 1)
// split [lo, hi] into pieces on which the polynomial is monotone, so each piece holds at
// most one root, located by Newton steps kept inside the piece's bracket.
int poly_roots(const double *c, int deg, double lo, double hi, double *out) {
  auto eval = [&](double x) {
    double v = c[deg];
    for (int k = deg - 1; k >= 0; k--) v = v * x + c[k];
    return v;
  };
  while (deg > 0 && c[deg] == 0.0) deg--;
  if (deg == 0) return 0;
  if (deg == 1) {
    const double x = -c[0] / c[1];
    if (x >= lo && x <= hi) {
      out[0] = x;
      return 1;
    }
    return 0;
  }
  double dc[4], crit[4];
  for (int k = 1; k <= deg; k++) dc[k - 1] = k * c[k];
  const int nc = poly_roots(dc, deg - 1, lo, hi, crit);
  double edge[6];
  int ne = 0;
  edge[ne++] = lo;
  for (int k = 0; k < nc; k++) edge[ne++] = crit[k];
  edge[ne++] = hi;
  int n = 0;
  for (int k = 0; k + 1 < ne; k++) {
    double a = edge[k], b = edge[k + 1];
    double fa = eval(a), fb = eval(b);
    if (fa == 0.0) {
      if (n == 0 || out[n - 1] != a) out[n++] = a;
      continue;
    }
    if (fa * fb > 0.0) continue;
    if (fb == 0.0) continue;  // taken as the left end of the next piece
    double x = 0.5 * (a + b);
    for (int it = 0; it < 200; it++) {
      const double fx = eval(x);
      if (fx == 0.0) break;
      if ((fx > 0.0) == (fa > 0.0)) { a = x; fa = fx; } else { b = x; }
      double d = dc[deg - 1];
      for (int m = deg - 2; m >= 0; m--) d = d * x + dc[m];
      double xn = d != 0.0 ? x - fx / d : 0.5 * (a + b);
      if (!(xn > a && xn < b)) xn = 0.5 * (a + b);
      if (std::fabs(xn - x) <= 1e-16 * std::fabs(x) || b - a <= 1e-16 * std::fabs(b)) {
        x = xn;
        break;
      }
      x = xn;
    }
    out[n++] = x;
  }
  return n;
}

// Upper end of the vapour branch of the Peng-Robinson isotherm (Eq. 11) at temperature T:
// its first maximum, where dP/drho = R T / (1 - b rho)^2 - 2 a phi rho (1 + b rho) / D^2
// vanishes (D = 1 + 2 b rho - b^2 rho^2), or 0.999 / b when the isotherm rises up to the
// pole (T >= Tc).  With x = b rho, dP/drho has the sign of the quartic
//   q(x) = D^2 - c x (1 + x) (1 - x)^2
//        = 1 + (4 - c) x + (2 + c) x^2 + (c - 4) x^3 + (1 - c) x^4,   c = 2 a phi / (b R T),
// and q(0) = 1 > 0, so the branch ends at the smallest root of q in (0, 1).
double vapour_branch_end(const lbm_params_t &p, double Tc, double T) {
  const double k = 0.37464 + 1.54226 * p.eos_omega - 0.26992 * p.eos_omega * p.eos_omega;
  const double r = 1.0 + k * (1.0 - std::sqrt(T / Tc));
  const double c = 2.0 * p.eos_a * r * r / (p.eos_b * p.eos_R * T);
  const double q[5] = {1.0, 4.0 - c, 2.0 + c, c - 4.0, 1.0 - c};
  double roots[4];
  const int n = poly_roots(q, 4, 0.0, 0.999, roots);
  return (n > 0 ? roots[0] : 0.999) / p.eos_b;
}

// Inlet density of the pressure inlet at time t: the density on the vapour branch whose
// pressure is p0 (1 + p_amp_frac sin(2 pi t / P)), p0 = P(rho_out, T_inlet).  P rises
// strictly on [0, branch end], so Newton steps on P(rho) - target with the analytic
// dP/drho, kept inside a shrinking bracket, converge from the ideal-gas estimate; a target
// above the branch's top pressure gives the branch end.
double inlet_density(const lbm_params_t &p, double Tc, double branch_end, long long t) {
  const double T = Tc * p.T_inlet;
  const double p0 = host_pressure(p, Tc, p.rho_out, T);
  const double s = p.u_period == 0.0 ? 1.0 : std::sin(2.0 * kPi * (double)t / p.u_period);
  const double target = p0 * (1.0 + p.p_amp_frac * s);
  double lo = 0.0, hi = branch_end;
  if (target >= host_pressure(p, Tc, hi, T)) return hi;
  if (target <= 0.0) return 0.0;
  const double k = 0.37464 + 1.54226 * p.eos_omega - 0.26992 * p.eos_omega * p.eos_omega;
  const double r = 1.0 + k * (1.0 - std::sqrt(T / Tc));
  const double aphi = p.eos_a * r * r;
  double rho = std::min(target / (p.eos_R * T), 0.5 * hi);
  for (int it = 0; it < 100; it++) {
    const double f = host_pressure(p, Tc, rho, T) - target;
    if (f == 0.0) break;
    if (f < 0.0) lo = rho; else hi = rho;
    const double br = p.eos_b * rho, D = 1.0 + 2.0 * br - br * br;
    const double dP = p.eos_R * T / ((1.0 - br) * (1.0 - br)) -
                      2.0 * aphi * rho * (1.0 + br) / (D * D);
    double next = dP > 0.0 ? rho - f / dP : 0.5 * (lo + hi);
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    if (std::fabs(next - rho) <= 1e-15 * rho) {
      rho = next;
      break;
    }
    rho = next;
  }
  return rho;
}

}  // namespace

lbm::StepScalars lbm_host::scalars_at(const lbm_lattice *h, long long t) {
  StepScalars s;
  double u = h->p.u_period == 0.0 ? h->p.u_amp
                                   : h->p.u_amp * std::sin(2.0 * kPi * (double)t / h->p.u_period);
  s.u_in = (float)u;
  s.gcos = (float)std::cos(h->p.g_omega * (double)t);
  s.rho_in = h->p.x_bc == LBM_X_PRESSURE_INLET
                 ? (float)inlet_density(h->p, h->Tc, h->rho_branch_end, t)
                 : 0.0f;
  return s;
}

namespace {

cudaEvent_t take_event(lbm_lattice *h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int drain_timing(lbm_lattice *h) {
  for (auto &tl : h->pending) {
    LBM_CUDA(cudaEventSynchronize(tl.b));
    float ms = 0.0f;
    LBM_CUDA(cudaEventElapsedTime(&ms, tl.a, tl.b));
    h->total_ms[tl.kind] += ms;
    h->launches[tl.kind] += 1;
    h->pool.push_back(tl.a);
    h->pool.push_back(tl.b);
  }
  h->pending.clear();
  return LBM_OK;
}

// launch wrapper that brackets the launch with events when timing is on
template <typename F>
int timed(lbm_lattice *h, int kind, cudaStream_t s, F &&launch) {
  if (!h->timing) return cuda_fail(launch());
  TimedLaunch tl{kind, take_event(h), take_event(h)};
  if (!tl.a || !tl.b) return LBM_ERR_CUDA;
  LBM_CUDA(cudaEventRecord(tl.a, s));
  cudaError_t e = launch();
  LBM_CUDA(cudaEventRecord(tl.b, s));
  h->pending.push_back(tl);
  if (h->pending.size() >= 32768) {
    int rc = drain_timing(h);
    if (rc) return rc;
  }
  return cuda_fail(e);
}

int compute_rho_psi(lbm_lattice *h, cudaStream_t s) {
  StepScalars sc = scalars_at(h, h->t);
  return cuda_fail(lbm::launch_density_psi(h->dp, h->p.storage, h->g[h->cur], h->T[h->tcur],
                                           h->rho, h->psi, h->status, sc, s));
}

void advance(lbm_lattice *h) {
  h->cur ^= 1;
  if (h->dp.thermal) h->tcur ^= 1;
  h->t += 1;
}

// one update through the split path (three launches)
int split_update(lbm_lattice *h, cudaStream_t s) {
  StepScalars sc = scalars_at(h, h->t);
  const DevParams &d = h->dp;
  int rc = timed(h, KN_DENSITY, s, [&] {
    return lbm::launch_density_psi(d, h->p.storage, h->g[h->cur], h->T[h->tcur], h->rho, h->psi,
                                   h->status, sc, s);
  });
  if (rc) return rc;
  rc = timed(h, KN_COLLIDE, s, [&] {
    return lbm::launch_collide(d, h->p.storage, h->g[h->cur], h->g[1 - h->cur], h->T[h->tcur],
                               h->psi, h->ux, h->uy, h->status, sc, true, s);
  });
  if (rc) return rc;
  if (d.thermal) {
    rc = timed(h, KN_ENERGY, s, [&] {
      return lbm::launch_energy(d, h->T[h->tcur], h->T[1 - h->tcur], h->rho, h->ux, h->uy,
                                h->status, sc, s);
    });
    if (rc) return rc;
  }
  advance(h);
  return LBM_OK;
}

// the two passes of the current update on the two-pass path, with the scalars of slot k
// of d_sc: A streams and collides (writing rho and u when the energy equation is on), B
// advances T
cudaError_t twopass_a(lbm_lattice *h, int k, cudaStream_t s) {
  return lbm::launch_stream_collide(h->dp, h->p.storage, h->g[h->cur], h->g[1 - h->cur],
                                    h->T[h->tcur], h->rho, h->ux, h->uy, h->status, h->d_sc + k,
                                    h->twopass.Ha, s);
}

cudaError_t twopass_b(lbm_lattice *h, int k, cudaStream_t s) {
  return lbm::launch_energy_rk4(h->dp, h->T[h->tcur], h->T[1 - h->tcur], h->rho, h->ux, h->uy,
                                h->status, h->d_sc + k, h->twopass.Hb, s);
}

// the launches of the current update on the fused or the two-pass path, with the scalars
// of slot k of d_sc
cudaError_t fused_launch(lbm_lattice *h, int k, cudaStream_t s) {
  if (h->kernel == LBM_KERNEL_TWOPASS) {
    cudaError_t e = twopass_a(h, k, s);
    if (e == cudaSuccess && h->dp.thermal) e = twopass_b(h, k, s);
    return e;
  }
  return lbm::launch_fused(h->dp, h->p.storage, h->g[h->cur], h->g[1 - h->cur], h->T[h->tcur],
                           h->T[1 - h->tcur], h->status, h->d_sc + k, h->fused, s);
}

// Scalars of updates t .. t + m - 1 into d_sc, through the staging buffer whose previous
// copy has completed.
int stage_scalars(lbm_lattice *h, int m, cudaStream_t s) {
  const int buf = h->sc_buf;
  if (h->sc_used[buf]) LBM_CUDA(cudaEventSynchronize(h->sc_ev[buf]));
  for (int k = 0; k < m; k++) h->h_sc[buf][k] = scalars_at(h, h->t + k);
  LBM_CUDA(cudaMemcpyAsync(h->d_sc, h->h_sc[buf], sizeof(StepScalars) * m,
                           cudaMemcpyHostToDevice, s));
  LBM_CUDA(cudaEventRecord(h->sc_ev[buf], s));
  h->sc_used[buf] = true;
  h->sc_buf ^= 1;
  return LBM_OK;
}

void drop_graphs(lbm_lattice *h) {
  for (int c = 0; c < 2; c++)
    for (int k = 0; k < 2; k++) {
      if (h->gexec[c][k]) cudaGraphExecDestroy(h->gexec[c][k]);
      if (h->graph[c][k]) cudaGraphDestroy(h->graph[c][k]);
      h->gexec[c][k] = nullptr;
      h->graph[c][k] = nullptr;
    }
}

// Capture the kChunk launches of a chunk that starts at the current buffer parity.
int capture_chunk(lbm_lattice *h) {
  const int c0 = h->cur, t0 = h->tcur;
  LBM_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < lbm_lattice::kChunk; k++) {
    if (e == cudaSuccess) e = fused_launch(h, k, h->cap_stream);
    h->cur ^= 1;
    if (h->dp.thermal) h->tcur ^= 1;
  }
  h->cur = c0;
  h->tcur = t0;
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &g);
  if (e == cudaSuccess) e = ee;
  cudaGraphExec_t x = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e);
  }
  h->graph[c0][t0] = g;
  h->gexec[c0][t0] = x;
  return LBM_OK;
}

// nsteps updates on the fused or two-pass path: chunks of kChunk, each a graph replay when
// graphs are on and per-launch timing is off, else the launches of one update at a time
int fused_steps(lbm_lattice *h, long nsteps, cudaStream_t s) {
  const int C = lbm_lattice::kChunk;
  for (long done = 0; done < nsteps;) {
    const int m = (int)std::min<long>(C, nsteps - done);
    int rc = stage_scalars(h, m, s);
    if (rc) return rc;
    if (m == C && h->use_graph && !h->timing) {
      if (!h->gexec[h->cur][h->tcur]) {
        rc = capture_chunk(h);
        if (rc) return rc;
      }
      LBM_CUDA(cudaGraphLaunch(h->gexec[h->cur][h->tcur], s));
      h->t += C;  // an even chunk ends at the parity it started from
    } else {
      for (int k = 0; k < m; k++) {
        if (h->kernel == LBM_KERNEL_TWOPASS) {
          rc = timed(h, KN_STREAM_COLLIDE, s, [&] { return twopass_a(h, k, s); });
          if (!rc && h->dp.thermal)
            rc = timed(h, KN_ENERGY_RK4, s, [&] { return twopass_b(h, k, s); });
        } else {
          rc = timed(h, KN_FUSED, s, [&] { return fused_launch(h, k, s); });
        }
        if (rc) return rc;
        advance(h);
      }
    }
    done += m;
  }
  return LBM_OK;
}

void free_all(lbm_lattice *h) {
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (int k = 0; k < 2; k++) {
    if (h->h_sc[k]) cudaFreeHost(h->h_sc[k]);
    if (h->sc_ev[k]) cudaEventDestroy(h->sc_ev[k]);
  }
  cudaFree(h->d_sc);
  cudaFree(h->g[0]);
  cudaFree(h->g[1]);
  cudaFree(h->T[0]);
  cudaFree(h->T[1]);
  cudaFree(h->rho);
  cudaFree(h->psi);
  cudaFree(h->ux);
  cudaFree(h->uy);
  cudaFree(h->status);
  cudaFree(h->partials);
  cudaFree(h->sums);
  cudaFree(h->rho0);
  if (h->host_sums) cudaFreeHost(h->host_sums);
  for (auto &tl : h->pending) {
    cudaEventDestroy(tl.a);
    cudaEventDestroy(tl.b);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
}

template <typename T>
cudaError_t dalloc(lbm_lattice *h, T **ptr, size_t count) {
  size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMalloc((void **)ptr, bytes);
  if (e == cudaSuccess) h->device_bytes += bytes;
  return e;
}

// Host fields in: rho (and T) go to the device staging array as they are, and kernels
// form the populations and the pitched FP32 temperature deviations there; the stream
// orders the reuse of the staging array.
// Device address of the host range [p, p + bytes) when all of it lies in one page-locked
// mapping that the device can address (cudaHostAlloc / cudaMallocHost / cudaHostRegister
// memory: the same registration at both ends and at the same offset), else nullptr.  The
// field transfers then read and write such host buffers from their kernels over the
// host link, with no staging copy; any other pointer (pageable memory) takes the copy path.
void *mapped_host(const void *p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  const char *lo = static_cast<const char *>(p), *hi = lo + bytes - 1;
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, lo) != cudaSuccess ||
      cudaPointerGetAttributes(&b, hi) != cudaSuccess) {
    cudaGetLastError();  // clear the error that the failed query recorded
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer ||
      !b.devicePointer)
    return nullptr;
  if (static_cast<const char *>(b.devicePointer) - static_cast<const char *>(a.devicePointer) !=
      (std::ptrdiff_t)(bytes - 1))
    return nullptr;
  return a.devicePointer;
}

int upload_fields(lbm_lattice *h, const double *rho, const double *T, cudaStream_t s) {
  const size_t n = (size_t)h->nx * h->ny;
  // page-locked host fields are read by the kernels directly
  const double *rho_src = static_cast<const double *>(mapped_host(rho, n * sizeof(double)));
  if (!rho_src) {
    LBM_CUDA(cudaMemcpyAsync(h->rho0, rho, n * sizeof(double), cudaMemcpyHostToDevice, s));
    rho_src = h->rho0;
  }
  LBM_CUDA(lbm::launch_init(h->dp, h->p.storage, rho_src, h->g[h->cur], s));
  if (T) {
    const double *T_src = static_cast<const double *>(mapped_host(T, n * sizeof(double)));
    if (!T_src) {
      LBM_CUDA(cudaMemcpyAsync(h->rho0, T, n * sizeof(double), cudaMemcpyHostToDevice, s));
      T_src = h->rho0;
    }
    LBM_CUDA(lbm::launch_pitch_T(T_src, h->nx, h->ny, h->pitch, h->T_ref, h->T[h->tcur], s));
  } else {
    LBM_CUDA(cudaMemsetAsync(h->T[h->tcur], 0, sizeof(float) * h->plane, s));
  }
  LBM_CUDA(cudaStreamSynchronize(s));
  return LBM_OK;
}

}  // namespace

extern "C" {

double lbm_critical_temperature(const lbm_params_t *p) {
  return p ? critical_temperature(*p) : 0.0;
}

int lbm_pressure_inlet_density(const lbm_params_t *p, long long t, double *rho) {
  if (!p || !rho) return LBM_ERR_ARG;
  if (!(p->eos_a > 0.0) || !(p->eos_b > 0.0) || !(p->eos_R > 0.0) || !(p->T_inlet > 0.0) ||
      !(p->rho_out > 0.0) || !(std::fabs(p->p_amp_frac) < 1.0) || p->u_period < 0.0)
    return LBM_ERR_ARG;
  const double Tc = critical_temperature(*p);
  *rho = inlet_density(*p, Tc, vapour_branch_end(*p, Tc, Tc * p->T_inlet), t);
  return LBM_OK;
}

const char *lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "out of memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_UNSTABLE: return "device status bits set (unstable or invalid state)";
    case LBM_ERR_TIMEOUT: return "timeout";
    case LBM_ERR_BUSY: return "admission refused";
    case LBM_ERR_STATE: return "malformed checkpoint";
    default: return "unknown error";
  }
}

int lbm_create(int nx, int ny, const lbm_params_t *p, lbm_h *out) {
  if (!p || !out) return LBM_ERR_ARG;
  *out = nullptr;
  int rc = validate(nx, ny, *p);
  if (rc) return rc;
  lbm_lattice *h = new (std::nothrow) lbm_lattice();
  if (!h) return LBM_ERR_OOM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return LBM_ERR_CUDA;
  }
  h->nx = nx;
  h->ny = ny;
  h->pitch = (nx + 31) / 32 * 32;
  h->plane = (long long)ny * h->pitch;
  h->p = *p;
  h->dp = derive(nx, ny, h->pitch, *p, h->Tc, h->T_ref, h->rho_ref);
  if (p->x_bc == LBM_X_PRESSURE_INLET)
    h->rho_branch_end = vapour_branch_end(*p, h->Tc, h->Tc * p->T_inlet);
  h->kernel = LBM_KERNEL_SPLIT;
  // The library's choice for the energy equation on lattices of at most 2^18 nodes is the
  // two-pass path: its halos are one row (collision) and four rows (energy update) where
  // the fused kernel's short row chunks on a small lattice spend most row steps filling
  // its six-stage pipeline (GB300: 200 x 50 9.6 against 11.1 us per update, 1024 x 256
  // 18.9 against 19.7 us; from 2048 x 256 on the fused kernel is faster).
  const bool auto_two = p->kernel == LBM_KERNEL_AUTO && p->thermal &&
                        (long long)nx * ny <= (1LL << 18) && lbm::fused_supported(h->dp);
  if (auto_two) {
    h->twopass = lbm::twopass_tiling(h->dp, p->storage, h->device);
    if (h->twopass.Ha > 0) h->kernel = LBM_KERNEL_TWOPASS;
  }
  if (p->kernel == LBM_KERNEL_TWOPASS) {
    // 32-bit element offsets, as on the fused path
    if (lbm::fused_supported(h->dp)) h->twopass = lbm::twopass_tiling(h->dp, p->storage, h->device);
    // LBM_TWOPASS_TILE="Ha,Hb" overrides the row-chunk heights (tuning experiments)
    if (const char *env = std::getenv("LBM_TWOPASS_TILE")) {
      int Ha = 0, Hb = 0;
      if (std::sscanf(env, "%d,%d", &Ha, &Hb) == 2 && Ha >= 1 && Hb >= 1 &&
          (ny + Ha - 1) / Ha <= 65535 && (ny + Hb - 1) / Hb <= 65535 && h->twopass.Ha > 0)
        h->twopass = lbm::TwoPassTiling{Ha, Hb};
    }
    if (h->twopass.Ha < 1) {
      delete h;
      return LBM_ERR_ARG;
    }
    h->kernel = LBM_KERNEL_TWOPASS;
  } else if (p->kernel != LBM_KERNEL_SPLIT && h->kernel != LBM_KERNEL_TWOPASS) {
    // lattice columns per thread of the fused kernel: as asked, else the library's
    // default, which LBM_FUSED_CPT=1|2 overrides (tuning experiments)
    int cpt = default_cpt(nx, ny);
    if (const char *env = std::getenv("LBM_FUSED_CPT")) {
      const int v = std::atoi(env);
      if (v == 1 || v == 2) cpt = v;
    }
    if (p->kernel == LBM_KERNEL_FUSED_1COL) cpt = 1;
    if (p->kernel == LBM_KERNEL_FUSED_2COL) cpt = 2;
    if (lbm::fused_supported(h->dp))
      h->fused = lbm::fused_tiling(h->dp, p->storage, h->device, cpt);
    // LBM_FUSED_TILE="W,H" overrides the tiling (tuning experiments)
    if (const char *env = std::getenv("LBM_FUSED_TILE")) {
      int W = 0, H = 0;
      if (std::sscanf(env, "%d,%d", &W, &H) == 2 && W >= 1 && W <= lbm::fused_max_width(cpt) &&
          H >= 1 && (ny + H - 1) / H <= 65535 && lbm::fused_supported(h->dp))
        h->fused = lbm::FusedTiling{W, H, cpt, 0};
    }
    if (h->fused.W > 0) {
      h->kernel = LBM_KERNEL_FUSED;
    } else if (p->kernel != LBM_KERNEL_AUTO) {
      delete h;
      return LBM_ERR_ARG;
    }
  }
  h->nblocks = lbm::mass_heat_blocks(h->dp);
  const size_t plane = (size_t)h->plane;
  cudaError_t e = cudaSuccess;
  h->esize = lbm::storage_bytes(p->storage);
  for (int k = 0; k < 2 && e == cudaSuccess; k++) {
    char *ptr = nullptr;
    e = dalloc(h, &ptr, 9 * plane * (size_t)h->esize);
    h->g[k] = ptr;
  }
  for (int k = 0; k < 2 && e == cudaSuccess; k++) e = dalloc(h, &h->T[k], plane);
  if (e == cudaSuccess) e = dalloc(h, &h->rho, plane);
  if (e == cudaSuccess) e = dalloc(h, &h->psi, plane);
  if (e == cudaSuccess) e = dalloc(h, &h->ux, plane);
  if (e == cudaSuccess) e = dalloc(h, &h->uy, plane);
  if (e == cudaSuccess) e = dalloc(h, &h->status, 1);
  if (e == cudaSuccess) e = dalloc(h, &h->partials, 2 * (size_t)h->nblocks);
  if (e == cudaSuccess) e = dalloc(h, &h->sums, 2);
  if (e == cudaSuccess) e = dalloc(h, &h->rho0, (size_t)nx * ny);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&h->host_sums, 2 * sizeof(double));
  if (h->kernel == LBM_KERNEL_FUSED || h->kernel == LBM_KERNEL_TWOPASS) {
    const int C = lbm_lattice::kChunk;
    if (e == cudaSuccess) e = dalloc(h, &h->d_sc, C);
    for (int k = 0; k < 2 && e == cudaSuccess; k++)
      e = cudaMallocHost((void **)&h->h_sc[k], C * sizeof(StepScalars));
    for (int k = 0; k < 2 && e == cudaSuccess; k++)
      e = cudaEventCreateWithFlags(&h->sc_ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(unsigned));
  // padding columns stay zero forever
  for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMemset(h->g[k], 0, 9 * plane * (size_t)h->esize);
  for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMemset(h->T[k], 0, plane * sizeof(float));
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return cuda_fail(e);
  }
  // rest equilibrium of rho_g, T = T0
  std::vector<double> r0((size_t)nx * ny, p->rho_g > 0.0 ? p->rho_g : h->rho_ref);
  rc = upload_fields(h, r0.data(), nullptr, 0);
  if (rc) {
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return LBM_OK;
}

void lbm_destroy(lbm_h h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
}

int lbm_write_fields(lbm_h h, const double *rho, const double *T, void *stream) {
  if (!h || !rho) return LBM_ERR_ARG;
  LBM_CUDA(cudaSetDevice(h->device));
  return upload_fields(h, rho, T, (cudaStream_t)stream);
}

int lbm_step(lbm_h h, long nsteps, void *stream) {
  if (!h || nsteps < 0) return LBM_ERR_ARG;
  LBM_CUDA(cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  // each call stages the boundary scalars of its own updates, so a captured call could
  // not be replayed; whole chunks are replayed from the handle's own graphs instead
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  LBM_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return LBM_ERR_ARG;
  if (h->kernel == LBM_KERNEL_FUSED || h->kernel == LBM_KERNEL_TWOPASS)
    return fused_steps(h, nsteps, s);
  for (long k = 0; k < nsteps; k++) {
    int rc = split_update(h, s);
    if (rc) return rc;
  }
  return LBM_OK;
}

int lbm_set_graph(lbm_h h, int enable) {
  if (!h) return LBM_ERR_ARG;
  h->use_graph = enable != 0;
  if (!h->use_graph) {
    LBM_CUDA(cudaSetDevice(h->device));
    drop_graphs(h);
  }
  return LBM_OK;
}

int lbm_status(lbm_h h, unsigned *bits, int clear, void *stream) {
  if (!h || !bits) return LBM_ERR_ARG;
  LBM_CUDA(cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  unsigned *hs = (unsigned *)h->host_sums;
  LBM_CUDA(cudaMemcpyAsync(hs, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  LBM_CUDA(cudaStreamSynchronize(s));
  *bits = *hs;
  if (clear) {
    LBM_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), s));
    LBM_CUDA(cudaStreamSynchronize(s));
  }
  return LBM_OK;
}

int lbm_read_fields(lbm_h h, double *rho, double *ux, double *uy, double *T, void *stream) {
  if (!h) return LBM_ERR_ARG;
  LBM_CUDA(cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  int rc = compute_rho_psi(h, s);
  if (rc) return rc;
  StepScalars sc = scalars_at(h, h->t);
  LBM_CUDA(lbm::launch_collide(h->dp, h->p.storage, h->g[h->cur], nullptr, h->T[h->tcur], h->psi,
                               h->ux, h->uy, h->status, sc, false, s));
  struct Out {
    double *dst;
    const float *src;
    double add;
  } outs[4] = {{rho, h->rho, 0.0}, {ux, h->ux, 0.0}, {uy, h->uy, 0.0}, {T, h->T[h->tcur], h->T_ref}};
  // each field is widened to FP64 in the caller's layout: straight into a page-locked
  // host buffer, else in the device staging array and copied out (the stream orders the
  // reuse of the array)
  const size_t n = (size_t)h->nx * h->ny;
  for (auto &o : outs) {
    if (!o.dst) continue;
    if (double *dst = static_cast<double *>(mapped_host(o.dst, n * sizeof(double)))) {
      LBM_CUDA(lbm::launch_unpitch(o.src, h->nx, h->ny, h->pitch, o.add, dst, s));
      continue;
    }
    LBM_CUDA(lbm::launch_unpitch(o.src, h->nx, h->ny, h->pitch, o.add, h->rho0, s));
    LBM_CUDA(cudaMemcpyAsync(o.dst, h->rho0, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  LBM_CUDA(cudaStreamSynchronize(s));
  unsigned bits = 0;
  rc = lbm_status(h, &bits, 0, stream);
  if (rc) return rc;
  return bits ? LBM_ERR_UNSTABLE : LBM_OK;
}

int lbm_reduce(lbm_h h, double *mass, double *heat, void *stream) {
  if (!h) return LBM_ERR_ARG;
  LBM_CUDA(cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  int rc = compute_rho_psi(h, s);
  if (rc) return rc;
  LBM_CUDA(lbm::launch_mass_heat(h->dp, h->rho, h->T[h->tcur], h->T_ref, h->p.Cv, h->partials,
                                 h->nblocks, h->sums, s));
  LBM_CUDA(cudaMemcpyAsync(h->host_sums, h->sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  LBM_CUDA(cudaStreamSynchronize(s));
  if (mass) *mass = h->host_sums[0];
  if (heat) *heat = h->host_sums[1];
  return LBM_OK;
}

int lbm_state_bytes(lbm_h h, size_t *bytes) {
  if (!h || !bytes) return LBM_ERR_ARG;
  *bytes = sizeof(StateHeader) + (size_t)h->plane * (9 * (size_t)h->esize + sizeof(float));
  return LBM_OK;
}

int lbm_read_state(lbm_h h, void *buf, size_t bytes, void *stream) {
  size_t need = 0;
  if (!h || !buf || lbm_state_bytes(h, &need) || bytes < need) return LBM_ERR_ARG;
  LBM_CUDA(cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  StateHeader hd{};
  hd.magic = kStateMagic;
  hd.version = kStateVersion;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.pitch = h->pitch;
  hd.storage = h->p.storage;
  hd.t = h->t;
  std::memcpy(buf, &hd, sizeof(hd));
  char *dst = (char *)buf + sizeof(hd);
  const size_t gbytes = (size_t)h->esize * 9 * h->plane;
  LBM_CUDA(cudaMemcpyAsync(dst, h->g[h->cur], gbytes, cudaMemcpyDeviceToHost, s));
  LBM_CUDA(cudaMemcpyAsync(dst + gbytes, h->T[h->tcur],
                           sizeof(float) * h->plane, cudaMemcpyDeviceToHost, s));
  LBM_CUDA(cudaStreamSynchronize(s));
  return LBM_OK;
}

int lbm_write_state(lbm_h h, const void *buf, size_t bytes, void *stream) {
  size_t need = 0;
  if (!h || !buf || lbm_state_bytes(h, &need)) return LBM_ERR_ARG;
  if (bytes < need) return LBM_ERR_STATE;
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kStateMagic || hd.version != kStateVersion || hd.nx != h->nx || hd.ny != h->ny ||
      hd.pitch != h->pitch || hd.storage != h->p.storage || hd.t < 0)
    return LBM_ERR_STATE;
  LBM_CUDA(cudaSetDevice(h->device));
  cudaStream_t s = (cudaStream_t)stream;
  const char *src = (const char *)buf + sizeof(hd);
  const size_t gbytes = (size_t)h->esize * 9 * h->plane;
  LBM_CUDA(cudaMemcpyAsync(h->g[h->cur], src, gbytes, cudaMemcpyHostToDevice, s));
  LBM_CUDA(cudaMemcpyAsync(h->T[h->tcur], src + gbytes,
                           sizeof(float) * h->plane, cudaMemcpyHostToDevice, s));
  LBM_CUDA(cudaStreamSynchronize(s));
  h->t = hd.t;
  return LBM_OK;
}

int lbm_info(lbm_h h, lbm_info_t *info) {
  if (!h || !info) return LBM_ERR_ARG;
  info->nx = h->nx;
  info->ny = h->ny;
  info->pitch = h->pitch;
  info->t = h->t;
  info->Tc = h->Tc;
  info->T_ref = h->T_ref;
  info->rho_ref = h->rho_ref;
  info->device_bytes = h->device_bytes;
  info->kernel = h->kernel;
  const bool fused = h->kernel == LBM_KERNEL_FUSED;
  const bool two = h->kernel == LBM_KERNEL_TWOPASS;
  info->tile_cols = fused ? h->fused.W : two ? lbm::twopass_width_a() : 0;
  info->tile_rows = fused ? h->fused.H : two ? h->twopass.Ha : 0;
  info->cols_per_thread = fused ? h->fused.cpt : two ? 1 : 0;
  return LBM_OK;
}

int lbm_timing_enable(lbm_h h, int enable) {
  if (!h) return LBM_ERR_ARG;
  h->timing = enable != 0;
  return LBM_OK;
}

int lbm_timing_get(lbm_h h, const char **names, double *total_ms, long *launches, int n,
                   int *count, void *stream) {
  if (!h || n < 0) return LBM_ERR_ARG;
  LBM_CUDA(cudaSetDevice(h->device));
  LBM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int rc = drain_timing(h);
  if (rc) return rc;
  int k = 0;
  for (int i = 0; i < KN_COUNT; i++) {
    if (h->launches[i] == 0) continue;
    if (k < n) {
      if (names) names[k] = kKernelNames[i];
      if (total_ms) total_ms[k] = h->total_ms[i];
      if (launches) launches[k] = h->launches[i];
    }
    k++;
  }
  if (count) *count = k;
  for (int i = 0; i < KN_COUNT; i++) {
    h->total_ms[i] = 0;
    h->launches[i] = 0;
  }
  return LBM_OK;
}

}  // extern "C"
