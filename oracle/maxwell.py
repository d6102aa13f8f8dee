"""Coexistence densities of the Peng-Robinson EOS (Eq. 11) by the Maxwell
equal-area construction.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The construction uses
the oracle's own pressure function; scipy's root finder and quadrature are the
library primitives.

For a given temperature the saturation pressure P_s is the value for which the
vapour root rho_g and liquid root rho_l of P(rho) = P_s satisfy the equal-area
rule in specific volume v = 1/rho:

    int_{v_l}^{v_g} (P(v) - P_s) dv = 0  <=>  int_{rho_g}^{rho_l} (P(rho) - P_s) / rho^2 drho = 0.
"""
from __future__ import annotations

from scipy import integrate, optimize

from . import critical_temperature, eos_pressure


def spinodals(params: dict, T: float, rho_max: float | None = None):
    """Densities where dP/drho = 0 (local max of P at the vapour spinodal, local min
    at the liquid spinodal)."""
    b = params["eos_b"]
    if rho_max is None:
        rho_max = 0.999 / b

    def dP(r, h=1e-6):
        return (eos_pressure(params, r + h, T) - eos_pressure(params, r - h, T)) / (2 * h)

    # scan for the two sign changes of dP/drho
    n = 4000
    grid = [1e-4 + (rho_max - 1e-4) * k / n for k in range(n + 1)]
    vals = [dP(r) for r in grid]
    roots = []
    for k in range(n):
        if vals[k] == 0 or vals[k] * vals[k + 1] < 0:
            roots.append(optimize.brentq(dP, grid[k], grid[k + 1], xtol=1e-14))
    if len(roots) < 2:
        raise ValueError("no two-phase region at this temperature")
    return roots[0], roots[1]


def coexistence(params: dict, T_over_Tc: float):
    """Return (rho_g, rho_l, P_sat) at T = T_over_Tc * Tc."""
    T = T_over_Tc * critical_temperature(params)
    sv, sl = spinodals(params, T)
    Pmax = eos_pressure(params, sv, T)  # local maximum (vapour spinodal)
    Pmin = max(eos_pressure(params, sl, T), 1e-12 * Pmax)  # local minimum (liquid spinodal)
    rho_hi = 0.999 / params["eos_b"]

    def roots(Ps):
        rg = optimize.brentq(lambda r: eos_pressure(params, r, T) - Ps, 0.0, sv, xtol=1e-15)
        rl = optimize.brentq(lambda r: eos_pressure(params, r, T) - Ps, sl, rho_hi, xtol=1e-15)
        return rg, rl

    def area(Ps):
        rg, rl = roots(Ps)
        val, _ = integrate.quad(lambda r: (eos_pressure(params, r, T) - Ps) / (r * r), rg, rl,
                                epsabs=1e-14, epsrel=1e-12, limit=200)
        return val

    lo, hi = Pmin * (1 + 1e-12), Pmax * (1 - 1e-12)
    Ps = optimize.brentq(area, lo, hi, xtol=1e-16, rtol=1e-14)
    rg, rl = roots(Ps)
    return rg, rl, Ps
