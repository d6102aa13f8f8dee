"""Write theta_calibration.json: the Li forcing constant theta of Eq. 8 chosen so
that a flat liquid slab at 0.86 Tc coexists with its vapour at the Maxwell
densities of the Peng-Robinson EOS.  Calls only the FP64 oracle.

Recipe: periodic 2 x 200 lattice, isothermal (thermal off), liquid slab between
y = 50 and y = 150 with tanh edges of width 3 (a sharp step excites a
non-decaying checkerboard mode), run until rho at the slab centre and in the
vapour change by less than 1e-9 per 1000 steps; bisect theta on the vapour
density.  Run from the repository root:  python tests/golden/make_theta_calibration.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

import oracle  # noqa: E402
from oracle import maxwell  # noqa: E402

NX, NY = 2, 200
PARAMS = dict(
    eos_a=2.0 / 49.0, eos_b=2.0 / 21.0, eos_R=1.0, eos_omega=0.344, G=-1.0, Gw=0.0,
    rho_w=0.0, tau_g=1.0, tau_l=1.0, rho_g=0.38, rho_l=6.5, s_e=0.8, s_zeta=0.8, s_q=1.1,
    Cv=5.0, gx=0.0, gy=0.0, g_omega=0.0, T0=0.86, T_wall_left=0.86, T_wall_right=0.86,
    T_inlet=0.86, x_bc=0, y_bc=0, u_amp=0.0, u_period=0.0, rho_out=0.38, thermal=0,
    multiphase=1, **{"lambda": 0.25})


def slab_profile(rho_g=0.38, rho_l=6.5):
    y = np.arange(NY, dtype=np.float64)[:, None] * np.ones((1, NX))
    return rho_g + (rho_l - rho_g) * 0.5 * (np.tanh((y - 50) / 3.0) - np.tanh((y - 150) / 3.0))


def coexistence_run(theta: float, max_steps: int = 80000):
    p = dict(PARAMS, theta=theta)
    o = oracle.Oracle(NX, NY, p)
    o.set_fields(slab_profile())
    prev = None
    while o.t < max_steps:
        o.step(1000)
        rho = o.fields()[0]
        cur = (rho[100, 0], rho[0, 0])
        if prev is not None and abs(cur[0] - prev[0]) < 1e-9 and abs(cur[1] - prev[1]) < 1e-9:
            break
        prev = cur
    return cur[1], cur[0], o.t


def main():
    rho_g_mx, rho_l_mx, _ = maxwell.coexistence(PARAMS, 0.86)
    lo, hi = 0.09, 0.13
    glo = coexistence_run(lo)[0] - rho_g_mx
    ghi = coexistence_run(hi)[0] - rho_g_mx
    assert glo < 0 < ghi, (glo, ghi)
    while hi - lo > 2e-4:
        mid = 0.5 * (lo + hi)
        g = coexistence_run(mid)[0] - rho_g_mx
        if g < 0:
            lo = mid
        else:
            hi = mid
    theta = round(0.5 * (lo + hi), 4)
    rg, rl, steps = coexistence_run(theta)
    out = dict(
        theta=theta, T_over_Tc=0.86, rho_g_flat=rg, rho_l_flat=rl, steps=steps,
        rho_g_maxwell=rho_g_mx, rho_l_maxwell=rho_l_mx,
        lattice=[NX, NY], s_e=PARAMS["s_e"], s_zeta=PARAMS["s_zeta"],
        recipe=__doc__.strip().splitlines()[0],
    )
    path = os.path.join(os.path.dirname(__file__), "theta_calibration.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
