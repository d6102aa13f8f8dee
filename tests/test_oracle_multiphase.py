"""Pins of the oracle's multiphase behaviour (Eqs. 8-11, 14) against the Maxwell
construction, the Laplace law and the ordering of contact angles with wall
strength."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import maxwell
from paper_1803_01756_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def slab(ny, nx, rho_g, rho_l, lo, hi, width=3.0):
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    return rho_g + (rho_l - rho_g) * 0.5 * (np.tanh((y - lo) / width) - np.tanh((y - hi) / width))


def flat_coexistence(theta, steps=30000):
    p = inputs.base_params(theta=theta, thermal=0, x_bc=0, y_bc=0, Gw=0.0)
    o = oracle.Oracle(2, 200, p)
    o.set_fields(slab(200, 2, 0.38, 6.5, 50, 150))
    o.step(steps)
    rho = o.fields()[0]
    return rho[0, 0], rho[100, 0]


def test_stored_calibration_reproduces_maxwell():
    with open(os.path.join(HERE, "golden", "theta_calibration.json")) as fh:
        cal = json.load(fh)
    assert inputs.THETA == cal["theta"]
    rg, rl = flat_coexistence(cal["theta"], steps=30000)
    mg, ml, _ = maxwell.coexistence(inputs.base_params(), 0.86)
    assert rg == pytest.approx(mg, rel=2e-3)
    assert rl == pytest.approx(ml, rel=2e-4)


def test_theta_moves_coexistence_towards_maxwell():
    """Li's term (Eq. 8, reading: minus sign in the epsilon entry) raises the vapour
    density of the pseudopotential model towards the Maxwell value."""
    mg, _, _ = maxwell.coexistence(inputs.base_params(), 0.86)
    g0, _ = flat_coexistence(0.0, steps=20000)
    g1, _ = flat_coexistence(0.06, steps=20000)
    assert g0 < g1 < mg
    assert abs(g1 - mg) < abs(g0 - mg)


def droplet(n, R, rho_g, rho_l, cx, cy, width=2.0):
    y, x = np.mgrid[0:n[0], 0:n[1]].astype(float)
    r = np.hypot(x - cx, y - cy)
    return rho_g + (rho_l - rho_g) * 0.5 * (1 - np.tanh((r - R) / width))


@pytest.mark.slow
def test_laplace_law():
    """Static droplets in a periodic box: the pressure jump p_in - p_out, with
    p = rho/3 + G psi^2 / 2 (Eq. 10), is linear in 1/R through the origin region."""
    n = 64
    p = inputs.base_params(thermal=0, x_bc=0, y_bc=0)
    T = 0.86 * oracle.critical_temperature(p)
    inv_r, dp = [], []
    for R in (9, 11, 13, 16):
        o = oracle.Oracle(n, n, p)
        o.set_fields(droplet((n, n), R, inputs.RHO_V_086, inputs.RHO_L_086, n / 2 - 0.5,
                             n / 2 - 0.5))
        o.step(3000)
        rho = o.fields()[0]
        pr = lambda r: r / 3 + p["G"] * oracle.psi(p, r, T)[0] ** 2 / 2  # noqa: E731
        r_in, r_out = rho[n // 2, n // 2], rho[0, 0]
        # equimolar radius: the disc of density r_in holding the same excess mass
        R_e = np.sqrt((rho - r_out).sum() / (np.pi * (r_in - r_out)))
        inv_r.append(1 / R_e)
        dp.append(pr(r_in) - pr(r_out))
    inv_r, dp = np.array(inv_r), np.array(dp)
    A = np.vstack([inv_r, np.ones_like(inv_r)]).T
    coef, res, _, _ = np.linalg.lstsq(A, dp, rcond=None)
    pred = A @ coef
    r2 = 1 - ((dp - pred) ** 2).sum() / ((dp - dp.mean()) ** 2).sum()
    assert coef[0] > 0  # positive surface tension
    assert r2 >= 0.999, r2
    assert abs(coef[1]) < 0.1 * np.abs(dp).max()


def contact_angle(rho, rho_mid):
    """Sessile cap on the bottom wall: CA = 2 atan(2h / w) (reading R20) from the cap
    height h and the base width w with sub-cell interpolation."""
    row = rho[0]
    xs = np.where(row > rho_mid)[0]
    if xs.size == 0:
        return 180.0  # the drop has lifted off the wall
    if xs.size == row.size:
        return 0.0  # a film covers the wall
    x0, x1 = xs.min(), xs.max()
    left = x0 - (row[x0] - rho_mid) / (row[x0] - row[x0 - 1])
    right = x1 + (row[x1] - rho_mid) / (row[x1] - row[x1 + 1])
    w = right - left
    # height along the centre column (wall at y = -1/2)
    c = int(round(0.5 * (x0 + x1)))
    colv = rho[:, c]
    ys = np.where(colv > rho_mid)[0]
    y1 = ys.max()
    h = y1 + (colv[y1] - rho_mid) / (colv[y1] - colv[y1 + 1]) + 0.5
    return np.degrees(2 * np.arctan(2 * h / w))


@pytest.mark.slow
def test_contact_angle_increases_with_wall_strength():
    """Eq. 14 with s = 1 on wall sites and psi_w = local psi: a more repulsive wall
    (larger G_w) gives a larger contact angle, and the neutral 90 degrees lies
    between G_w = -1.2 and -1.1 at 0.86 Tc."""
    nx, ny = 80, 40
    angles = []
    for Gw in (-1.2, -1.15, -1.1):
        p = inputs.base_params(thermal=0, x_bc=0, y_bc=1, Gw=Gw)
        o = oracle.Oracle(nx, ny, p)
        o.set_fields(droplet((ny, nx), 14, inputs.RHO_V_086, inputs.RHO_L_086, nx / 2, -0.5))
        o.step(8000)
        rho = o.fields()[0]
        angles.append(contact_angle(rho, 0.5 * (inputs.RHO_V_086 + inputs.RHO_L_086)))
    assert angles[0] < angles[1] < angles[2], angles
    assert angles[0] < 90 < angles[2], angles


def test_contact_angle_table_literals_match_the_oracle_table():
    """The workload generator's G_w -> contact-angle literals are the oracle's table
    (tests/golden/contact_angle_table.json), monotone and spanning 45-135 degrees."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "contact_angle_table.json")) as fh:
        tab = json.load(fh)
    pairs = [(g, a) for g, a in zip(tab["Gw"], tab["angle_deg"]) if a < 179]
    assert list(inputs.CA_TABLE_GW) == pytest.approx([g for g, _ in pairs], abs=1e-12)
    assert list(inputs.CA_TABLE_DEG) == pytest.approx([a for _, a in pairs], abs=5e-4)
    assert all(np.diff(inputs.CA_TABLE_DEG) > 0)
    assert inputs.CA_TABLE_DEG[0] < 45 and inputs.CA_TABLE_DEG[-1] > 135
    # the table agrees with the ordering pin above: 90 degrees between -1.2 and -1.1
    assert -1.2 < inputs.wall_strength_for_angle(90.0) < -1.1
