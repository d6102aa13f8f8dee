"""Pins of the oracle's thermal wall conditions (Section 3.2: an isothermal cold
segment of the top wall with adiabatic parts beside it, an isothermal bottom wall).

On a fluid at rest (uniform density, no force, so u stays exactly zero) the energy
equation reduces to conduction, lambda lap T / (rho Cv), for which:
  - with both walls adiabatic the discrete heat content sum T is conserved exactly
    (each interior pair of the 9-point Laplacian cancels, and a mirrored ghost row
    contributes nothing across the wall);
  - with two isothermal walls the steady state is the linear profile through the
    ghost rows, T(y) = T_b + (T_t - T_b) (y + 1) / (ny + 1), since linear functions
    are harmonic for the 9-point stencil;
  - with an isothermal bottom and an adiabatic top the steady state is uniform T_b.
"""
import numpy as np
import pytest

import oracle
from paper_1803_01756_gb300 import inputs


def conduction_params(**over):
    p = inputs.base_params(x_bc=oracle.X_PERIODIC, y_bc=oracle.Y_WALLS, multiphase=0,
                           thermal=1, u_amp=0.0, rho_g=1.0, rho_out=1.0, T0=0.86,
                           T_wall_left=0.86, T_wall_right=0.86)
    p.update(over)
    return p


def run(nx, ny, p, T, steps):
    o = oracle.Oracle(nx, ny, p)
    o.set_fields(np.ones((ny, nx)), T)
    o.step(steps)
    return o


def bump(nx, ny, Tc, amp=0.02):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    return Tc * (0.86 + amp * np.exp(-((x - nx / 3) ** 2 + (y - ny / 4) ** 2) / 8.0))


def test_adiabatic_walls_conserve_heat_exactly():
    nx, ny = 24, 14
    # isothermal windows outside the lattice: both walls adiabatic on every column
    p = conduction_params(top_iso_x0=nx, top_iso_x1=nx + 1, bot_iso_x0=nx, bot_iso_x1=nx + 1,
                          T_wall_left=0.5, T_wall_right=0.5)
    Tc = oracle.critical_temperature(p)
    T0 = bump(nx, ny, Tc)
    o = run(nx, ny, p, T0, 300)
    rho, ux, uy, T = o.fields()
    assert np.abs(ux).max() == 0.0 and np.abs(uy).max() == 0.0
    assert T.sum() == pytest.approx(T0.sum(), rel=1e-13)
    assert np.abs(T - T0).max() > 1e-3 * Tc  # the bump did spread
    # the same lattice with isothermal walls at a colder temperature loses heat
    p_iso = conduction_params(T_wall_left=0.5, T_wall_right=0.5)
    T_iso = run(nx, ny, p_iso, T0, 300).fields()[3]
    assert T_iso.sum() < T0.sum() * (1 - 1e-4)


def test_two_isothermal_walls_give_the_linear_profile():
    nx, ny = 4, 12
    p = conduction_params(T_wall_left=0.90, T_wall_right=0.90, T_top_left=0.80,
                          T_top_right=0.80)
    Tc = oracle.critical_temperature(p)
    o = run(nx, ny, p, np.full((ny, nx), 0.86 * Tc), 12000)
    T = o.fields()[3] / Tc
    y = np.arange(ny)
    expect = 0.90 + (0.80 - 0.90) * (y + 1) / (ny + 1)
    np.testing.assert_allclose(T, np.repeat(expect[:, None], nx, axis=1), atol=1e-9)


def test_adiabatic_top_relaxes_to_the_bottom_temperature():
    # the slowest mode is a quarter wave over ny + 1 rows: 6 rows relax in ~400 steps
    nx, ny = 4, 6
    p = conduction_params(T_wall_left=0.90, T_wall_right=0.90, T_top_left=0.60,
                          T_top_right=0.60, top_iso_x0=nx, top_iso_x1=nx + 1)
    Tc = oracle.critical_temperature(p)
    o = run(nx, ny, p, np.full((ny, nx), 0.86 * Tc), 12000)
    np.testing.assert_allclose(o.fields()[3] / Tc, 0.90, atol=1e-9)


def test_isothermal_window_sets_which_columns_feel_the_cold_wall():
    """Top wall cold only on columns [8, 16) and adiabatic elsewhere: the columns
    under the window end colder than the adiabatic ones, symmetrically about the
    window's centre (periodic x)."""
    nx, ny = 24, 10
    p = conduction_params(T_top_left=0.70, T_top_right=0.70, top_iso_x0=8, top_iso_x1=16)
    Tc = oracle.critical_temperature(p)
    T = run(nx, ny, p, np.full((ny, nx), 0.86 * Tc), 400).fields()[3]
    top = T[-1] / Tc
    assert top[8:16].max() < top[:6].min() - 1e-3
    # mirror symmetry about x = 11.5 (column k <-> 23 - k)
    np.testing.assert_allclose(top, top[::-1], atol=1e-12)


def test_adiabatic_columns_never_read_the_wall_temperature():
    nx, ny = 16, 8
    Tc = oracle.critical_temperature(conduction_params())
    T0 = bump(nx, ny, Tc)
    kw = dict(top_iso_x0=nx, top_iso_x1=nx + 1)
    a = run(nx, ny, conduction_params(T_top_left=0.70, T_top_right=0.70, **kw), T0, 100)
    b = run(nx, ny, conduction_params(T_top_left=0.30, T_top_right=1.20, **kw), T0, 100)
    np.testing.assert_array_equal(a.fields()[3], b.fields()[3])
