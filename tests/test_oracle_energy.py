"""Pins of the oracle's energy equation (Eqs. 16-18): the isotropic stencils on
Fourier modes, K(T) on analytic fields, and the RK4 amplification factor."""
import numpy as np
import pytest

import oracle
from paper_1803_01756_gb300 import inputs


def grid(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    return x, y


@pytest.mark.parametrize("kx,ky", [(1, 0), (2, 3), (5, 1)])
def test_gradient_of_fourier_mode(kx, ky):
    nx, ny = 32, 24
    x, y = grid(nx, ny)
    a, b = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    phi = np.sin(a * x) * np.cos(b * y)
    gx, gy = oracle.grad_periodic(phi)
    # 3 sum_i w_i phi(x+e_i) e_i on this mode: the axis and diagonal terms combine to
    # sin(a) (2 + cos b)/3 for d/dx and -sin(b) (2 + cos a)/3 for d/dy
    np.testing.assert_allclose(gx, np.sin(a) * (2 + np.cos(b)) / 3 * np.cos(a * x) * np.cos(b * y),
                               atol=1e-14)
    np.testing.assert_allclose(gy, -np.sin(b) * (2 + np.cos(a)) / 3 * np.sin(a * x) * np.sin(b * y),
                               atol=1e-14)


@pytest.mark.parametrize("kx,ky", [(1, 0), (2, 3), (5, 1)])
def test_laplacian_of_fourier_mode(kx, ky):
    nx, ny = 32, 24
    x, y = grid(nx, ny)
    a, b = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    phi = np.sin(a * x) * np.sin(b * y)
    lap = oracle.lap_periodic(phi)
    eig = 6 * ((2 * np.cos(a) + 2 * np.cos(b) - 4) / 9 + (4 * np.cos(a) * np.cos(b) - 4) / 36)
    np.testing.assert_allclose(lap, eig * phi, atol=1e-14)
    # long-wave limit: the symbol tends to -(a^2 + b^2)
    assert eig == pytest.approx(-(a * a + b * b), rel=0.3)


def test_stencils_exact_on_low_polynomials_in_the_interior():
    # periodic wrap spoils polynomials only at the seam: check away from it
    nx, ny = 20, 20
    x, y = grid(nx, ny)
    phi = 0.3 * x - 0.7 * y + 0.05 * x * x + 0.02 * x * y - 0.03 * y * y
    gx, gy = oracle.grad_periodic(phi)
    lap = oracle.lap_periodic(phi)
    s = (slice(2, -2), slice(2, -2))
    np.testing.assert_allclose(gx[s], (0.3 + 0.1 * x + 0.02 * y)[s], atol=1e-12)
    np.testing.assert_allclose(gy[s], (-0.7 + 0.02 * x - 0.06 * y)[s], atol=1e-12)
    np.testing.assert_allclose(lap[s], 0.1 - 0.06, atol=1e-12)


def test_energy_rhs_on_analytic_fields():
    """K(T) of Eq. 16 on periodic Fourier fields, with the stencils' exact symbols
    and (dP/dT)_rho taken by finite differences of the EOS."""
    nx, ny = 24, 16
    p = inputs.base_params(x_bc=0, y_bc=0)
    o = oracle.Oracle(nx, ny, p)
    x, y = grid(nx, ny)
    ka, kb = 2 * np.pi * 2 / nx, 2 * np.pi * 1 / ny
    Tc = o.Tc
    T = Tc * (0.86 + 0.01 * np.sin(ka * x))
    rho = 0.5 + 0.1 * np.cos(kb * y)
    ux = 0.01 * np.cos(ka * x)
    uy = 0.02 * np.sin(kb * y)
    K = o.energy_rhs(rho, ux, uy, T)
    gradT_x = 0.01 * Tc * np.sin(ka) * np.cos(ka * x)
    lapT = 0.01 * Tc * (2 * np.cos(ka) - 2) * np.sin(ka * x)
    divu = -0.01 * np.sin(ka) * np.sin(ka * x) + 0.02 * np.sin(kb) * np.cos(kb * y)
    h = 1e-6 * Tc
    dPdT = np.vectorize(lambda r, t: (oracle.eos_pressure(p, r, t + h)
                                      - oracle.eos_pressure(p, r, t - h)) / (2 * h))(rho, T)
    rcv = rho * p["Cv"]
    expect = -ux * gradT_x + p["lambda"] * lapT / rcv - T * dPdT * divu / rcv
    np.testing.assert_allclose(K, expect, rtol=1e-7, atol=1e-12)


def test_uniform_temperature_at_rest_is_steady():
    p = inputs.base_params(x_bc=0, y_bc=0, multiphase=0)
    o = oracle.Oracle(12, 10, p)
    o.set_fields(np.full((10, 12), 0.5))
    o.step(20)
    rho, ux, uy, T = o.fields()
    assert np.abs(ux).max() == 0 and np.abs(uy).max() == 0
    np.testing.assert_allclose(T, 0.86 * o.Tc, rtol=1e-15)


def test_rk4_amplification_of_a_diffusion_mode():
    """With u = 0 the update is T <- T + (h1 + 2 h2 + 2 h3 + h4)/6 with K linear:
    a Fourier mode is multiplied by 1 + z + z^2/2 + z^3/6 + z^4/24 per step, where
    z = lambda/(rho Cv) times the Laplacian symbol (fixes the RK4 weights, Eq. 17)."""
    nx, ny, steps = 16, 4, 10
    p = inputs.base_params(x_bc=0, y_bc=0, multiphase=0, **{"lambda": 0.6})
    o = oracle.Oracle(nx, ny, p)
    x, _ = grid(nx, ny)
    k = 2 * np.pi / nx
    rho = 0.5
    T0 = 0.86 * o.Tc
    eps = 1e-3 * T0
    o.set_fields(np.full((ny, nx), rho), T0 + eps * np.sin(k * x))
    o.step(steps)
    T = o.fields()[3]
    z = p["lambda"] / (rho * p["Cv"]) * (2 * np.cos(k) - 2)
    R = 1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24
    np.testing.assert_allclose(T - T0, eps * R**steps * np.sin(k * x), rtol=0, atol=1e-9 * eps)
