"""Pins of the oracle's moment-space algebra (Eqs. 2, 6-8, 13) against
identities that the D2Q9 lattice and the MRT method fix."""
import numpy as np
import pytest

import oracle

# D2Q9 velocities (Eq. 2) and the second-order equilibrium weights, written out
# here independently of the oracle
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def textbook_feq(rho, u):
    eu = E @ u
    return W * rho * (1 + 3 * eu + 4.5 * eu**2 - 1.5 * (u @ u))


def guo_source(u, F):
    """Guo's discrete forcing without the (1 - 1/2tau) factor: w_i [3(e_i - u) + 9 (e_i.u) e_i].F"""
    eu = E @ u
    return W * (3 * ((E - u) @ F) + 9 * eu * (E @ F))


def test_transform_rows_are_orthogonal():
    M = oracle.moment_matrix()
    G = M @ M.T
    assert np.array_equal(G, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]))


def test_transform_rows_are_velocity_polynomials():
    # rows of Eq. 6 are polynomials of e: 1, e(energy), eps, jx, qx, jy, qy, pxx, pxy
    M = oracle.moment_matrix()
    ex, ey = E[:, 0], E[:, 1]
    c2 = ex**2 + ey**2
    rows = [np.ones(9), 3 * c2 - 4, (9 * c2**2 - 21 * c2 + 8) / 2, ex, (3 * c2 - 5) * ex, ey,
            (3 * c2 - 5) * ey, ex**2 - ey**2, ex * ey]
    for r, ref in enumerate(rows):
        assert np.array_equal(M[r], ref.astype(np.int64)), r


@pytest.mark.parametrize("seed", range(5))
def test_meq_is_transform_of_second_order_equilibrium(seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 8.0)
    u = rng.uniform(-0.1, 0.1, 2)
    M = oracle.moment_matrix()
    np.testing.assert_allclose(oracle.meq(rho, *u), M @ textbook_feq(rho, u), rtol=0,
                               atol=1e-13 * rho)
    np.testing.assert_allclose(oracle.feq(rho, *u), textbook_feq(rho, u), rtol=1e-14, atol=0)


@pytest.mark.parametrize("seed", range(5))
def test_forcing_moments_are_transform_of_guo_source(seed):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-0.1, 0.1, 2)
    F = rng.uniform(-0.01, 0.01, 2)
    M = oracle.moment_matrix()
    np.testing.assert_allclose(oracle.forcing_moments(*u, *F), M @ guo_source(u, F), rtol=0,
                               atol=1e-15)


def test_theta_term_enters_energy_moments_with_opposite_signs():
    base = oracle.forcing_moments(0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.8, 0.8)
    with_theta = oracle.forcing_moments(0.0, 0.0, 0.0, 0.0, 0.5, 0.1, 0.8, 0.8)
    d = with_theta - base
    # 12 theta |F_m|^2 / psi^2 / (tau - 1/2) with tau = 1.25
    assert d[1] == pytest.approx(12 * 0.1 * 0.5 / 0.75, rel=1e-14)
    assert d[2] == pytest.approx(-12 * 0.1 * 0.5 / 0.75, rel=1e-14)
    assert np.all(d[[0, 3, 4, 5, 6, 7, 8]] == 0)


PARAMS = dict(eos_a=2 / 49, eos_b=2 / 21, eos_R=1.0, eos_omega=0.344, G=-1.0, theta=0.11,
              tau_g=1.0, tau_l=1.0, rho_g=0.38, rho_l=6.5, s_e=0.8, s_zeta=0.8, s_q=1.1)


@pytest.mark.parametrize("seed", range(5))
def test_collision_conserves_mass_and_adds_the_force(seed):
    rng = np.random.default_rng(seed)
    f = textbook_feq(rng.uniform(0.2, 7), rng.uniform(-0.05, 0.05, 2)) * rng.uniform(0.9, 1.1, 9)
    F = rng.uniform(-0.01, 0.01, 2)
    fs = oracle.collide_node(PARAMS, f, *F, Fm2_over_psi2=rng.uniform(0, 0.1))
    assert fs.sum() == pytest.approx(f.sum(), rel=1e-14)
    np.testing.assert_allclose(E.T @ fs, E.T @ f + F, rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_equilibrium_is_a_fixed_point_without_force(seed):
    rng = np.random.default_rng(seed)
    f = textbook_feq(rng.uniform(0.2, 7), rng.uniform(-0.05, 0.05, 2))
    np.testing.assert_allclose(oracle.collide_node(PARAMS, f, 0.0, 0.0), f, rtol=0, atol=1e-14)


@pytest.mark.parametrize("k,rate", [(1, 0.8), (2, 0.8), (4, 1.1), (6, 1.1), (7, 1.0), (8, 1.0)])
def test_each_moment_relaxes_at_its_own_rate(k, rate):
    """m* - m^eq = (1 - s_k)(m - m^eq) moment by moment (Eq. 7 with Eq. 3 rates)."""
    M = oracle.moment_matrix().astype(float)
    rho, u = 0.9, np.array([0.02, -0.01])
    feq = textbook_feq(rho, u)
    dm = np.zeros(9)
    dm[k] = 1e-3
    f = feq + np.linalg.solve(M, dm)
    fs = oracle.collide_node(PARAMS, f, 0.0, 0.0)
    dms = M @ fs - M @ feq
    expect = np.zeros(9)
    expect[k] = (1 - rate) * 1e-3
    np.testing.assert_allclose(dms, expect, rtol=0, atol=1e-15)


def test_variable_viscosity_rate_follows_eq5():
    """s_7 = s_8 = 1 / tau_nu with tau_nu linear in the liquid fraction (Eq. 5 reading)."""
    p = dict(PARAMS, tau_g=1.0, tau_l=0.8)
    M = oracle.moment_matrix().astype(float)
    for rho, frac in [(0.38, 0.0), (3.44, 0.5), (6.5, 1.0), (8.0, 1.0), (0.2, 0.0)]:
        feq = textbook_feq(rho, np.zeros(2))
        dm = np.zeros(9)
        dm[7] = 1e-3
        fs = oracle.collide_node(p, feq + np.linalg.solve(M, dm), 0.0, 0.0)
        tau = 1.0 + frac * (0.8 - 1.0)
        assert (M @ fs)[7] - (M @ feq)[7] == pytest.approx((1 - 1 / tau) * 1e-3, abs=1e-15)
