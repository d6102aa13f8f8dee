"""Pins of the oracle's boundary rules of the energy equation (Eq. 16 with the
walls, inlet and outlet of Sections 3.2-3.3) and of the Zou-He corner nodes.

The ghost values that the nine-point stencils of Eq. 16 read outside the fluid
are fixed by the readings of the boundaries:
  - wall rows: velocity 0; temperature the wall's linear profile at the wall
    site's column (clamped to [0, nx - 1] at the open ends);
  - the inlet column x = -1: velocity (u_in(t), 0) for the velocity inlet at the
    lattice's time t, a copy of column 0 for the pressure inlet; temperature T_inlet;
  - the outlet column x = nx: copies of column nx - 1;
  - wall rows take precedence at the corners.
On linear fields every stencil value then has a short closed form, derived by
hand below node class by node class (interior, wall rows, inlet and outlet
columns, the four corners).  The oracle exposes K(T) of Eq. 16 only, so each pin
isolates one term: a uniform temperature equal to every ghost temperature leaves
the div u term alone; a fluid at rest leaves the Laplacian alone; uniform velocity
with a copying inlet leaves advection plus the Laplacian.

Zou-He corners (reading: bounce-back first, then the force-free Zou-He formulas
for the unknowns that enter from outside the x range through fluid rows): the
Zou-He rule sets three unknowns so that sum f = rho_b, j_x = rho_b U and j_y = 0.
At a corner one of the three is a bounce-back value instead, which shifts the
three moments by that population's excess delta times (1, e_x, e_y).  So at each
corner  sum f - rho_b = delta,  j_x - rho_b U = e_x delta,  j_y = e_y delta,
with rho_b and U from the known populations by the mass-flux identity.
"""
import numpy as np
import pytest

import oracle
from paper_1803_01756_gb300 import inputs

NX, NY = 9, 7
RHO = 0.5


def dpdt(p, rho, T):
    """(dP/dT)_rho of the oracle (pinned against finite differences of Eq. 11 in
    test_oracle_eos), so that the div u term can be divided out to round-off."""
    return oracle.eos_dpdt(p, rho, T)


def lattice_at_time(p, t):
    """An oracle lattice whose clock reads t (its state is not used by the pins)."""
    o = oracle.Oracle(NX, NY, p)
    o.set_fields(np.full((NY, NX), inputs.RHO_V_086))
    o.step(t)
    assert o.t == t
    return o


def divergence_from_K(o, p, ux, uy, T0):
    """Run K(T) with a temperature equal to every ghost temperature: grad T and
    lap T vanish, so K = -T (dP/dT) div u / (rho Cv) gives div u back."""
    rho = np.full((NY, NX), RHO)
    T = np.full((NY, NX), T0)
    K = o.energy_rhs(rho, ux, uy, T)
    return -K * RHO * p["Cv"] / (T0 * dpdt(p, RHO, T0))


def velocity_inlet_divergence(b, e, v, u_in):
    """Closed forms of 3 sum_i w_i u(x+e_i).e_i for u = (b x + e, v) in the fluid,
    velocity inlet ghost (u_in, 0), zero-velocity walls, copying outlet."""
    d = np.zeros((NY, NX))
    # x part: interior b; the wall rows lose their two solid diagonals (b/6 of 3*2b/36)
    d[1:-1, 1:-1] += b
    d[[0, -1], 1:-1] += 5 * b / 6
    # inlet column: (u(1) - u_in)/2, at the corners 3 (1/9 + 1/36) (u(1) - u_in)
    u1 = b + e
    d[1:-1, 0] += (u1 - u_in) / 2
    d[[0, -1], 0] += 5 * (u1 - u_in) / 12
    # outlet column copies itself: (u(nx-1) - u(nx-2))/2, corners 5 b / 12
    d[1:-1, -1] += b / 2
    d[[0, -1], -1] += 5 * b / 12
    # y part: zero inside; bottom wall row +v/2, top -v/2 (3 (1/9 + 2/36) v); at the
    # inlet corners the inlet ghost diagonal carries u_y = 0: 3 (1/9 + 1/36) v
    d[0, 1:] += v / 2
    d[-1, 1:] -= v / 2
    d[0, 0] += 5 * v / 12
    d[-1, 0] -= 5 * v / 12
    return d


@pytest.mark.parametrize("t", [7, 8, 23])
def test_divergence_with_velocity_inlet_walls_and_outlet(t):
    """ghost_u (inlet velocity at the lattice's own time t, zero at walls, copy at the
    outlet) and the divergence stencil, on u = (b x + e, v); a time level off by one
    step, a dropped wall zero or a wrong outlet copy changes a boundary class."""
    period, amp = 40.0, 0.03
    T0 = 0.86
    p = inputs.base_params(multiphase=0, u_amp=amp, u_period=period, T0=T0, T_inlet=T0,
                           T_wall_left=T0, T_wall_right=T0)
    o = lattice_at_time(p, t)
    Tabs = T0 * o.Tc
    x = np.arange(NX)[None, :].repeat(NY, 0).astype(float)
    b, e, v = 2e-3, 5e-3, -4e-3
    ux, uy = b * x + e, np.full((NY, NX), v)
    got = divergence_from_K(o, p, ux, uy, Tabs)
    u_in = amp * np.sin(2 * np.pi * t / period)
    expect = velocity_inlet_divergence(b, e, v, u_in)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-13)
    # the inlet column really depends on the time level
    other = velocity_inlet_divergence(b, e, v, amp * np.sin(2 * np.pi * (t + 1) / period))
    assert np.abs(other[:, 0] - expect[:, 0]).max() > 1e-5


def test_divergence_with_pressure_inlet_copies_column_zero():
    """With the pressure inlet the ghost velocity copies column 0: on u = (b x + e, v)
    the inlet column sees (u(1) - u(0))/2 = b/2 (5 b/12 at the corners) whatever e, and
    its corner diagonals carry v, so the wall rows give +-v/2 up to the inlet."""
    T0 = 0.86
    p = inputs.base_params(multiphase=0, x_bc=2, p_amp_frac=0.1, u_period=40.0, T0=T0,
                           T_inlet=T0, T_wall_left=T0, T_wall_right=T0)
    o = lattice_at_time(p, 5)
    x = np.arange(NX)[None, :].repeat(NY, 0).astype(float)
    b, e, v = 2e-3, 5e-3, -4e-3
    got = divergence_from_K(o, p, b * x + e, np.full((NY, NX), v), T0 * o.Tc)
    expect = np.zeros((NY, NX))
    expect[1:-1, 1:-1] = b
    expect[[0, -1], 1:-1] = 5 * b / 6
    expect[1:-1, [0, -1]] = b / 2
    expect[[0, -1], 0] = 5 * b / 12
    expect[[0, -1], -1] = 5 * b / 12
    expect[0, :] += v / 2
    expect[-1, :] -= v / 2
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-13)


def lap_at(vals, c):
    """6 sum_i w_i (T_i - T_c) for neighbour values listed in D2Q9 order 1..8."""
    w = [1 / 9] * 4 + [1 / 36] * 4
    return 6 * sum(wi * (vi - c) for wi, vi in zip(w, vals))


def test_temperature_ghosts_of_walls_inlet_and_outlet():
    """ghost_T on a fluid at rest (K = lambda lap T / (rho Cv)) with T = T0 + c x, the
    bottom wall at T0 + db + c x, the top wall at its own profile T0 + dt + c' x and an
    inlet temperature T0 + di.  Closed forms: lap = 0 inside; db and dt + (c' - c) x on
    the wall rows; c + di on the inlet column; -c on the outlet column; the corners
    from their neighbour lists (walls win at corners, wall columns clamp)."""
    Tc = oracle.critical_temperature(inputs.base_params())
    T0, c, db, dt, c2, di = 0.86 * Tc, 1e-4, -3e-3, 2e-3, 3e-4, 5e-3
    Tw = lambda x: T0 + db + c * x  # noqa: E731
    Tt = lambda x: T0 + dt + c2 * x  # noqa: E731
    p = inputs.base_params(multiphase=0, u_amp=0.0, T0=0.86, T_inlet=(T0 + di) / Tc,
                           T_wall_left=Tw(0) / Tc, T_wall_right=Tw(NX - 1) / Tc,
                           T_top_left=Tt(0) / Tc, T_top_right=Tt(NX - 1) / Tc)
    o = lattice_at_time(p, 3)
    x = np.arange(NX)[None, :].repeat(NY, 0).astype(float)
    T = T0 + c * x
    zero = np.zeros((NY, NX))
    K = o.energy_rhs(np.full((NY, NX), RHO), zero, zero, T)
    got = K * RHO * p["Cv"] / p["lambda"]

    expect = np.zeros((NY, NX))
    xs = np.arange(1, NX - 1)
    expect[0, 1:-1] = db                              # Tw(x) - T(x)
    expect[-1, 1:-1] = dt + (c2 - c) * xs             # Tt(x) - T(x)
    expect[1:-1, 0] = c + di                          # T(1) + T_in - 2 T(0)
    expect[1:-1, -1] = -c                             # T(nx-2) - T(nx-1)
    Tin, e = T0 + di, NX - 1
    Te = T0 + c * e
    # neighbours in the order e_1..e_8 = (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
    expect[0, 0] = lap_at([T0 + c, T0, Tin, Tw(0), T0 + c, Tin, Tw(0), Tw(1)], T0)
    expect[-1, 0] = lap_at([T0 + c, Tt(0), Tin, T0, Tt(1), Tt(0), Tin, T0 + c], T0)
    expect[0, -1] = lap_at([Te, Te, Te - c, Tw(e), Te, Te - c, Tw(e - 1), Tw(e)], Te)
    expect[-1, -1] = lap_at([Te, Tt(e), Te - c, Te, Tt(e), Tt(e - 1), Te - c, Te], Te)
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-13)


def test_temperature_gradient_ghosts_under_uniform_flow():
    """-u.grad T on the same ghosts: uniform u = (U, V) with the pressure inlet (its
    ghost copies the velocity, so div u is +-V/2 on the wall rows only), T = T0 + c x,
    walls offset by db (bottom) and dt (top), inlet T0 + di.  Closed forms of the
    gradient: (c, 0) inside; (c, -db/2) bottom, (c, dt/2) top rows; x part
    (T(1) - T_in)/2 on the inlet column, c/2 on the outlet column."""
    Tc = oracle.critical_temperature(inputs.base_params())
    T0, c, db, dt, di = 0.86 * Tc, 1e-4, -3e-3, 2e-3, 5e-3
    U, V = 0.02, -0.01
    p = inputs.base_params(multiphase=0, x_bc=2, p_amp_frac=0.1, u_period=40.0, T0=0.86,
                           T_inlet=(T0 + di) / Tc,
                           T_wall_left=(T0 + db) / Tc, T_wall_right=(T0 + db + c * (NX - 1)) / Tc,
                           T_top_left=(T0 + dt) / Tc, T_top_right=(T0 + dt + c * (NX - 1)) / Tc)
    o = lattice_at_time(p, 2)
    x = np.arange(NX)[None, :].repeat(NY, 0).astype(float)
    T = T0 + c * x
    rho = np.full((NY, NX), RHO)
    K = o.energy_rhs(rho, np.full((NY, NX), U), np.full((NY, NX), V), T)

    gx = np.full((NY, NX), c)
    gy = np.zeros((NY, NX))
    lap = np.zeros((NY, NX))
    div = np.zeros((NY, NX))
    gy[0, 1:-1], lap[0, 1:-1] = -db / 2, db
    gy[-1, 1:-1], lap[-1, 1:-1] = dt / 2, dt
    gx[1:-1, 0] = (c - di) / 2
    lap[1:-1, 0] = c + di
    gx[1:-1, -1], lap[1:-1, -1] = c / 2, -c
    div[0, :], div[-1, :] = V / 2, -V / 2
    core = (slice(1, -1), slice(None))
    rcv = RHO * p["Cv"]
    dP = np.vectorize(lambda tt: dpdt(p, RHO, tt))(T)
    expect = -(U * gx + V * gy) + p["lambda"] * lap / rcv - T * dP * div / rcv
    # the rows and columns with closed forms above (the corners are covered by the
    # two pins before this one)
    np.testing.assert_allclose(K[core], expect[core], rtol=0, atol=1e-13)
    np.testing.assert_allclose(K[[0, -1], 1:-1], expect[[0, -1], 1:-1], rtol=0, atol=1e-15)


def moments(f):
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    return f.sum(0), np.tensordot(ex, f, 1), np.tensordot(ey, f, 1)


@pytest.mark.parametrize("x_bc", [1, 2])
@pytest.mark.parametrize("multiphase", [0, 1])
def test_zou_he_corner_nodes(x_bc, multiphase):
    nx, ny, t = 24, 10, 37
    period, amp = 30.0, 0.03
    p = inputs.base_params(multiphase=multiphase, thermal=0, x_bc=x_bc, u_amp=amp,
                           u_period=period, p_amp_frac=0.1, rho_out=inputs.RHO_V_086)
    o = oracle.Oracle(nx, ny, p)
    o.set_fields(inputs.noisy_density(nx, ny, inputs.RHO_V_086, 0.02, seed=9))
    o.step(t)
    f = o.populations()
    rho, jx, jy = moments(f)

    # inlet: known populations f0 f2 f4 and the outgoing f3 f6 f7
    def inlet_rho_U(y):
        k = f[0, y, 0] + f[2, y, 0] + f[4, y, 0] + 2 * (f[3, y, 0] + f[6, y, 0] + f[7, y, 0])
        if x_bc == 1:
            U = amp * np.sin(2 * np.pi * t / period)
            return k / (1 - U), U
        rb = oracle.inlet_density(p, t)
        return rb, 1 - k / rb

    def outlet_rho_U(y):
        k = f[0, y, -1] + f[2, y, -1] + f[4, y, -1] + 2 * (f[1, y, -1] + f[5, y, -1] + f[8, y, -1])
        ro = p["rho_out"]
        return ro, k / ro - 1

    deltas = []
    # (column, row, (e_x, e_y) of the bounced-back population that replaces an unknown)
    for col, row, (cx, cy), rU in [(0, 0, (1, 1), inlet_rho_U), (0, ny - 1, (1, -1), inlet_rho_U),
                                   (-1, 0, (-1, 1), outlet_rho_U),
                                   (-1, ny - 1, (-1, -1), outlet_rho_U)]:
        rb, U = rU(row)
        delta = rho[row, col] - rb
        assert jx[row, col] - rb * U == pytest.approx(cx * delta, abs=1e-14)
        assert jy[row, col] == pytest.approx(cy * delta, abs=1e-14)
        deltas.append(abs(delta))
    # the corners do differ from full Zou-He nodes
    assert min(deltas) > 1e-6
    # and the rows between them carry the full Zou-He moments
    for row in range(1, ny - 1):
        rb, U = inlet_rho_U(row)
        assert rho[row, 0] == pytest.approx(rb, rel=1e-13)
        assert jx[row, 0] == pytest.approx(rb * U, abs=1e-14)
        assert jy[row, 0] == pytest.approx(0.0, abs=1e-14)
        ro, Uo = outlet_rho_U(row)
        assert rho[row, -1] == pytest.approx(ro, rel=1e-13)
        assert jx[row, -1] == pytest.approx(ro * Uo, abs=1e-14)
        assert jy[row, -1] == pytest.approx(0.0, abs=1e-14)


def test_inlet_density_near_the_critical_point():
    """The pressure inlet's vapour-branch density at 0.97 Tc and 0.99 Tc, where the
    branch between 0 and the first maximum of the isotherm is narrow, against a
    brute-force answer: P sampled on 2 million densities, the first sample where it
    stops rising, and the last sample below the target before it."""
    for Tr in (0.97, 0.99):
        rho_out = 0.6 if Tr < 0.98 else 1.2
        p = inputs.base_params(x_bc=2, p_amp_frac=0.05, u_period=40.0, T_inlet=Tr,
                               rho_out=rho_out)
        Tabs = Tr * oracle.critical_temperature(p)
        r = np.linspace(1e-6, 0.999 / p["eos_b"], 2_000_001)
        a, b, R = p["eos_a"], p["eos_b"], p["eos_R"]
        om = p["eos_omega"]
        kap = 0.37464 + 1.54226 * om - 0.26992 * om * om
        phi = (1 + kap * (1 - np.sqrt(Tr))) ** 2
        P = r * R * Tabs / (1 - b * r) - a * phi * r * r / (1 + 2 * b * r - b * b * r * r)
        top = np.argmax(np.diff(P) <= 0)
        assert 0 < top < len(r) - 2, "the isotherm has a maximum below Tc"
        for t in (0, 10, 30):
            p0 = oracle.eos_pressure(p, rho_out, Tabs)
            target = p0 * (1 + 0.05 * np.sin(2 * np.pi * t / 40.0))
            brute = r[np.searchsorted(P[:top + 1], target) - 1]
            got = oracle.inlet_density(p, t)
            assert got <= r[top + 1]
            assert got == pytest.approx(brute, abs=2 * (r[1] - r[0]))
