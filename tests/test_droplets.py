"""The droplet measure of the condensation runs (the channel of Section 3.3 and its
closing wettability discussion of droplet number and spacing): droplet count and
spacing per wall, condensed mass.

Pins: hand-built density fields whose answers follow from their construction (caps
on the walls at known positions, a floating blob, diagonal contacts that 8-connectivity
joins, a blob across the periodic seam, a bridge between the walls).  Both the oracle's
measure (scipy labelling) and the library's (lbm_droplet_stats, native union-find,
host-only) are held to them, then to each other on seeded random fields."""
import numpy as np
import pytest

from oracle.droplets import droplet_stats as oracle_stats
from paper_1803_01756_gb300 import inputs

RL, RV = 6.0, 0.4
THR = 0.5 * (RL + RV)


@pytest.fixture(scope="module")
def lib_stats():
    from paper_1803_01756_gb300 import build, lattice
    build.build()
    return lattice.droplet_stats


def caps_field(nx=96, ny=24):
    """Half-discs of radius 4 centred on the bottom wall at x = 10, 30, 50 and on the top
    wall at x = 20, 45; a square blob in the middle touching neither wall."""
    rho = np.full((ny, nx), RV)
    y, x = np.mgrid[0:ny, 0:nx]
    for xc in (10, 30, 50):
        rho[(x - xc) ** 2 + y ** 2 <= 16] = RL
    for xc in (20, 45):
        rho[(x - xc) ** 2 + (ny - 1 - y) ** 2 <= 16] = RL
    rho[10:13, 70:74] = RL
    return rho


def check_caps(stats, rho):
    assert stats["count"] == [3, 2]
    assert stats["spacing"] == pytest.approx([20.0, 25.0], abs=1e-12)
    assert stats["detached"] == 1
    n = int((rho > THR).sum())
    assert stats["liquid_nodes"] == n
    assert stats["condensed_mass"] == pytest.approx(n * (RL - RV), rel=1e-14)


def test_oracle_measure_on_caps():
    rho = caps_field()
    check_caps(oracle_stats(rho, THR, RV), rho)


def test_library_measure_on_caps(lib_stats):
    rho = caps_field()
    check_caps(lib_stats(rho, THR, RV), rho)


def diagonal_field():
    """Two bottom caps joined only through a diagonal contact (one 8-connected droplet),
    and a third cap one node apart (a droplet of its own)."""
    rho = np.full((10, 30), RV)
    rho[0:2, 3:6] = RL
    rho[2, 6] = RL      # touches (1, 5) diagonally
    rho[3, 7] = RL      # touches (2, 6) diagonally
    rho[0:4, 8:10] = RL  # touches (3, 7) sideways at (3, 8)
    rho[0:2, 12:14] = RL  # separated by column 10-11 from the rest
    return rho


@pytest.mark.parametrize("which", ["oracle", "library"])
def test_eight_connectivity(which, lib_stats):
    rho = diagonal_field()
    st = oracle_stats(rho, THR, RV) if which == "oracle" else lib_stats(rho, THR, RV)
    assert st["count"] == [2, 0]
    xs_a = [3, 4, 5, 3, 4, 5, 6, 7] + [8, 9] * 4
    expect = (12.5 - np.mean(xs_a)) / 1
    assert st["spacing"][0] == pytest.approx(expect, abs=1e-12)


@pytest.mark.parametrize("which", ["oracle", "library"])
def test_periodic_seam_and_bridge(which, lib_stats):
    """A bottom cap across the periodic seam (columns 38-39 and 0-1 of 40) is one droplet
    centred at x = 0 (the circular mean); a liquid bridge from wall to wall counts once on
    each wall."""
    rho = np.full((12, 40), RV)
    rho[0:3, [38, 39, 0, 1]] = RL
    rho[:, 20:23] = RL
    f = oracle_stats if which == "oracle" else lib_stats
    st = f(rho, THR, RV, periodic_x=True)
    assert st["count"] == [2, 1]
    assert st["spacing"] == pytest.approx([20.0, 0.0])
    open_st = f(rho, THR, RV, periodic_x=False)
    assert open_st["count"] == [3, 1]  # without the wrap the seam cap is two caps


def random_field(seed, nx=150, ny=40):
    """Seeded random caps and blobs (radii 1-6) on a vapour background with noise."""
    u = inputs.uniform01(64, seed)
    rho = RV * (1 + 0.01 * (2 * inputs.uniform01(nx * ny, seed + 1).reshape(ny, nx) - 1))
    y, x = np.mgrid[0:ny, 0:nx]
    for k in range(16):
        xc, yc, r = u[4 * k] * nx, u[4 * k + 1] * ny, 1 + 5 * u[4 * k + 2]
        if u[4 * k + 3] < 0.4:
            yc = 0.0
        elif u[4 * k + 3] < 0.8:
            yc = ny - 1.0
        rho[(x - xc) ** 2 + (y - yc) ** 2 <= r * r] = RL * (0.95 + 0.1 * u[4 * k + 3])
    return rho


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("periodic", [False, True])
def test_library_equals_oracle_on_random_fields(seed, periodic, lib_stats):
    rho = random_field(seed)
    a, b = lib_stats(rho, THR, RV, periodic), oracle_stats(rho, THR, RV, periodic)
    assert a["count"] == b["count"] and a["detached"] == b["detached"]
    assert a["liquid_nodes"] == b["liquid_nodes"]
    assert a["spacing"] == pytest.approx(b["spacing"], rel=1e-12, abs=1e-12)
    assert a["condensed_mass"] == pytest.approx(b["condensed_mass"], rel=1e-12)


def test_library_rejects_bad_arguments(lib_stats):
    from paper_1803_01756_gb300.lattice import LbmError
    with pytest.raises(LbmError):
        lib_stats(np.zeros((4, 4)), float("nan"), 0.0)


@pytest.mark.parametrize("theta", [50.0, 90.0, 130.0])
def test_oracle_contact_angle_of_synthetic_caps(theta):
    """A circular cap of radius R meeting the wall (y = -1/2) at angle theta, drawn with a
    smooth tanh interface: the measure 2 atan(2h / w) returns theta within 2 degrees."""
    from oracle.droplets import contact_angle
    nx, ny, R = 160, 80, 22.0
    yc = -0.5 - R * np.cos(np.radians(theta))
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = np.hypot(x - nx / 2, y - yc)
    rho = RV + (RL - RV) * 0.5 * (1 - np.tanh((r - R) / 1.5))
    assert contact_angle(rho, THR) == pytest.approx(theta, abs=2.0)
