"""Batched persistent updates: a lattice's fields after stepping inside a batch of
uneven lattices equal its fields after stepping alone, within the FP32 parity
tolerance (1e-5, same metric as the oracle parity tests).  Not bitwise: the batched
kernel reads the lattice parameters from shared memory and the single-lattice kernel
from the constant bank, and the compiler contracts a few products differently
(measured differences ~2e-6 relative near the walls)."""
import numpy as np
import pytest

from paper_1803_01756_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_01756_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def channel_set(n, seed, angles=()):
    """Uneven channels: lengths 40..400, widths 8..72, contact angles 45..135 degrees
    (wall strengths from the oracle's G_w -> angle table) and inlet periods drawn from a
    seeded generator; then one channel for each angle in `angles`."""
    u = inputs.uniform01(4 * (n + len(angles)), seed).reshape(-1, 4)
    specs = []
    for k in range(n + len(angles)):
        nx = int(40 + u[k, 0] * 360)
        ny = int(8 + u[k, 1] * 64)
        ca = 45.0 + 90.0 * u[k, 2] if k < n else angles[k - n]
        p = inputs.base_params(Gw=inputs.wall_strength_for_angle(ca), u_amp=0.02,
                               u_period=float(200 + int(1800 * u[k, 3])))
        specs.append((nx, ny, p, inputs.noisy_density(nx, ny, inputs.RHO_V_086, 0.01, seed + k)))
    return specs


def run_alone(specs, steps):
    from paper_1803_01756_gb300.lattice import Lattice
    out = []
    for nx, ny, p, rho0 in specs:
        lat = Lattice(nx, ny, p, kernel=2)
        lat.write_fields(rho0)
        lat.step(steps)
        out.append(lat.read_fields())
        lat.close()
    return out


@pytest.mark.parametrize("graph,tile_rows,tiling", [(False, 64, None), (True, 24, None),
                                                    (False, 7, None), (False, 0, (24, 94, 1)),
                                                    (True, 0, (16, 244, 2)),
                                                    (False, 0, (40, 120, 2))])
def test_batch_equals_alone(graph, tile_rows, tiling):
    """Default tilings, narrower tiles and two lattice columns per thread."""
    from paper_1803_01756_gb300.lattice import Batch, Lattice
    specs = channel_set(12, seed=30)
    steps = 37  # two graph chunks of 16 and a partial chunk of odd length
    alone = run_alone(specs, steps)
    lats = []
    for nx, ny, p, rho0 in specs:
        lat = Lattice(nx, ny, p, kernel=2)
        lat.write_fields(rho0)
        lats.append(lat)
    b = Batch(lats, graph=graph, tile_rows=tile_rows or None)
    if tiling:
        b.set_tiling(*tiling)
        info = b.info()
        assert (info["tile_rows"], info["tile_cols"], info["cols_per_thread"]) == tiling
    b.step(steps)
    for lat, ref in zip(lats, alone):
        assert lat.t == steps
        rho, ux, uy, T = lat.read_fields()
        rr, rux, ruy, rT = ref
        assert np.abs(rho - rr).max() <= 1e-5 * np.abs(rr).max()
        assert np.hypot(ux - rux, uy - ruy).max() <= 1e-5 * max(np.hypot(rux, ruy).max(), 1e-3)
        assert np.abs(T - rT).max() <= 1e-5 * np.abs(rT).max()
        assert lat.status() == 0
    b.close()
    for lat in lats:
        lat.close()


def test_batch_takes_lattices_of_the_default_kernel_choice():
    """Small lattices created with the library's kernel choice run on the two-pass path;
    a batch takes them like fused-path lattices, and their fields equal the fields of the
    same lattices stepped alone (two-pass) within the FP32 parity tolerance."""
    from paper_1803_01756_gb300.lattice import Batch, Lattice, KERNEL_TWOPASS
    specs = channel_set(4, seed=50)
    steps = 21
    alone = []
    for nx, ny, p, rho0 in specs:
        lat = Lattice(nx, ny, p)
        assert lat.info()["kernel"] == KERNEL_TWOPASS
        lat.write_fields(rho0)
        lat.step(steps)
        alone.append(lat.read_fields())
        lat.close()
    lats = []
    for nx, ny, p, rho0 in specs:
        lat = Lattice(nx, ny, p)
        lat.write_fields(rho0)
        lats.append(lat)
    b = Batch(lats)
    b.step(steps)
    for lat, ref in zip(lats, alone):
        rho, ux, uy, T = lat.read_fields()
        rr, rux, ruy, rT = ref
        assert np.abs(rho - rr).max() <= 1e-5 * np.abs(rr).max()
        assert np.hypot(ux - rux, uy - ruy).max() <= 1e-5 * max(np.hypot(rux, ruy).max(), 1e-3)
        assert np.abs(T - rT).max() <= 1e-5 * np.abs(rT).max()
    b.close()
    for lat in lats:
        lat.close()


def test_batch_rejects_mixed_modes():
    from paper_1803_01756_gb300.lattice import Batch, Lattice, LbmError
    a = Lattice(40, 10, inputs.base_params(), kernel=2)
    c = Lattice(40, 10, inputs.base_params(x_bc=0), kernel=2)
    with pytest.raises(LbmError):
        Batch([a, c])
    with pytest.raises(LbmError):
        Batch([a, a])
    a.close()
    c.close()


def test_autotune_picks_a_candidate_and_keeps_results_finite():
    from paper_1803_01756_gb300.lattice import Batch, Lattice
    specs = channel_set(6, seed=50)
    lats = []
    for nx, ny, p, rho0 in specs:
        lat = Lattice(nx, ny, p, kernel=2)
        lat.write_fields(rho0)
        lats.append(lat)
    b = Batch(lats)
    best = b.autotune(3)
    info = b.info()
    assert best in (16, 24, 32, 48, 64, 96, 128)
    assert info["tile_rows"] == best
    # two column counts are tried for this mode: 7 heights each, then two widths
    assert all(lat.t == (7 * 2 + 2) * 5 for lat in lats)
    assert info["cols_per_thread"] in (1, 2)
    widths = {1: (118, 88, 59), 2: (244, 182, 122)}[info["cols_per_thread"]]
    assert info["tile_cols"] in widths
    for lat in lats:
        assert all(np.isfinite(a).all() for a in lat.read_fields())
    b.close()
    for lat in lats:
        lat.close()


def test_default_tile_height_follows_the_batch_size():
    """A few small lattices get short tiles (so that more CTAs get work: every tile sweeps
    H + 15 row steps whatever the batch size), one large lattice taller ones."""
    from paper_1803_01756_gb300.lattice import Batch, Lattice
    small = [Lattice(512, 64, inputs.base_params(), kernel=2) for _ in range(12)]
    b = Batch(small)
    assert b.info()["tile_rows"] == 16
    b.close()
    big = Lattice(4096, 512, inputs.base_params(), kernel=2)
    b = Batch([big])
    info = b.info()
    assert info["tile_rows"] >= 24 and info["tiles"] <= info["grid"]
    b.close()
    # fewer tiles than SMs at 16 rows: heights below 16 spread the lattice over the SMs
    tiny = Lattice(200, 50, inputs.base_params(), kernel=2)
    b = Batch([tiny])
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    info = b.info()
    assert info["tile_rows"] < 16 and 16 <= info["tiles"] <= sms, info
    b.close()
    for lat in small + [big, tiny]:
        lat.close()


@pytest.mark.parametrize("storage", [0, 2])
def test_batch_against_the_oracle(storage):
    """Each lattice of a batch of uneven channels (default tile height) against the FP64
    oracle after 150 updates: within 1e-5 with FP32 storage, within the FP16 bounds of
    the precision tests with FP16 storage.  The batch includes channels at both ends of
    the contact-angle range of the batch workload (45 and 135 degrees)."""
    import oracle
    from paper_1803_01756_gb300.lattice import Batch, Lattice
    specs = channel_set(5, seed=60, angles=(45.0, 135.0))
    lats = []
    for nx, ny, p, rho0 in specs:
        lat = Lattice(nx, ny, p, kernel=2, storage=storage)
        lat.write_fields(rho0)
        lats.append(lat)
    b = Batch(lats)
    b.step(150)
    b.close()
    tol = {"rho": 1e-5, "u": 1e-5, "T": 1e-5} if storage == 0 else \
        {"rho": 2e-3, "u": 1.5e-2, "T": 5e-4}
    for lat, (nx, ny, p, rho0) in zip(lats, specs):
        rho, ux, uy, T = lat.read_fields()
        o = oracle.Oracle(nx, ny, p)
        o.set_fields(rho0)
        o.step(150)
        rr, rux, ruy, rT = o.fields()
        assert np.abs(rho - rr).max() <= tol["rho"] * np.abs(rr).max()
        assert np.hypot(ux - rux, uy - ruy).max() <= tol["u"] * max(np.hypot(rux, ruy).max(), 1e-3)
        assert np.abs(T - rT).max() <= tol["T"] * np.abs(rT).max()
        lat.close()


def test_batch_tiling_is_validated():
    """Two columns per thread need even tile widths up to 244 and the modes with the
    energy equation and the pseudopotential; one column allows widths up to 118."""
    from paper_1803_01756_gb300.lattice import Batch, Lattice, LbmError
    a = Lattice(64, 16, inputs.base_params(), kernel=2)
    b = Batch([a])
    for bad in [(16, 119, 1), (16, 245, 2), (16, 101, 2), (0, 64, 1), (16, 64, 3)]:
        with pytest.raises(LbmError):
            b.set_tiling(*bad)
    b.set_tiling(16, 244, 2)
    b.close()
    a.close()
    c = Lattice(64, 16, inputs.base_params(thermal=0), kernel=2)
    b = Batch([c])
    with pytest.raises(LbmError):
        b.set_tiling(16, 64, 2)
    b.close()
    c.close()
