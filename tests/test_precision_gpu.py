"""Reduced-precision population storage (BF16 / FP16 of f_i/w_i - rho_ref, FP32
arithmetic, FP64 reductions) against the FP64 oracle.

The bounds below (max |X - X_oracle| / max |X_oracle|; velocity as a vector,
floored at 1e-3 like the FP32 parity tests) are the stated accuracy of each storage
format, set above the errors measured on GB300; the FP32 row is the 1e-5 parity
bound for comparison.
"""
import numpy as np
import pytest

import oracle
from paper_1803_01756_gb300 import inputs

pytestmark = pytest.mark.gpu

STORAGES = {"f32": 0, "bf16": 1, "f16": 2}
# every update path stores the populations in the chosen format at the same point, so
# each is held to the same bounds (the library's own choice differs with the lattice size)
KERNELS = ["split", "fused1", "fused2", "twopass"]


def kernel_id(name):
    from paper_1803_01756_gb300 import lattice
    return {"split": lattice.KERNEL_SPLIT, "fused1": lattice.KERNEL_FUSED_1COL,
            "fused2": lattice.KERNEL_FUSED_2COL, "twopass": lattice.KERNEL_TWOPASS}[name]
# stated bounds after 1000 updates of the 200 x 50 channel
# (measured on GB300: f32 9.1e-7 / 5.8e-6 / 2.0e-7, f16 8.3e-4 / 5.2e-3 / 1.5e-4,
#  bf16 1.6e-2 / 9.0e-2 / 2.5e-3 for rho / u / T)
CHANNEL_BOUNDS = {
    "f32": {"rho": 1e-5, "u": 1e-5, "T": 1e-5},
    "f16": {"rho": 2e-3, "u": 1.5e-2, "T": 5e-4},
    "bf16": {"rho": 5e-2, "u": 0.25, "T": 1e-2},
}


# equimolar radius of the sessile drop (about 14 nodes) against the oracle's, in nodes
# (measured on GB300: f32 2.9e-4, f16 6.2e-2, bf16 0.36)
RADIUS_BOUNDS = {"f32": 1e-3, "f16": 0.1, "bf16": 0.4}
# the 4096 x 512 benchmark channel's parameters on a 128 x 32 cut, 20000 updates
# (measured on GB300: f32 1.2e-6 / 2.5e-6 / 1.8e-7, f16 9.8e-4 / 2.3e-3 / 1.3e-4,
#  bf16 3.5e-2 / 0.31 / 3.3e-3 for rho / u / T)
LONG_BOUNDS = {"f32": {"rho": 1e-5, "u": 1e-5, "T": 1e-5},
               "f16": {"rho": 3e-3, "u": 1e-2, "T": 5e-4},
               "bf16": {"rho": 0.1, "u": 0.6, "T": 1e-2}}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_01756_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def errors(gpu, ref):
    rho, ux, uy, T = gpu
    rrho, rux, ruy, rT = ref
    return {
        "rho": np.abs(rho - rrho).max() / np.abs(rrho).max(),
        "u": np.hypot(ux - rux, uy - ruy).max() / max(np.hypot(rux, ruy).max(), 1e-3),
        "T": np.abs(T - rT).max() / np.abs(rT).max(),
    }


@pytest.fixture(scope="module")
def channel_reference():
    w = inputs.workload("channel_200x50")
    o = oracle.Oracle(w["nx"], w["ny"], w["params"])
    o.set_fields(inputs.initial_density(w))
    o.step(1000)
    return o.fields()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_channel_error_against_oracle(storage, kernel, channel_reference):
    from paper_1803_01756_gb300.lattice import Lattice
    w = inputs.workload("channel_200x50")
    lat = Lattice(w["nx"], w["ny"], w["params"], kernel=kernel_id(kernel),
                  storage=STORAGES[storage])
    lat.write_fields(inputs.initial_density(w))
    lat.step(1000)
    err = errors(lat.read_fields(), channel_reference)
    lat.close()
    print(f"\n200x50 channel, 1000 updates, {kernel}, {storage}: " +
          ", ".join(f"{k} {v:.2e}" for k, v in err.items()))
    for k, bound in CHANNEL_BOUNDS[storage].items():
        assert err[k] <= bound, (storage, err)


def sessile_drop(nx=80, ny=40):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = np.hypot(x - nx / 2, y + 0.5)
    return inputs.RHO_V_086 + (inputs.RHO_L_086 - inputs.RHO_V_086) * 0.5 * (1 - np.tanh((r - 14) / 2))


def contact_angle(rho):
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_multiphase import contact_angle as ca
    return ca(rho, 0.5 * (inputs.RHO_V_086 + inputs.RHO_L_086))


def equimolar_radius(rho):
    """Radius of the half-disc holding the drop's condensed mass at liquid density:
    sqrt(2 A / pi), A = sum(rho - rho_v) / (rho_l - rho_v)."""
    A = (rho - inputs.RHO_V_086).sum() / (inputs.RHO_L_086 - inputs.RHO_V_086)
    return float(np.sqrt(2 * A / np.pi))


@pytest.fixture(scope="module")
def drop_reference():
    p = inputs.base_params(thermal=0, x_bc=0, y_bc=1, Gw=-1.15)
    o = oracle.Oracle(80, 40, p)
    o.set_fields(sessile_drop())
    o.step(4000)
    rho = o.fields()[0]
    return p, rho, contact_angle(rho)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_liquid_drop_density_and_contact_angle(storage, kernel, drop_reference):
    """Sessile drop (density ratio 17): liquid density and contact angle after 4000
    updates, against the oracle.  Over this many updates the interface amplifies
    rounding, so even FP32 departs by ~1e-4 in density near the interface (measured
    8.5e-5) while the contact angle agrees to 0.01 degree; measured f16 1.8e-2 and
    0.07 degree, bf16 8.9e-2 and 0.84 degree (the split path: 0.24 and 3.9 degrees)."""
    from paper_1803_01756_gb300.lattice import Lattice
    p, rho_ref, ca_ref = drop_reference
    lat = Lattice(80, 40, p, kernel=kernel_id(kernel), storage=STORAGES[storage])
    lat.write_fields(sessile_drop())
    lat.step(4000)
    rho = lat.read_fields()[0]
    lat.close()
    err = np.abs(rho - rho_ref).max() / rho_ref.max()
    ca = contact_angle(rho)
    dr = abs(equimolar_radius(rho) - equimolar_radius(rho_ref))
    print(f"\nsessile drop, {kernel}, {storage}: rho error {err:.2e}, contact angle {ca:.2f} "
          f"(oracle {ca_ref:.2f}), equimolar radius error {dr:.2e}")
    bound = {"f32": 2e-4, "f16": 8e-2, "bf16": 0.25}[storage]
    assert err <= bound
    assert abs(ca - ca_ref) <= {"f32": 0.01, "f16": 0.5, "bf16": 6.0}[storage]
    assert dr <= RADIUS_BOUNDS[storage], (storage, dr)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_16bit_checkpoint_round_trip(storage):
    from paper_1803_01756_gb300.lattice import Lattice
    w = inputs.workload("channel_200x50")
    a = Lattice(w["nx"], w["ny"], w["params"], storage=STORAGES[storage])
    a.write_fields(inputs.initial_density(w))
    a.step(40)
    state = a.read_state()
    a.step(20)
    fa = a.read_fields()
    b = Lattice(w["nx"], w["ny"], w["params"], storage=STORAGES[storage])
    b.write_state(state)
    b.step(20)
    fb = b.read_fields()
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    a.close()
    b.close()


@pytest.fixture(scope="module")
def long_reference():
    """FP64 oracle on a 128 x 32 cut of the 4096 x 512 benchmark channel (its parameters
    and noise seed), 20000 updates (about 40 s of host time)."""
    w = inputs.workload("channel_4096x512")
    rho0 = inputs.noisy_density(128, 32, inputs.RHO_V_086, w["noise"], w["seed"])
    o = oracle.Oracle(128, 32, w["params"])
    o.set_fields(rho0)
    o.step(20000)
    assert o.status == 0
    return w["params"], rho0, o.fields()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_benchmark_channel_20000_updates(storage, kernel, long_reference):
    """The benchmark channel's parameters over its 20000 updates, on a 128 x 32 cut that
    the oracle finishes in about 40 s: errors of rho, u and T per storage format."""
    from paper_1803_01756_gb300.lattice import Lattice
    p, rho0, ref = long_reference
    lat = Lattice(128, 32, p, kernel=kernel_id(kernel), storage=STORAGES[storage])
    lat.write_fields(rho0)
    lat.step(20000)
    err = errors(lat.read_fields(), ref)
    assert lat.status() == 0
    lat.close()
    print(f"\n128x32 cut of the 4096x512 channel, 20000 updates, {kernel}, {storage}: " +
          ", ".join(f"{k} {v:.2e}" for k, v in err.items()))
    for k, bound in LONG_BOUNDS[storage].items():
        assert err[k] <= bound, (storage, err)
