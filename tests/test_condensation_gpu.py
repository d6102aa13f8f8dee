"""Condensation statistics of the Section 3.3 channel on the GPU against the FP64
oracle (tests/golden/condensation_stats.json, written by make_condensation_stats.py,
which calls only the oracle), on the 128 x 32 cut-down of the 1024 x 128 channel.

Statistics, not fields: once vapour condenses, small differences grow, so the test
compares the droplet measure of the library (lbm_droplet_stats) on the GPU's density
with the oracle's measure on the oracle's density: droplet count and spacing per wall,
liquid nodes and condensed mass.
  - The channel as configured (walls at 0.80 Tc): the vapour stays metastable for all
    50000 updates (the model has no thermal fluctuations to nucleate it); no droplet
    and no condensed mass on either side, and the largest density agrees to 1e-5.
  - Walls at 0.65 Tc: both walls condense from the inlet side; one condensate per wall
    on both sides at 5000, 10000 and 15000 updates, liquid nodes and condensed mass
    within COND_TOL of the oracle's.
"""
import json
import os

import numpy as np
import pytest

from paper_1803_01756_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
COND_TOL = 0.02


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_01756_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "condensation_stats.json")) as fh:
        return json.load(fh)


def gpu_stats(name, times):
    from paper_1803_01756_gb300.lattice import Lattice, droplet_stats
    w = inputs.workload(name)
    lat = Lattice(w["nx"], w["ny"], w["params"])
    lat.write_fields(inputs.initial_density(w))
    thr = 0.5 * (inputs.RHO_L_086 + inputs.RHO_V_086)
    out = {}
    for t in times:
        lat.step(t - lat.t)
        rho = lat.read_fields()[0]
        st = droplet_stats(rho, thr, inputs.RHO_V_086)
        st["rho_max"] = float(rho.max())
        st["status"] = lat.status()
        out[str(t)] = st
    lat.close()
    return out


def test_configured_channel_stays_vapour(golden):
    ref = golden["channel_128x32"]
    got = gpu_stats("channel_128x32", sorted(int(t) for t in ref))
    for t, g in got.items():
        r = ref[t]
        assert g["status"] == 0 and r["status"] == 0
        assert g["count"] == r["count"] == [0, 0]
        assert g["liquid_nodes"] == r["liquid_nodes"] == 0
        assert g["rho_max"] == pytest.approx(r["rho_max"], rel=1e-5)


def test_cold_wall_condensate_matches_oracle(golden):
    ref = golden["cold_128x32"]
    got = gpu_stats("cold_128x32", sorted(int(t) for t in ref))
    for t, g in got.items():
        r = ref[t]
        assert g["status"] == 0 and r["status"] == 0
        assert g["count"] == r["count"], (t, g, r)
        assert g["detached"] == r["detached"]
        assert g["spacing"] == pytest.approx(r["spacing"], abs=1.0)
        assert g["liquid_nodes"] == pytest.approx(r["liquid_nodes"], rel=COND_TOL), (t, g, r)
        assert g["condensed_mass"] == pytest.approx(r["condensed_mass"], rel=COND_TOL), (t, g, r)
