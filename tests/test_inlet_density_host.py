"""The pressure inlet's density (Section 3.3) as the CUDA library's host runtime
computes it, against the oracle's, without a GPU.

The two are written independently: the library isolates the isotherm's first
maximum as the smallest root of the quartic that dP/drho of Eq. 11 reduces to and
solves P(rho) = target by bracketed Newton steps; the oracle scans the isotherm
and bisects.  Both must give the same vapour-branch root, also close to Tc where
the branch is narrow, and the same branch end when the target lies above it.

Tolerance 1e-8 relative: the isotherm is flat at its maximum, and the oracle locates
that maximum from differences of P taken 2e-7 apart, which resolve it to a few 1e-9;
the lattice receives this density in FP32 (about 6e-8 relative), far coarser."""
import numpy as np
import pytest

import oracle
from paper_1803_01756_gb300 import inputs


@pytest.fixture(scope="module")
def lattice_mod():
    from paper_1803_01756_gb300 import build, lattice
    build.build()
    return lattice


CASES = [
    # (T_inlet / Tc, rho_out, p_amp_frac)
    (0.86, inputs.RHO_V_086, 0.1),
    (0.80, 0.19, 0.3),
    (0.70, 0.05, 0.5),
    (0.93, 0.8, 0.05),
    (0.97, 0.6, 0.05),
    (0.99, 1.2, 0.05),
    (0.99, 1.2, 0.5),   # targets above the branch's top pressure: the branch end
    (1.02, 1.0, 0.2),   # above Tc the isotherm rises up to the pole
]


@pytest.mark.parametrize("Tr,rho_out,amp", CASES)
def test_library_inlet_density_matches_oracle(lattice_mod, Tr, rho_out, amp):
    p = inputs.base_params(x_bc=2, p_amp_frac=amp, u_period=40.0, T_inlet=Tr, rho_out=rho_out)
    for t in range(0, 40, 3):
        got = lattice_mod.pressure_inlet_density(p, t)
        ref = oracle.inlet_density(p, t)
        assert got == pytest.approx(ref, rel=1e-8, abs=1e-12), (Tr, t, got, ref)


def test_library_rejects_bad_inlet_parameters(lattice_mod):
    from paper_1803_01756_gb300.lattice import LbmError
    with pytest.raises(LbmError):
        lattice_mod.pressure_inlet_density(inputs.base_params(x_bc=2, p_amp_frac=1.5), 0)
    with pytest.raises(LbmError):
        lattice_mod.pressure_inlet_density(inputs.base_params(x_bc=2, rho_out=0.0), 0)
