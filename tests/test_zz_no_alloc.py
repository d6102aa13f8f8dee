"""The allocation-free mass/heat entry point against the handle-based one.

lbm_mass_heat_noalloc serves callers that cannot call cudaMalloc (a framework or
serving loop that owns the whole device-memory budget, or a loop that must not
risk the synchronisation an allocation can cause).  It keeps its partial sums in
a fixed array in the library's device memory instead of allocating.  This test
gives it the fields of a stepped lattice in caller-owned device buffers and
checks, on two calls in a row, that it returns the sums lbm_reduce returns for
the same lattice.  The file sorts last so that a stop-at-first-failure run has
already run every other test.
"""
import ctypes

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


def test_noalloc_sums_match_lbm_reduce_on_two_calls():
    import torch
    from paper_1803_01756_gb300.lattice import Lattice, load_library
    w = inputs.workload("channel_200x50")
    nx, ny = w["nx"], w["ny"]
    lat = Lattice(nx, ny, w["params"])
    lat.write_fields(inputs.initial_density(w))
    lat.step(300)
    mass, heat = lat.reduce()
    rho, _, _, T = lat.read_fields()
    T_ref = lat.info()["T_ref"]
    lat.close()

    lib = load_library()
    d_rho = torch.tensor(rho, dtype=torch.float32, device="cuda").contiguous()
    d_T = torch.tensor(T - T_ref, dtype=torch.float32, device="cuda").contiguous()
    d_out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        d_out.fill_(-1.0)
        rc = lib.lbm_mass_heat_noalloc(
            ctypes.c_void_p(d_rho.data_ptr()), ctypes.c_void_p(d_T.data_ptr()), nx, ny, nx,
            T_ref, w["params"]["Cv"], ctypes.c_void_p(d_out.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, (call, rc)
        got = d_out.cpu().numpy()
        np.testing.assert_allclose(got, [mass, heat], rtol=1e-12, atol=0)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch
    from paper_1803_01756_gb300.lattice import load_library
    lib = load_library()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    o = ctypes.c_void_p(out.data_ptr())
    too_big = (1 << 20) + 1
    assert lib.lbm_mass_heat_noalloc(p, p, too_big, 1, too_big, 0.0, 1.0, o, None) == -1
    assert lib.lbm_mass_heat_noalloc(p, p, 4, 4, 3, 0.0, 1.0, o, None) == -1
    assert lib.lbm_mass_heat_noalloc(None, p, 4, 4, 4, 0.0, 1.0, o, None) == -1


def _noalloc(lib, d_rho, d_T, nx, ny, pitch, T_ref, Cv, d_out, stream):
    rc = lib.lbm_mass_heat_noalloc(
        ctypes.c_void_p(d_rho.data_ptr()), ctypes.c_void_p(d_T.data_ptr()), nx, ny, pitch,
        T_ref, Cv, ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, rc
    return d_out.cpu().numpy()


def _fields(nx, ny, pitch, seed):
    """FP32 density and temperature deviation, row y at element y * pitch; the padding
    columns hold NaN, which a read of them would carry into the sums."""
    rho = (0.4 + inputs.uniform01(nx * ny, seed).reshape(ny, nx)).astype(np.float32)
    Td = (1e-3 * (inputs.uniform01(nx * ny, seed + 1).reshape(ny, nx) - 0.5)).astype(np.float32)
    pr = np.full((ny, pitch), np.nan, dtype=np.float32)
    pT = np.full((ny, pitch), np.nan, dtype=np.float32)
    pr[:, :nx], pT[:, :nx] = rho, Td
    return pr, pT, rho.astype(np.float64), Td.astype(np.float64)


def test_noalloc_pitched_fields_large_then_small():
    """Pitched rows with NaN padding; a field large enough that the first stage uses all
    1216 partial pairs, followed by a one-block field: the second call must read only the
    pair it wrote, never the stale pairs of the first."""
    import torch
    from paper_1803_01756_gb300.lattice import load_library
    lib = load_library()
    stream = torch.cuda.current_stream()
    T_ref, Cv = 0.0627, 5.0
    d_out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for nx, ny, pitch, seed in [(2560, 1024, 2592, 31), (37, 5, 64, 33), (2560, 1024, 2560, 35),
                                (200, 50, 224, 37)]:
        pr, pT, rho, Td = _fields(nx, ny, pitch, seed)
        d_rho = torch.from_numpy(pr).cuda()
        d_T = torch.from_numpy(pT).cuda()
        d_out.fill_(-1.0)
        got = _noalloc(lib, d_rho, d_T, nx, ny, pitch, T_ref, Cv, d_out, stream)
        expect = [rho.sum(), (rho * Cv * (T_ref + Td)).sum()]
        np.testing.assert_allclose(got, expect, rtol=1e-12, atol=0)
