"""The C ABI library builds, loads without a GPU and exports every entry point
that include/lbm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_01756_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_step", "lbm_read_fields", "lbm_destroy",
                     "lbm_write_fields", "lbm_reduce"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1803_01756_gb300 import lattice
    declared = set(declared_functions())
    bound = set(lattice.SIGNATURES)
    assert declared == bound, (declared ^ bound)


def _header_fields(struct, typedef):
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (struct, typedef), text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        typ, rest = re.match(r"(long long|size_t|double|int)\s+(.*)", decl).groups()
        for name in rest.split(","):
            fields.append((typ, name.strip()))
    return fields


CTYPE = {"double": ctypes.c_double, "int": ctypes.c_int, "long long": ctypes.c_longlong,
         "size_t": ctypes.c_size_t}


def test_params_struct_layout_matches_header():
    """The ctypes mirror lists the struct fields of include/lbm.h in order."""
    from paper_1803_01756_gb300 import lattice
    fields = _header_fields("lbm_params", "lbm_params_t")
    mirror = [(f[0], f[1]) for f in lattice.LbmParams._fields_]
    assert len(fields) == len(mirror)
    for (typ, name), (mname, mtype) in zip(fields, mirror):
        assert (mname if mname != "lam" else "lambda") == name
        assert mtype is CTYPE[typ]


def test_info_struct_layout_matches_header():
    from paper_1803_01756_gb300 import lattice
    fields = _header_fields("lbm_info", "lbm_info_t")
    mirror = [(f[0], f[1]) for f in lattice.LbmInfo._fields_]
    assert [(n, CTYPE[t]) for t, n in fields] == mirror


def test_host_only_entry_points(lib):
    from paper_1803_01756_gb300 import lattice
    L = lattice.load_library()
    p = lattice.make_params({"eos_a": 2 / 49, "eos_b": 2 / 21, "eos_R": 1.0})
    assert L.lbm_critical_temperature(ctypes.byref(p)) == pytest.approx(
        0.0778 * (2 / 49) / (0.45724 * (2 / 21)), rel=1e-15)
    assert L.lbm_strerror(-4).decode().startswith("device status")
    h = ctypes.c_void_p()
    # invalid sizes are rejected before any device call
    assert L.lbm_create(0, 10, ctypes.byref(p), ctypes.byref(h)) == -1
    L.lbm_destroy(None)


@pytest.mark.parametrize("nx,ny,over", [
    (0, 8, dict()), (8, 0, dict()), ((1 << 20) + 1, 4, dict()), (4, (1 << 20) + 1, dict()),
    (1, 8, dict()),                 # an open x end needs two columns
    (16, 8, dict(x_bc=7)), (16, 8, dict(y_bc=3)), (16, 8, dict(tau_g=0.5)),
    (16, 8, dict(s_q=2.0)), (16, 8, dict(x_bc=2, p_amp_frac=1.0)),
])
def test_invalid_arguments_are_rejected(lib, nx, ny, over):
    """lbm_create validates sizes and parameters before any device call (no GPU needed)."""
    from paper_1803_01756_gb300 import inputs
    from paper_1803_01756_gb300.lattice import Lattice, LbmError
    with pytest.raises(LbmError) as ei:
        Lattice(nx, ny, inputs.base_params(**over))
    assert ei.value.code == -1  # LBM_ERR_ARG


def test_null_handles_are_rejected_before_any_device_call(lib):
    """Every entry point that takes a handle returns LBM_ERR_ARG for a null one (the
    destroy calls do nothing), without touching the device: this runs without a GPU."""
    from paper_1803_01756_gb300 import lattice
    L = lattice.load_library()
    n = None
    d = ctypes.c_double()
    u = ctypes.c_uint()
    z = ctypes.c_size_t()
    i = ctypes.c_int()
    lg = ctypes.c_long()
    info = lattice.LbmInfo()
    p = lattice.make_params({})
    calls = {
        "lbm_write_fields": lambda: L.lbm_write_fields(n, None, None, n),
        "lbm_step": lambda: L.lbm_step(n, 1, n),
        "lbm_set_graph": lambda: L.lbm_set_graph(n, 1),
        "lbm_status": lambda: L.lbm_status(n, ctypes.byref(u), 0, n),
        "lbm_read_fields": lambda: L.lbm_read_fields(n, None, None, None, None, n),
        "lbm_reduce": lambda: L.lbm_reduce(n, ctypes.byref(d), ctypes.byref(d), n),
        "lbm_state_bytes": lambda: L.lbm_state_bytes(n, ctypes.byref(z)),
        "lbm_read_state": lambda: L.lbm_read_state(n, None, 0, n),
        "lbm_write_state": lambda: L.lbm_write_state(n, None, 0, n),
        "lbm_info": lambda: L.lbm_info(n, ctypes.byref(info)),
        "lbm_timing_enable": lambda: L.lbm_timing_enable(n, 1),
        "lbm_timing_get": lambda: L.lbm_timing_get(n, None, None, None, 0, ctypes.byref(i), n),
        "lbm_batch_create": lambda: L.lbm_batch_create(None, 0, ctypes.byref(ctypes.c_void_p())),
        "lbm_batch_step": lambda: L.lbm_batch_step(n, 1, n),
        "lbm_batch_set_graph": lambda: L.lbm_batch_set_graph(n, 1),
        "lbm_batch_set_tile_rows": lambda: L.lbm_batch_set_tile_rows(n, 16),
        "lbm_batch_autotune": lambda: L.lbm_batch_autotune(n, 4, ctypes.byref(i), n),
        "lbm_batch_info": lambda: L.lbm_batch_info(n, None, None, None),
        "lbm_submit": lambda: L.lbm_submit(n, 8, 8, ctypes.byref(p), None, 1, ctypes.byref(lg)),
        "lbm_poll": lambda: L.lbm_poll(n, 0, ctypes.byref(i), None, None, None, None, None),
        "lbm_wait": lambda: L.lbm_wait(n, 0, 0.0, ctypes.byref(i)),
        "lbm_server_stats": lambda: L.lbm_server_stats(n, None),
    }
    for name, call in calls.items():
        assert call() == -1, name
    L.lbm_batch_destroy(n)
    L.lbm_server_destroy(n)
