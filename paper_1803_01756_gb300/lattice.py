"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the lattice update runs in the CUDA library; if the library has
not been built, or no CUDA device is present, the calls raise.  There is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm_gb300.so")

LBM_OK = 0
ERRORS = {-1: "LBM_ERR_ARG", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA", -4: "LBM_ERR_UNSTABLE",
          -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_BUSY", -7: "LBM_ERR_STATE"}
KERNEL_AUTO, KERNEL_SPLIT, KERNEL_FUSED, KERNEL_FUSED_1COL, KERNEL_FUSED_2COL, KERNEL_TWOPASS = (
    0, 1, 2, 3, 4, 5)
STORAGE_F32 = 0


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({_strerror(code)})")
        self.code = code


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("eos_a", ctypes.c_double), ("eos_b", ctypes.c_double),
        ("eos_R", ctypes.c_double), ("eos_omega", ctypes.c_double),
        ("G", ctypes.c_double), ("Gw", ctypes.c_double), ("rho_w", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("tau_g", ctypes.c_double), ("tau_l", ctypes.c_double),
        ("rho_g", ctypes.c_double), ("rho_l", ctypes.c_double),
        ("s_e", ctypes.c_double), ("s_zeta", ctypes.c_double), ("s_q", ctypes.c_double),
        ("Cv", ctypes.c_double), ("lam", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("g_omega", ctypes.c_double),
        ("T0", ctypes.c_double), ("T_wall_left", ctypes.c_double),
        ("T_wall_right", ctypes.c_double), ("T_inlet", ctypes.c_double),
        ("x_bc", ctypes.c_int), ("y_bc", ctypes.c_int),
        ("u_amp", ctypes.c_double), ("u_period", ctypes.c_double),
        ("rho_out", ctypes.c_double),
        ("thermal", ctypes.c_int), ("multiphase", ctypes.c_int),
        ("storage", ctypes.c_int), ("rho_ref", ctypes.c_double), ("kernel", ctypes.c_int),
        ("p_amp_frac", ctypes.c_double),
        ("T_top_left", ctypes.c_double), ("T_top_right", ctypes.c_double),
        ("top_iso_x0", ctypes.c_int), ("top_iso_x1", ctypes.c_int),
        ("bot_iso_x0", ctypes.c_int), ("bot_iso_x1", ctypes.c_int),
    ]


class LbmInfo(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pitch", ctypes.c_int),
                ("t", ctypes.c_longlong), ("Tc", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("rho_ref", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("kernel", ctypes.c_int), ("tile_cols", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("cols_per_thread", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget", ctypes.c_size_t),
                ("max_active", ctypes.c_int), ("chunk_steps", ctypes.c_long)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_long), ("active", ctypes.c_long),
                ("completed", ctypes.c_long), ("failed", ctypes.c_long),
                ("rounds", ctypes.c_long), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t)]


class DropletStats(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int * 2), ("spacing", ctypes.c_double * 2),
                ("condensed_mass", ctypes.c_double), ("liquid_nodes", ctypes.c_longlong),
                ("detached", ctypes.c_int)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE = 0, 1, 2

# every symbol declared in include/lbm.h, with its ctypes signature
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
SIGNATURES = {
    "lbm_create": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(LbmParams),
                    ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "lbm_write_fields": ([_vp, _dp, _dp, _vp], ctypes.c_int),
    "lbm_step": ([_vp, ctypes.c_long, _vp], ctypes.c_int),
    "lbm_read_fields": ([_vp, _dp, _dp, _dp, _dp, _vp], ctypes.c_int),
    "lbm_reduce": ([_vp, _dp, _dp, _vp], ctypes.c_int),
    "lbm_status": ([_vp, ctypes.POINTER(ctypes.c_uint), ctypes.c_int, _vp], ctypes.c_int),
    "lbm_state_bytes": ([_vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "lbm_read_state": ([_vp, _vp, ctypes.c_size_t, _vp], ctypes.c_int),
    "lbm_write_state": ([_vp, _vp, ctypes.c_size_t, _vp], ctypes.c_int),
    "lbm_info": ([_vp, ctypes.POINTER(LbmInfo)], ctypes.c_int),
    "lbm_timing_enable": ([_vp, ctypes.c_int], ctypes.c_int),
    "lbm_set_graph": ([_vp, ctypes.c_int], ctypes.c_int),
    "lbm_timing_get": ([_vp, ctypes.POINTER(ctypes.c_char_p), _dp, ctypes.POINTER(ctypes.c_long),
                        ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp], ctypes.c_int),
    "lbm_destroy": ([_vp], None),
    "lbm_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "lbm_critical_temperature": ([ctypes.POINTER(LbmParams)], ctypes.c_double),
    "lbm_pressure_inlet_density": ([ctypes.POINTER(LbmParams), ctypes.c_longlong, _dp],
                                   ctypes.c_int),
    "lbm_batch_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                          ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "lbm_batch_step": ([_vp, ctypes.c_long, _vp], ctypes.c_int),
    "lbm_batch_set_graph": ([_vp, ctypes.c_int], ctypes.c_int),
    "lbm_batch_set_tile_rows": ([_vp, ctypes.c_int], ctypes.c_int),
    "lbm_batch_autotune": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp], ctypes.c_int),
    "lbm_batch_set_tiling": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "lbm_batch_tiling": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "lbm_batch_info": ([_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                        ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "lbm_batch_destroy": ([_vp], None),
    "lbm_server_create": ([ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)],
                          ctypes.c_int),
    "lbm_submit": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(LbmParams), _dp, ctypes.c_long,
                    ctypes.POINTER(ctypes.c_long)], ctypes.c_int),
    "lbm_poll": ([_vp, ctypes.c_long, ctypes.POINTER(ctypes.c_int), _dp, _dp, _dp, _dp, _dp],
                 ctypes.c_int),
    "lbm_wait": ([_vp, ctypes.c_long, ctypes.c_double, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "lbm_server_stats": ([_vp, ctypes.POINTER(ServerStats)], ctypes.c_int),
    "lbm_server_destroy": ([_vp], None),
    "lbm_droplet_stats": ([_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                           ctypes.c_int, ctypes.POINTER(DropletStats)], ctypes.c_int),
    "lbm_mass_heat_noalloc": ([_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, _vp, _vp], ctypes.c_int),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load the built CUDA library (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library {path} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _strerror(code: int) -> str:
    try:
        return load_library().lbm_strerror(code).decode()
    except Exception:
        return "?"


def _check(rc: int, where: str):
    if rc != LBM_OK:
        raise LbmError(rc, where)


def make_params(d: dict, **extra) -> LbmParams:
    p = LbmParams()
    names = {f[0] for f in LbmParams._fields_}
    for k, v in {**d, **extra}.items():
        key = "lam" if k == "lambda" else k
        if key not in names:
            raise KeyError(f"unknown parameter {k!r}")
        setattr(p, key, v)
    return p


def _stream_ptr(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def droplet_stats(rho: np.ndarray, threshold: float, rho_v: float,
                  periodic_x: bool = False) -> dict:
    """Droplet count and spacing per wall, condensed mass and liquid nodes of a host
    density field [ny][nx] (lbm_droplet_stats; host-side call, no GPU needed)."""
    r = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = r.shape
    out = DropletStats()
    _check(load_library().lbm_droplet_stats(_dptr(r), nx, ny, float(threshold), float(rho_v),
                                            int(bool(periodic_x)), ctypes.byref(out)),
           "lbm_droplet_stats")
    return {"count": list(out.count), "spacing": list(out.spacing),
            "condensed_mass": out.condensed_mass, "liquid_nodes": out.liquid_nodes,
            "detached": out.detached}


def pressure_inlet_density(params: dict, t: int) -> float:
    """Density the pressure inlet imposes at time t (host-side call, no GPU needed)."""
    out = ctypes.c_double()
    p = make_params(params)
    _check(load_library().lbm_pressure_inlet_density(ctypes.byref(p), int(t), ctypes.byref(out)),
           "lbm_pressure_inlet_density")
    return out.value


class Lattice:
    """One lattice of nx * ny nodes on the current CUDA device.

    Host arrays are [ny][nx] float64.  ``stream`` arguments accept a
    torch.cuda.Stream, a raw cudaStream_t integer, or None for torch's current
    stream.
    """

    def __init__(self, nx: int, ny: int, params: dict, kernel: int = KERNEL_AUTO,
                 storage: int = STORAGE_F32, rho_ref: float = 0.0):
        self._lib = load_library()
        self.nx, self.ny = int(nx), int(ny)
        self.params = dict(params)
        self._p = make_params(params, kernel=kernel, storage=storage, rho_ref=rho_ref)
        h = ctypes.c_void_p()
        _check(self._lib.lbm_create(self.nx, self.ny, ctypes.byref(self._p), ctypes.byref(h)),
               "lbm_create")
        self._h = h

    # -- life cycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state --------------------------------------------------------------
    def write_fields(self, rho: np.ndarray, T: np.ndarray | None = None, stream=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ny, self.nx)
        Tc = None
        if T is not None:
            Tc = np.ascontiguousarray(T, dtype=np.float64).reshape(self.ny, self.nx)
        _check(self._lib.lbm_write_fields(self._h, _dptr(rho), _dptr(Tc), _stream_ptr(stream)),
               "lbm_write_fields")

    def step(self, nsteps: int = 1, stream=None):
        _check(self._lib.lbm_step(self._h, int(nsteps), _stream_ptr(stream)), "lbm_step")

    def set_graph(self, enable: bool = True):
        _check(self._lib.lbm_set_graph(self._h, int(bool(enable))), "lbm_set_graph")

    def read_fields(self, stream=None, check: bool = True, out=None):
        """(rho, ux, uy, T) as [ny][nx] FP64 arrays.  out: four C-contiguous FP64 arrays of
        that shape to fill instead of new ones (page-locked ones are written by the kernels
        directly, with no staging copy)."""
        shp = (self.ny, self.nx)
        if out is None:
            rho, ux, uy, T = (np.empty(shp) for _ in range(4))
        else:
            rho, ux, uy, T = out
            for a in out:
                if a.shape != shp or a.dtype != np.float64 or not a.flags.c_contiguous:
                    raise ValueError(f"out arrays must be C-contiguous float64 of shape {shp}")
        rc = self._lib.lbm_read_fields(self._h, _dptr(rho), _dptr(ux), _dptr(uy), _dptr(T),
                                       _stream_ptr(stream))
        if check:
            _check(rc, "lbm_read_fields")
        return rho, ux, uy, T

    def reduce(self, stream=None):
        m = ctypes.c_double()
        h = ctypes.c_double()
        _check(self._lib.lbm_reduce(self._h, ctypes.byref(m), ctypes.byref(h),
                                    _stream_ptr(stream)), "lbm_reduce")
        return m.value, h.value

    def status(self, clear: bool = False, stream=None) -> int:
        bits = ctypes.c_uint()
        _check(self._lib.lbm_status(self._h, ctypes.byref(bits), int(clear), _stream_ptr(stream)),
               "lbm_status")
        return bits.value

    def read_state(self, stream=None) -> bytes:
        n = ctypes.c_size_t()
        _check(self._lib.lbm_state_bytes(self._h, ctypes.byref(n)), "lbm_state_bytes")
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.lbm_read_state(self._h, buf, n.value, _stream_ptr(stream)),
               "lbm_read_state")
        return buf.raw

    def write_state(self, data: bytes, stream=None):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(self._lib.lbm_write_state(self._h, buf, len(data), _stream_ptr(stream)),
               "lbm_write_state")

    def info(self) -> dict:
        inf = LbmInfo()
        _check(self._lib.lbm_info(self._h, ctypes.byref(inf)), "lbm_info")
        return {f[0]: getattr(inf, f[0]) for f in LbmInfo._fields_}

    @property
    def t(self) -> int:
        return self.info()["t"]

    @property
    def Tc(self) -> float:
        return self.info()["Tc"]

    # -- timing -------------------------------------------------------------
    def timing_enable(self, on: bool = True):
        _check(self._lib.lbm_timing_enable(self._h, int(on)), "lbm_timing_enable")

    def timing_get(self, stream=None) -> dict:
        n = 8
        names = (ctypes.c_char_p * n)()
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_long * n)()
        count = ctypes.c_int()
        _check(self._lib.lbm_timing_get(self._h, names, ms, cnt, n, ctypes.byref(count),
                                        _stream_ptr(stream)), "lbm_timing_get")
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(count.value, n))}


class Batch:
    """Lattices advanced together, one persistent launch per step (lbm_batch_*).

    The lattices stay owned by the caller and must outlive the batch."""

    def __init__(self, lattices, graph: bool = False, tile_rows: int | None = None):
        self._lib = load_library()
        self.lattices = list(lattices)
        arr = (ctypes.c_void_p * len(self.lattices))(*[l._h.value for l in self.lattices])
        h = ctypes.c_void_p()
        _check(self._lib.lbm_batch_create(arr, len(self.lattices), ctypes.byref(h)),
               "lbm_batch_create")
        self._h = h
        if graph:
            _check(self._lib.lbm_batch_set_graph(self._h, 1), "lbm_batch_set_graph")
        if tile_rows:
            _check(self._lib.lbm_batch_set_tile_rows(self._h, int(tile_rows)),
                   "lbm_batch_set_tile_rows")

    def step(self, nsteps: int = 1, stream=None):
        _check(self._lib.lbm_batch_step(self._h, int(nsteps), _stream_ptr(stream)),
               "lbm_batch_step")

    def autotune(self, steps_per_candidate: int = 4, stream=None) -> int:
        best = ctypes.c_int()
        _check(self._lib.lbm_batch_autotune(self._h, int(steps_per_candidate), ctypes.byref(best),
                                            _stream_ptr(stream)), "lbm_batch_autotune")
        return best.value

    def info(self) -> dict:
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lbm_batch_info(self._h, ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(c)), "lbm_batch_info")
        r, w, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lbm_batch_tiling(self._h, ctypes.byref(r), ctypes.byref(w),
                                          ctypes.byref(k)), "lbm_batch_tiling")
        return {"tiles": a.value, "grid": b.value, "tile_rows": c.value, "tile_cols": w.value,
                "cols_per_thread": k.value}

    def set_tiling(self, rows: int, cols: int, cols_per_thread: int = 1):
        _check(self._lib.lbm_batch_set_tiling(self._h, int(rows), int(cols),
                                              int(cols_per_thread)), "lbm_batch_set_tiling")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching job server (lbm_server_*): jobs are admitted by device
    footprint and advanced together in batched launches by a worker thread."""

    def __init__(self, hbm_budget: int, max_active: int = 64, chunk_steps: int = 500,
                 device: int = 0):
        self._lib = load_library()
        cfg = ServerConfig(device, int(hbm_budget), int(max_active), int(chunk_steps))
        h = ctypes.c_void_p()
        _check(self._lib.lbm_server_create(ctypes.byref(cfg), ctypes.byref(h)), "lbm_server_create")
        self._h = h
        self._shape = {}

    def submit(self, nx: int, ny: int, params: dict, nsteps: int, rho0=None,
               storage: int = STORAGE_F32, rho_ref: float = 0.0) -> int:
        p = make_params(params, kernel=KERNEL_FUSED, storage=storage, rho_ref=rho_ref)
        r = None
        if rho0 is not None:
            r = np.ascontiguousarray(rho0, dtype=np.float64).reshape(ny, nx)
        jid = ctypes.c_long()
        _check(self._lib.lbm_submit(self._h, int(nx), int(ny), ctypes.byref(p), _dptr(r),
                                    int(nsteps), ctypes.byref(jid)), "lbm_submit")
        self._shape[jid.value] = (ny, nx)
        return jid.value

    def poll(self, job_id: int, fields: bool = False):
        """(state, fields or None, latency seconds or None); non-blocking."""
        st = ctypes.c_int()
        lat = ctypes.c_double(-1.0)
        arrs = [None] * 4
        if fields:
            arrs = [np.empty(self._shape[job_id]) for _ in range(4)]
        _check(self._lib.lbm_poll(self._h, int(job_id), ctypes.byref(st),
                                  *[_dptr(a) for a in arrs], ctypes.byref(lat)), "lbm_poll")
        done = st.value == JOB_DONE
        return st.value, (tuple(arrs) if (fields and done) else None), (lat.value if done else None)

    def wait(self, job_id: int, timeout_s: float = 600.0) -> int:
        st = ctypes.c_int()
        rc = self._lib.lbm_wait(self._h, int(job_id), float(timeout_s), ctypes.byref(st))
        if rc not in (LBM_OK, -5):
            _check(rc, "lbm_wait")
        return st.value if rc == LBM_OK else -5

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._lib.lbm_server_stats(self._h, ctypes.byref(st)), "lbm_server_stats")
        return {f[0]: getattr(st, f[0]) for f in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
