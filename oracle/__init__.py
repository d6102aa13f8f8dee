"""Plain FP64 CPU oracle of the pseudopotential MRT-LBM lattice update.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product package never does.  The numerical work is in
``pplbm_oracle.c`` (Section 2 of arXiv:1803.01756, Eqs. 1-18, one whole-grid
loop nest per stage); this module only compiles it with gcc and marshals
arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pplbm_oracle.c")
_HDR = os.path.join(_HERE, "pplbm_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libpplbm_oracle.so")
_lock = threading.Lock()
_lib = None

X_PERIODIC, X_INLET_OUTLET, X_PRESSURE_INLET = 0, 1, 2
Y_PERIODIC, Y_WALLS = 0, 1


class OrcParams(ctypes.Structure):
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
        ("p_amp_frac", ctypes.c_double),
        ("T_top_left", ctypes.c_double), ("T_top_right", ctypes.c_double),
        ("top_iso_x0", ctypes.c_int), ("top_iso_x1", ctypes.c_int),
        ("bot_iso_x0", ctypes.c_int), ("bot_iso_x1", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction, so x86 and
    Arm hosts give identical results)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(OrcParams)
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        L.orc_critical_temperature.argtypes = [P]
        L.orc_critical_temperature.restype = ctypes.c_double
        L.orc_eos_pressure.argtypes = [P, ctypes.c_double, ctypes.c_double]
        L.orc_eos_pressure.restype = ctypes.c_double
        L.orc_eos_dpdt.argtypes = [P, ctypes.c_double, ctypes.c_double]
        L.orc_eos_dpdt.restype = ctypes.c_double
        L.orc_psi.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
        L.orc_psi.restype = ctypes.c_double
        L.orc_moment_matrix.argtypes = [ctypes.POINTER(ctypes.c_int)]
        L.orc_feq.argtypes = [ctypes.c_double] * 3 + [dp]
        L.orc_meq.argtypes = [ctypes.c_double] * 3 + [dp]
        L.orc_forcing_moments.argtypes = [ctypes.c_double] * 8 + [dp]
        L.orc_collide_node.argtypes = [P, dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, dp]
        L.orc_grad_periodic.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_lap_periodic.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, P]
        L.orc_create.restype = vp
        L.orc_destroy.argtypes = [vp]
        L.orc_set_fields.argtypes = [vp, dp, dp]
        L.orc_step.argtypes = [vp, ctypes.c_long]
        L.orc_fields.argtypes = [vp, dp, dp, dp, dp]
        L.orc_populations.argtypes = [vp, dp]
        L.orc_set_populations.argtypes = [vp, dp]
        L.orc_mass_heat.argtypes = [vp, dp, dp]
        L.orc_time.argtypes = [vp]
        L.orc_time.restype = ctypes.c_long
        L.orc_status.argtypes = [vp]
        L.orc_status.restype = ctypes.c_uint
        L.orc_energy_rhs.argtypes = [vp, dp, dp, dp, dp, dp]
        L.orc_inlet_density.argtypes = [P, ctypes.c_long]
        L.orc_inlet_density.restype = ctypes.c_double
        _lib = L
    return _lib


_PARAM_KEYS = [f[0] for f in OrcParams._fields_]


def make_params(d: dict) -> OrcParams:
    """Build the oracle's parameter struct from a plain dict (key ``lambda`` maps
    to the struct field ``lam``)."""
    p = OrcParams()
    for k, v in d.items():
        key = "lam" if k == "lambda" else k
        if key not in _PARAM_KEYS:
            raise KeyError(f"unknown parameter {k!r}")
        setattr(p, key, v)
    return p


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def critical_temperature(params: dict) -> float:
    return lib().orc_critical_temperature(ctypes.byref(make_params(params)))


def eos_pressure(params: dict, rho: float, T: float) -> float:
    return lib().orc_eos_pressure(ctypes.byref(make_params(params)), rho, T)


def eos_dpdt(params: dict, rho: float, T: float) -> float:
    return lib().orc_eos_dpdt(ctypes.byref(make_params(params)), rho, T)


def psi(params: dict, rho: float, T: float):
    neg = ctypes.c_int(0)
    v = lib().orc_psi(ctypes.byref(make_params(params)), rho, T, ctypes.byref(neg))
    return v, bool(neg.value)


def inlet_density(params: dict, t: int) -> float:
    return lib().orc_inlet_density(ctypes.byref(make_params(params)), t)


def moment_matrix() -> np.ndarray:
    M = (ctypes.c_int * 81)()
    lib().orc_moment_matrix(M)
    return np.array(list(M), dtype=np.int64).reshape(9, 9)


def feq(rho, ux, uy) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, _dp(out))
    return out


def meq(rho, ux, uy) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_meq(rho, ux, uy, _dp(out))
    return out


def forcing_moments(ux, uy, Fx, Fy, Fm2_over_psi2=0.0, theta=0.0, s_e=1.0, s_zeta=1.0):
    out = np.zeros(9)
    lib().orc_forcing_moments(ux, uy, Fx, Fy, Fm2_over_psi2, theta, s_e, s_zeta, _dp(out))
    return out


def collide_node(params: dict, f, Fx, Fy, Fm2_over_psi2=0.0) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(9)
    lib().orc_collide_node(ctypes.byref(make_params(params)), _dp(f), Fx, Fy,
                           Fm2_over_psi2, _dp(out))
    return out


def grad_periodic(phi: np.ndarray):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ny, nx = phi.shape
    gx = np.zeros_like(phi)
    gy = np.zeros_like(phi)
    lib().orc_grad_periodic(nx, ny, _dp(phi), _dp(gx), _dp(gy))
    return gx, gy


def lap_periodic(phi: np.ndarray):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ny, nx = phi.shape
    out = np.zeros_like(phi)
    lib().orc_lap_periodic(nx, ny, _dp(phi), _dp(out))
    return out


class Oracle:
    """One FP64 lattice of nx * ny fluid nodes (arrays are [ny][nx], row-major)."""

    def __init__(self, nx: int, ny: int, params: dict):
        self.nx, self.ny = nx, ny
        self.params = dict(params)
        self._p = make_params(params)
        self._h = lib().orc_create(nx, ny, ctypes.byref(self._p))
        if not self._h:
            raise ValueError("orc_create rejected the lattice size")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def Tc(self) -> float:
        return lib().orc_critical_temperature(ctypes.byref(self._p))

    def set_fields(self, rho0: np.ndarray, T: np.ndarray | None = None):
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64).reshape(self.ny, self.nx)
        Tp = None
        if T is not None:
            T = np.ascontiguousarray(T, dtype=np.float64).reshape(self.ny, self.nx)
            Tp = _dp(T)
        lib().orc_set_fields(self._h, _dp(rho0), Tp)

    def step(self, n: int = 1) -> int:
        return lib().orc_step(self._h, n)

    def fields(self):
        shp = (self.ny, self.nx)
        rho, ux, uy, T = (np.zeros(shp) for _ in range(4))
        lib().orc_fields(self._h, _dp(rho), _dp(ux), _dp(uy), _dp(T))
        return rho, ux, uy, T

    def populations(self) -> np.ndarray:
        f = np.zeros((9, self.ny, self.nx))
        lib().orc_populations(self._h, _dp(f))
        return f

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        lib().orc_set_populations(self._h, _dp(f))

    def mass_heat(self):
        m = ctypes.c_double()
        h = ctypes.c_double()
        lib().orc_mass_heat(self._h, ctypes.byref(m), ctypes.byref(h))
        return m.value, h.value

    def energy_rhs(self, rho, ux, uy, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.ny, self.nx)
                for a in (rho, ux, uy, T)]
        K = np.zeros((self.ny, self.nx))
        lib().orc_energy_rhs(self._h, *[_dp(a) for a in arrs], _dp(K))
        return K

    @property
    def t(self) -> int:
        return lib().orc_time(self._h)

    @property
    def status(self) -> int:
        return lib().orc_status(self._h)
