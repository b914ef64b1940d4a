"""ctypes front end of the FP64 CPU oracle (``oracle/lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg load it; the CUDA library never does.  The C source restates
Sec. 2 of Mukherjee, Basu & Mondal (arXiv 2009.05264) node by node; this module
only marshals numpy arrays and a parameter mapping into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

GEOMETRY = {"periodic": 0, "channel": 1, "walls": 2, "pool": 3}
DIAG_NAMES = ("step", "mass", "energy", "rho_avg", "dp", "dtstar", "flux_in", "flux_out", "source",
              "vapor_area", "wall_vapor", "heater_vapor", "zone_vapor")


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("geometry", ctypes.c_int32),
        ("thermal", ctypes.c_int32),
        ("multiphase", ctypes.c_int32),
        ("tau_f", ctypes.c_double),
        ("tau_g", ctypes.c_double),
        ("a", ctypes.c_double),
        ("b", ctypes.c_double),
        ("R", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("c0", ctypes.c_double),
        ("G", ctypes.c_double),
        ("T0_R", ctypes.c_double),
        ("Tin_R", ctypes.c_double),
        ("dTheat_R", ctypes.c_double),
        ("u_in", ctypes.c_double),
        ("rho_out", ctypes.c_double),
        ("rho_w", ctypes.c_double),
        ("G_wet", ctypes.c_double),
        ("g_a", ctypes.c_double),
        ("c_v", ctypes.c_double),
        ("heater_x0", ctypes.c_int32),
        ("heater_len", ctypes.c_int32),
        ("heat_on_step", ctypes.c_int64),
        ("rho_vapor", ctypes.c_double),
        ("source_model", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
    ]


CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]


def compile_oracle(src: str, out: str) -> None:
    """gcc, plain -O2, no fast-math, no contraction; with OpenMP for the optional threaded
    loops where the compiler has it, else without (the pragmas are then ignored)."""
    try:
        subprocess.check_call(["gcc"] + CFLAGS + ["-fopenmp", "-o", out, src, "-lm"],
                              stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(["gcc"] + CFLAGS + ["-o", out, src, "-lm"])


def build(force: bool = False) -> str:
    """Compile liboracle.so from the C source."""
    hdr = os.path.join(_HERE, "lbm_oracle.h")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(hdr)):
        compile_oracle(_SRC, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER(OrcParams)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int32, ctypes.c_int32]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_init_fields.argtypes = [ctypes.c_void_p, P, dp, dp, dp, dp]
        L.orc_set_populations.argtypes = [ctypes.c_void_p, dp, dp, ctypes.c_int64, ctypes.c_double]
        L.orc_get_populations.argtypes = [ctypes.c_void_p, dp, dp]
        L.orc_get_step.restype = ctypes.c_int64
        L.orc_get_step.argtypes = [ctypes.c_void_p]
        L.orc_get_rho_avg_prev.restype = ctypes.c_double
        L.orc_get_rho_avg_prev.argtypes = [ctypes.c_void_p]
        L.orc_step.argtypes = [ctypes.c_void_p, P, ctypes.c_int64]
        L.orc_fields.argtypes = [ctypes.c_void_p, P, dp, dp, dp, dp, dp, dp]
        L.orc_last_diag.argtypes = [ctypes.c_void_p, dp]
        for name in ("orc_pressure", "orc_dpdT", "orc_psi"):
            fn = getattr(L, name)
            fn.restype = ctypes.c_double
            fn.argtypes = [P, ctypes.c_double, ctypes.c_double]
        L.orc_Tc.restype = ctypes.c_double
        L.orc_Tc.argtypes = [P]
        L.orc_maxwell.argtypes = [P, ctypes.c_double, dp, dp, dp]
        _lib = L
    return _lib


def make_params(p: dict) -> OrcParams:
    """Build the C parameter struct from a mapping of field name -> value."""
    s = OrcParams()
    for name, _ in OrcParams._fields_:
        v = p[name]
        if name == "geometry" and isinstance(v, str):
            v = GEOMETRY[v]
        setattr(s, name, v)
    return s


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


class Oracle:
    """One lattice of the oracle: post-stream populations f^n, g^n, shape (9, ny, nx)."""

    def __init__(self, nx: int, ny: int, params: dict, threads: int = 1):
        self.nx, self.ny = int(nx), int(ny)
        self.params = make_params(params)
        self._h = lib().orc_create(self.nx, self.ny)
        if not self._h:
            raise MemoryError("orc_create failed")
        if threads != 1 and lib().orc_set_threads(self._h, int(threads)) != 0:
            raise ValueError("threads must be >= 1")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_params(self, params: dict):
        self.params = make_params(params)

    def init_fields(self, rho, ux, uy, T=None):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.ny, self.nx) if a is not None else None
                for a in (rho, ux, uy, T)]
        st = lib().orc_init_fields(self._h, ctypes.byref(self.params), *[_ptr(a) for a in arrs])
        if st != 0:
            raise RuntimeError(f"orc_init_fields -> {st}")

    def set_populations(self, f, g=None, step=0, rho_avg_prev=None):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        g = None if g is None else np.ascontiguousarray(g, dtype=np.float64).reshape(9, self.ny, self.nx)
        if rho_avg_prev is None:
            rho_avg_prev = float(f.sum(axis=0).mean())
        lib().orc_set_populations(self._h, _ptr(f), _ptr(g), int(step), float(rho_avg_prev))

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        lib().orc_get_populations(self._h, _ptr(f), _ptr(g))
        return f, g

    @property
    def step_count(self) -> int:
        return int(lib().orc_get_step(self._h))

    @property
    def rho_avg_prev(self) -> float:
        return float(lib().orc_get_rho_avg_prev(self._h))

    def step(self, n: int = 1) -> int:
        """Advance n steps; returns the status (0 ok, 3 unstable)."""
        return int(lib().orc_step(self._h, ctypes.byref(self.params), int(n)))

    def fields(self):
        """dict of rho, ux, uy (actual velocity, Eq. 7), T, Fx, Fy, each (ny, nx)."""
        out = {k: np.empty((self.ny, self.nx)) for k in ("rho", "ux", "uy", "T", "Fx", "Fy")}
        st = lib().orc_fields(self._h, ctypes.byref(self.params),
                              *[_ptr(out[k]) for k in ("rho", "ux", "uy", "T", "Fx", "Fy")])
        out["status"] = int(st)
        return out

    def last_diag(self) -> dict:
        d = np.empty(len(DIAG_NAMES))
        lib().orc_last_diag(self._h, _ptr(d))
        return dict(zip(DIAG_NAMES, d.tolist()))


def Tc(params: dict) -> float:
    return float(lib().orc_Tc(ctypes.byref(make_params(params))))


def pressure(params: dict, rho: float, T: float) -> float:
    return float(lib().orc_pressure(ctypes.byref(make_params(params)), float(rho), float(T)))


def dpdT(params: dict, rho: float, T: float) -> float:
    return float(lib().orc_dpdT(ctypes.byref(make_params(params)), float(rho), float(T)))


def psi(params: dict, rho: float, T: float) -> float:
    return float(lib().orc_psi(ctypes.byref(make_params(params)), float(rho), float(T)))


def maxwell(params: dict, T: float):
    """(rho_v, rho_l, p_sat) by the equal-area construction on Eq. 12 at absolute T."""
    rv, rl, ps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib().orc_maxwell(ctypes.byref(make_params(params)), float(T), ctypes.byref(rv),
                           ctypes.byref(rl), ctypes.byref(ps))
    if st != 0:
        raise ValueError("no coexistence at this temperature")
    return rv.value, rl.value, ps.value
