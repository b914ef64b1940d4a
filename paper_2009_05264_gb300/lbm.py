"""Python binding of the pplbm C ABI (``include/pplbm.h``): argument marshalling only.

Every step of the lattice update runs in the CUDA library ``_lib/libpplbm.so``;
this module converts numpy arrays and parameter mappings to pointers and
sizes.  Device memory comes from PyTorch (one uint8 tensor per lattice, passed
to ``lbm_create_ex``) and work is ordered on PyTorch's current CUDA stream
unless another stream is given.  There is no CPU fallback: if the library
is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build
from .params import GEOMETRY, resolve

_lib = None

STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_EUNSTABLE", 4: "LBM_ETIMEOUT",
          5: "LBM_ECUDA", 6: "LBM_EBUDGET", 7: "LBM_ESTATE", 8: "LBM_EBOUNDS"}
FP32, FP64 = 0, 1
DIAG_NAMES = ("step", "mass", "energy", "rho_avg", "dp", "dtstar", "flux_in", "flux_out", "vapor_area",
              "wall_vapor", "heater_vapor", "zone_vapor")

# Every function the header declares (checked against the shared library's exports).
EXPORTS = (
    "lbm_default_params", "lbm_required_bytes", "lbm_create", "lbm_create_ex", "lbm_set_params",
    "lbm_init_fields", "lbm_step", "lbm_step_async", "lbm_sync", "lbm_read_fields", "lbm_get_populations",
    "lbm_set_populations", "lbm_read_diagnostics", "lbm_read_diagnostics_range", "lbm_state_bytes",
    "lbm_save_state", "lbm_load_state",
    "lbm_set_tiling", "lbm_autotune", "lbm_get_tiling", "lbm_default_band_plan", "lbm_set_kernel", "lbm_step_kernel",
    "lbm_set_step_loop", "lbm_step_loop", "lbm_set_wait_limit", "lbm_get_step", "lbm_launch_count", "lbm_get_stream",
    "lbm_critical_temperature",
    "lbm_destroy", "lbm_status_string", "lbm_last_error", "lbm_step_noalloc", "lbm_probe_fma_rate",
    "lbm_batch_create", "lbm_batch_add", "lbm_batch_remove", "lbm_batch_member", "lbm_batch_size",
    "lbm_batch_set_tiling", "lbm_batch_set_kernel", "lbm_batch_get_tiling", "lbm_batch_autotune", "lbm_batch_step",
    "lbm_batch_step_async", "lbm_batch_sync", "lbm_batch_set_step_loop", "lbm_batch_step_loop",
    "lbm_batch_set_wait_limit", "lbm_batch_read_fields", "lbm_batch_launch_count",
    "lbm_batch_get_stream", "lbm_batch_last_error", "lbm_batch_destroy",
)


KERNELS = {"auto": 0, "scalar": 1, "paired": 2, "tma": 3, "interior": 4}
KERNEL_NAMES = {v: k for k, v in KERNELS.items()}
LOOPS = {"auto": 0, "launches": 1, "persistent": 2}
LOOP_NAMES = {0: "auto", 1: "launches", 2: "persistent", 3: "overlapped"}


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint32), ("geometry", ctypes.c_int32), ("thermal", ctypes.c_int32),
        ("multiphase", ctypes.c_int32), ("tau_f", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double), ("omega", ctypes.c_double),
        ("beta", ctypes.c_double), ("c0", ctypes.c_double), ("G", ctypes.c_double), ("T0_R", ctypes.c_double),
        ("Tin_R", ctypes.c_double), ("dTheat_R", ctypes.c_double), ("u_in", ctypes.c_double),
        ("rho_out", ctypes.c_double), ("rho_w", ctypes.c_double), ("G_wet", ctypes.c_double),
        ("g_a", ctypes.c_double), ("c_v", ctypes.c_double), ("heater_x0", ctypes.c_int32),
        ("heater_len", ctypes.c_int32), ("heat_on_step", ctypes.c_int64), ("init_kind", ctypes.c_int32),
        ("reserved0", ctypes.c_int32), ("init_rho_in", ctypes.c_double), ("init_rho_out", ctypes.c_double),
        ("init_radius", ctypes.c_double), ("init_width", ctypes.c_double), ("perturb_amp", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("rho_vapor", ctypes.c_double), ("source_model", ctypes.c_int32),
        ("bubble_stats", ctypes.c_int32),
    ]


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True, path: str | None = None):
    """Load libpplbm.so (building it with nvcc first if needed).  `path` loads another build
    of the same library instead (the bounds-checked test build); the first load of a process
    fixes the library for the rest of it."""
    global _lib
    if _lib is not None:
        return _lib
    lib = path or _build.LIB
    if build_if_missing and path is None:
        _build.build()
    if not os.path.exists(lib):
        raise RuntimeError(f"CUDA library not built: {lib}")
    L = ctypes.CDLL(lib)
    vp, i32, i64, sz, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)
    P = ctypes.POINTER(LbmParams)
    sig = {
        "lbm_default_params": (None, [P]),
        "lbm_required_bytes": (sz, [i32, i32, ctypes.c_int]),
        "lbm_create": (ctypes.c_int, [ctypes.POINTER(vp), i32, i32, ctypes.c_int, i32, vp]),
        "lbm_create_ex": (ctypes.c_int, [ctypes.POINTER(vp), i32, i32, ctypes.c_int, i32, vp, vp, sz]),
        "lbm_set_params": (ctypes.c_int, [vp, P]),
        "lbm_init_fields": (ctypes.c_int, [vp, dp, dp, dp, dp, sz]),
        "lbm_step": (ctypes.c_int, [vp, i64]),
        "lbm_step_async": (ctypes.c_int, [vp, i64]),
        "lbm_sync": (ctypes.c_int, [vp]),
        "lbm_read_fields": (ctypes.c_int, [vp, dp, dp, dp, dp, sz]),
        "lbm_get_populations": (ctypes.c_int, [vp, dp, dp, sz]),
        "lbm_set_populations": (ctypes.c_int, [vp, dp, dp, sz, i64, ctypes.c_double]),
        "lbm_read_diagnostics": (ctypes.c_int, [vp, dp, sz]),
        "lbm_read_diagnostics_range": (ctypes.c_int, [vp, i64, i64, dp]),
        "lbm_state_bytes": (sz, [vp]),
        "lbm_save_state": (ctypes.c_int, [vp, vp, sz]),
        "lbm_load_state": (ctypes.c_int, [vp, vp, sz]),
        "lbm_set_tiling": (ctypes.c_int, [vp, i32, i32]),
        "lbm_set_kernel": (ctypes.c_int, [vp, i32]),
        "lbm_step_kernel": (i32, [vp]),
        "lbm_set_step_loop": (ctypes.c_int, [vp, i32]),
        "lbm_step_loop": (i32, [vp]),
        "lbm_set_wait_limit": (ctypes.c_int, [vp, i64]),
        "lbm_get_tiling": (ctypes.c_int, [vp] + [ctypes.POINTER(i32)] * 4),
        "lbm_autotune": (ctypes.c_int, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "lbm_default_band_plan": (ctypes.c_int, [i32, i32, i32, i64] + [ctypes.POINTER(i32)] * 3),
        "lbm_get_step": (i64, [vp]),
        "lbm_launch_count": (i64, [vp]),
        "lbm_get_stream": (vp, [vp]),
        "lbm_critical_temperature": (ctypes.c_double, [P]),
        "lbm_destroy": (ctypes.c_int, [vp]),
        "lbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "lbm_last_error": (ctypes.c_char_p, [vp]),
        "lbm_step_noalloc": (ctypes.c_int, [P, i32, i32, ctypes.c_int, vp, vp, vp, vp, i32, i64, ctypes.c_double,
                                            dp, vp]),
        "lbm_probe_fma_rate": (ctypes.c_int, [i32, i64, vp, dp]),
        "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, i32, i32, vp]),
        "lbm_batch_add": (ctypes.c_int, [vp, i32, i32, P, ctypes.POINTER(i32)]),
        "lbm_batch_remove": (ctypes.c_int, [vp, i32]),
        "lbm_batch_member": (vp, [vp, i32]),
        "lbm_batch_size": (i32, [vp]),
        "lbm_batch_set_tiling": (ctypes.c_int, [vp, i32, i32]),
        "lbm_batch_set_kernel": (ctypes.c_int, [vp, i32]),
        "lbm_batch_get_tiling": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "lbm_batch_autotune": (ctypes.c_int, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "lbm_batch_step": (ctypes.c_int, [vp, i64]),
        "lbm_batch_step_async": (ctypes.c_int, [vp, i64]),
        "lbm_batch_set_step_loop": (ctypes.c_int, [vp, i32]),
        "lbm_batch_step_loop": (i32, [vp]),
        "lbm_batch_set_wait_limit": (ctypes.c_int, [vp, i64]),
        "lbm_batch_sync": (ctypes.c_int, [vp, ctypes.POINTER(i32)]),
        "lbm_batch_read_fields": (ctypes.c_int, [vp, i32, dp, dp, dp, dp, sz]),
        "lbm_batch_launch_count": (i64, [vp]),
        "lbm_batch_get_stream": (vp, [vp]),
        "lbm_batch_last_error": (ctypes.c_char_p, [vp]),
        "lbm_batch_destroy": (ctypes.c_int, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def make_params(p: dict, nx: int) -> LbmParams:
    """C parameter struct from a parameter mapping (see params.default_params)."""
    q = resolve(p, nx)
    s = LbmParams()
    load().lbm_default_params(ctypes.byref(s))
    for name, _ in LbmParams._fields_:
        if name in ("size", "reserved0"):
            continue
        if name in q:
            v = q[name]
            if name == "geometry" and isinstance(v, str):
                v = GEOMETRY[v]
            setattr(s, name, v)
    return s


def critical_temperature(p: dict) -> float:
    return float(load().lbm_critical_temperature(ctypes.byref(make_params(p, 8))))


def default_band_plan(nx: int, ny: int, cols: int, slots: int) -> dict:
    """The library's default step tiling for `slots` CTA slots (host-only): per strip,
    tall_count bands of tall_rows, then bands of short_rows."""
    out = [ctypes.c_int32() for _ in range(3)]
    st = load().lbm_default_band_plan(int(nx), int(ny), int(cols), int(slots), *[ctypes.byref(o) for o in out])
    if st != 0:
        raise LbmError(st, "lbm_default_band_plan: invalid arguments")
    return {"tall_rows": out[0].value, "tall_count": out[1].value, "short_rows": out[2].value}


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(shape)


class Lattice:
    """One nx x ny lattice resident on a CUDA device."""

    def __init__(self, nx: int, ny: int, precision: str = "fp32", device: int = 0, stream=None,
                 torch_memory: bool = True):
        import torch  # device memory and streams

        self.nx, self.ny = int(nx), int(ny)
        self.precision = FP64 if precision in ("fp64", "f64", FP64) else FP32
        self.device = int(device)
        self._L = load()
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self._stream = stream
        sptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = ctypes.c_void_p()
        if torch_memory:
            nbytes = int(self._L.lbm_required_bytes(self.nx, self.ny, self.precision))
            if nbytes == 0:
                raise LbmError(1, "invalid lattice size")
            self._mem = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
            base = self._mem.data_ptr()
            aligned = (base + 255) // 256 * 256
            st = self._L.lbm_create_ex(ctypes.byref(h), self.nx, self.ny, self.precision, self.device, sptr,
                                       ctypes.c_void_p(aligned), nbytes)
        else:
            self._mem = None
            st = self._L.lbm_create(ctypes.byref(h), self.nx, self.ny, self.precision, self.device, sptr)
        if st != 0:
            raise LbmError(st, "lbm_create failed")
        self._h = h
        self.params = None

    # --- lifetime ---------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.lbm_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise LbmError(st, self._L.lbm_last_error(self._h).decode())

    # --- setup ------------------------------------------------------------
    def set_params(self, p: dict):
        self.params = dict(p)
        self._cparams = make_params(p, self.nx)
        self._check(self._L.lbm_set_params(self._h, ctypes.byref(self._cparams)))

    def init_fields(self, rho, ux, uy, T=None):
        shp = (self.ny, self.nx)
        a = [_f64(x, shp) for x in (rho, ux, uy, T)]
        self._check(self._L.lbm_init_fields(self._h, *[_dptr(x) for x in a], self.nx * self.ny))

    def set_tiling(self, cols: int, rows: int):
        self._check(self._L.lbm_set_tiling(self._h, int(cols), int(rows)))

    def set_kernel(self, kernel: str):
        """Step kernel form: "auto", "scalar", "interior", "paired" or "tma"."""
        self._check(self._L.lbm_set_kernel(self._h, KERNELS[kernel]))

    @property
    def step_kernel(self) -> str:
        """The kernel form the step launches take ("scalar", "interior", "paired" or "tma")."""
        return KERNEL_NAMES[int(self._L.lbm_step_kernel(self._h))]

    def set_step_loop(self, loop: str):
        """How multi-step calls run: "auto", "launches" (one launch per step) or "persistent"
        (one cooperative launch per call, bounded grid barriers between steps)."""
        self._check(self._L.lbm_set_step_loop(self._h, LOOPS[loop]))

    @property
    def step_loop(self) -> str:
        """The loop a multi-step call takes now: "launches", "persistent" (a barrier between
        steps) or "overlapped" (a persistent launch that overlaps consecutive steps)."""
        return LOOP_NAMES[int(self._L.lbm_step_loop(self._h))]

    def set_wait_limit(self, max_polls: int):
        """Polls before a persistent launch's barrier wait gives up (0: its 5 s time limit only)."""
        self._check(self._L.lbm_set_wait_limit(self._h, int(max_polls)))

    def autotune(self, trial_steps: int = 20) -> tuple[int, int]:
        """Time each candidate tiling for trial_steps steps and keep the fastest; returns
        (cols, rows), rows 0 for the default plan.  The trials advance the lattice."""
        c, r = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._L.lbm_autotune(self._h, int(trial_steps), ctypes.byref(c), ctypes.byref(r)))
        return c.value, r.value

    @property
    def tiling(self) -> dict:
        """The current step tiling: cols, and per strip tall_count bands of tall_rows, then
        bands of short_rows."""
        out = [ctypes.c_int32() for _ in range(4)]
        self._check(self._L.lbm_get_tiling(self._h, *[ctypes.byref(o) for o in out]))
        return dict(zip(("cols", "tall_rows", "tall_count", "short_rows"), (o.value for o in out)))

    # --- stepping ---------------------------------------------------------
    def step(self, n: int = 1):
        self._check(self._L.lbm_step(self._h, int(n)))

    def step_async(self, n: int = 1):
        self._check(self._L.lbm_step_async(self._h, int(n)))

    def sync(self):
        self._check(self._L.lbm_sync(self._h))

    @property
    def step_count(self) -> int:
        return int(self._L.lbm_get_step(self._h))

    @property
    def launches(self) -> int:
        return int(self._L.lbm_launch_count(self._h))

    @property
    def stream_handle(self) -> int:
        return int(self._L.lbm_get_stream(self._h) or 0)

    @property
    def stream(self):
        """The CUDA stream the lattice's kernels run on, as a torch stream (for events)."""
        import torch

        return torch.cuda.ExternalStream(self.stream_handle, device=torch.device("cuda", self.device))

    # --- readback ---------------------------------------------------------
    def fields(self, out: dict | None = None) -> dict:
        """rho, u_act (Eq. 7) and T of the current state as (ny, nx) float64 arrays.  `out`: the
        caller's arrays to fill (C-contiguous float64 of that shape, e.g. views of pinned host
        memory, which the device then writes directly); missing keys are not read."""
        keys = ("rho", "ux", "uy", "T")
        if out is None:
            out = {k: np.empty((self.ny, self.nx)) for k in keys}
        for k, a in out.items():
            if k not in keys or a.dtype != np.float64 or a.shape != (self.ny, self.nx) or not a.flags.c_contiguous \
                    or not a.flags.writeable:
                raise ValueError(f"out[{k!r}] must be a writeable C-contiguous float64 array of shape {(self.ny, self.nx)}")
        self._check(self._L.lbm_read_fields(self._h, *[_dptr(out.get(k)) for k in keys], self.nx * self.ny))
        return out

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        self._check(self._L.lbm_get_populations(self._h, _dptr(f), _dptr(g), f.size))
        return f, g

    def set_populations(self, f, g=None, step: int = 0, rho_avg_prev: float | None = None):
        shp = (9, self.ny, self.nx)
        f, g = _f64(f, shp), _f64(g, shp)
        r = float("nan") if rho_avg_prev is None else float(rho_avg_prev)
        self._check(self._L.lbm_set_populations(self._h, _dptr(f), _dptr(g), f.size, int(step), r))

    def diagnostics(self) -> dict:
        d = np.empty(len(DIAG_NAMES))
        self._check(self._L.lbm_read_diagnostics(self._h, _dptr(d), d.size))
        return dict(zip(DIAG_NAMES, d.tolist()))

    def diagnostics_range(self, first: int, count: int) -> np.ndarray:
        """Records of steps first .. first + count - 1 as a (count, len(DIAG_NAMES)) array
        (columns in DIAG_NAMES order); the context holds its last 1024 steps."""
        out = np.empty((int(count), len(DIAG_NAMES)))
        self._check(self._L.lbm_read_diagnostics_range(self._h, int(first), int(count), _dptr(out)))
        return out

    # --- checkpoint -------------------------------------------------------
    def save_state(self) -> bytes:
        n = int(self._L.lbm_state_bytes(self._h))
        buf = ctypes.create_string_buffer(n)
        self._check(self._L.lbm_save_state(self._h, buf, n))
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(self._L.lbm_load_state(self._h, buf, len(blob)))


class Member(Lattice):
    """A batch member: a lattice whose context the batch owns (never destroyed here)."""

    def __init__(self, batch, slot: int, nx: int, ny: int):
        self.nx, self.ny = int(nx), int(ny)
        self.precision = batch.precision
        self.device = batch.device
        self._L = batch._L
        self._h = ctypes.c_void_p(batch._L.lbm_batch_member(batch._h, slot))
        self._mem = None
        self._batch = batch  # keeps the batch (and so the context) alive
        self.slot = slot
        self.params = None

    def close(self):
        self._h = None

    def set_params(self, p: dict):
        raise LbmError(7, "a member's parameters are fixed when it is added to the batch")


class Batch:
    """Many independent lattices advanced by one fused launch per step (C ABI lbm_batch_*)."""

    def __init__(self, precision: str = "fp32", thermal: bool = True, device: int = 0, stream=None):
        self._L = load()
        self.precision = FP64 if precision in ("fp64", "f64", FP64) else FP32
        self.thermal = 1 if thermal else 0
        self.device = int(device)
        sptr = None
        if stream is not None:
            sptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = ctypes.c_void_p()
        st = self._L.lbm_batch_create(ctypes.byref(h), self.precision, self.thermal, self.device, sptr)
        if st != 0:
            raise LbmError(st, "lbm_batch_create failed")
        self._h = h
        self.members = {}

    def _check(self, st: int):
        if st != 0:
            raise LbmError(st, self._L.lbm_batch_last_error(self._h).decode())

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.members.clear()
            self._L.lbm_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, nx: int, ny: int, p: dict) -> Member:
        slot = ctypes.c_int32()
        self._check(self._L.lbm_batch_add(self._h, int(nx), int(ny), ctypes.byref(make_params(p, nx)),
                                          ctypes.byref(slot)))
        m = Member(self, slot.value, nx, ny)
        m.params = dict(p)
        self.members[slot.value] = m
        return m

    def remove(self, slot: int):
        self._check(self._L.lbm_batch_remove(self._h, int(slot)))
        m = self.members.pop(slot, None)
        if m is not None:
            m.close()  # its context is gone

    def __len__(self):
        return int(self._L.lbm_batch_size(self._h))

    def set_tiling(self, cols: int, rows: int = 0):
        self._check(self._L.lbm_batch_set_tiling(self._h, int(cols), int(rows)))

    def set_kernel(self, kernel: str):
        self._check(self._L.lbm_batch_set_kernel(self._h, KERNELS[kernel]))

    def set_step_loop(self, loop: str):
        """"auto", "launches" (graph-replayed launches, one per step) or "persistent"."""
        self._check(self._L.lbm_batch_set_step_loop(self._h, LOOPS[loop]))

    @property
    def step_loop(self) -> str:
        return LOOP_NAMES[int(self._L.lbm_batch_step_loop(self._h))]

    def set_wait_limit(self, max_polls: int):
        self._check(self._L.lbm_batch_set_wait_limit(self._h, int(max_polls)))

    @property
    def tiling(self):
        c, r = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._L.lbm_batch_get_tiling(self._h, ctypes.byref(c), ctypes.byref(r)))
        return c.value, r.value

    def autotune(self, trial_steps: int = 20):
        c, r = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._L.lbm_batch_autotune(self._h, int(trial_steps), ctypes.byref(c), ctypes.byref(r)))
        return c.value, r.value

    def step(self, n: int = 1):
        self.step_async(n)
        self.sync()

    def step_async(self, n: int = 1):
        self._check(self._L.lbm_batch_step_async(self._h, int(n)))

    def sync(self):
        slot = ctypes.c_int32(-1)
        st = self._L.lbm_batch_sync(self._h, ctypes.byref(slot))
        if st != 0:
            raise LbmError(st, f"member {slot.value}: " + self._L.lbm_batch_last_error(self._h).decode())

    @property
    def launches(self) -> int:
        return int(self._L.lbm_batch_launch_count(self._h))

    @property
    def stream(self):
        import torch

        return torch.cuda.ExternalStream(int(self._L.lbm_batch_get_stream(self._h) or 0),
                                         device=torch.device("cuda", self.device))


def probe_fma_rate(precision: str = "fp64", iters: int = 1 << 16, stream=None) -> float:
    """Fused multiply-add rate (flop/s, two per FMA) of independent FMA chains on the current
    device in "fp64" or "fp32" (the FP64 step's arithmetic roofline)."""
    L = load()
    out = ctypes.c_double(0.0)
    st = L.lbm_probe_fma_rate(1 if precision == "fp64" else 0, int(iters), stream, ctypes.byref(out))
    if st != 0:
        raise LbmError(st, "lbm_probe_fma_rate failed")
    return out.value
