"""The bounds-checked build (-DLBM_BOUNDS_CHECK) on every step form, on small and ragged lattices.

In that build every global access of the kernels checks its element index against the buffer it
addresses; an index outside it is skipped, counted and reported as LBM_EBOUNDS (nothing traps).
A child process that loads the checked library runs each kernel form (interior path, general
loop, paired columns, TMA staging, the persistent loop with a barrier and overlapped), each
geometry (channel, walls, periodic, pool), FP32 and FP64, thermal and isothermal, the
Hazi-Markus source and the bubble counters (the full form), 64-column tiles, a batch of uneven
members and the allocation-free step, on lattices whose tiles end raggedly (3 x 2 up to
3000 x 160), then reads fields and populations back.  No access may be rejected, and the
populations must equal the default build's to rounding (the two builds are compiled
separately).  A probe compiled from the kernel header with the flag shows that the check itself
rejects and counts an index outside its buffer without dereferencing it.
"""
import ctypes
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2009_05264_gb300 import build as B
from paper_2009_05264_gb300 import inputs as I
from paper_2009_05264_gb300 import params as PP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ROUNDING = {"fp64": 1e-12, "fp32": 1e-6}
STEPS = 25

# name, precision, geometry, nx, ny, parameter overrides, kernel form, step loop, tiling
CASES = [
    ("channel_fp32", "fp32", "channel", 150, 37, {}, "auto", "launches", None),
    ("channel_fp64", "fp64", "channel", 150, 37, {}, "auto", "launches", None),
    ("channel_3x2", "fp32", "channel", 3, 2, {}, "scalar", "launches", None),
    ("channel_64col", "fp32", "channel", 150, 37, {}, "auto", "launches", (64, 4)),
    ("walls_33x17", "fp32", "walls", 33, 17, {}, "auto", "launches", None),
    ("periodic_isothermal_16x8", "fp32", "periodic", 16, 8, {"thermal": 0, "g_a": 0.0}, "auto", "launches", None),
    ("periodic_6x5_fp64", "fp64", "periodic", 6, 5, {"g_a": 0.0}, "auto", "launches", None),
    ("pool_33x17", "fp32", "pool", 33, 17, {}, "auto", "launches", None),
    ("channel_paired", "fp32", "channel", 150, 37, {}, "paired", "launches", None),
    ("channel_tma", "fp32", "channel", 257, 37, {}, "tma", "launches", (128, 0)),
    ("channel_persistent", "fp32", "channel", 150, 37, {}, "auto", "persistent", None),
    ("channel_overlapped", "fp32", "channel", 3000, 160, {}, "auto", "persistent", (128, 4)),
    ("walls_overlapped_fp64", "fp64", "walls", 2600, 121, {}, "auto", "persistent", (128, 4)),
    ("channel_hazi_markus", "fp32", "channel", 150, 37, {"source_model": 1}, "auto", "launches", None),
    ("channel_bubbles_fp64", "fp64", "channel", 150, 37, {"bubble_stats": 1}, "auto", "launches", None),
]
BATCH = [(40, 12), (33, 17), (70, 9)]


def params_for(geometry, nx, extra):
    base = dict(geometry=geometry, u_in=0.02, dTheat_R=0.1, heat_on_step=5, heater_x0=nx // 3,
                heater_len=max(1, nx // 6), g_a=2e-4)
    base.update(extra)
    return PP.resolve(PP.default_params(**base), nx)


def fields_for(p, nx, ny, seed):
    return I.smooth_random(nx, ny, 5.95, 0.9 * oracle.Tc(p), seed=seed, drho=0.002, du=0.004, dT=0.002)


def run_cases(L):
    """Every case through the library L is bound to: populations and fields after STEPS steps."""
    out = {}
    for k, (name, prec, geometry, nx, ny, extra, kernel, loop, tiling) in enumerate(CASES):
        p = params_for(geometry, nx, extra)
        lat = L.Lattice(nx, ny, prec)
        lat.set_params(p)
        lat.set_kernel(kernel)
        lat.set_step_loop(loop)
        if tiling:
            lat.set_tiling(*tiling)
        lat.init_fields(*fields_for(p, nx, ny, 100 + k))
        lat.step(STEPS)
        f, g = lat.populations()
        out[name + ".f"], out[name + ".g"] = f, g
        out[name + ".rho"] = lat.fields()["rho"]
        out[name + ".kernel"] = np.array([kernel if kernel != "auto" else lat.step_kernel], dtype="U16")
        lat.close()
    b = L.Batch("fp32", thermal=True)
    members = []
    for k, (nx, ny) in enumerate(BATCH):
        p = params_for("channel", nx, {"u_in": 0.01 + 0.005 * k})
        m = b.add(nx, ny, p)
        m.init_fields(*fields_for(p, nx, ny, 200 + k))
        members.append(m)
    b.step(STEPS)
    for k, m in enumerate(members):
        out[f"batch{k}.f"], out[f"batch{k}.g"] = m.populations()
    b.close()
    out["noalloc.f"] = noalloc_step(L)
    return out


def noalloc_step(L):
    """Three allocation-free steps of a 33 x 17 channel from its initialised state (storage form)."""
    nx, ny = 33, 17
    p = params_for("channel", nx, {})
    lat = L.Lattice(nx, ny, "fp32")
    lat.set_params(p)
    lat.init_fields(*fields_for(p, nx, ny, 300))
    blob = lat.save_state()
    n = 9 * nx * ny
    hdr = len(blob) - (2 * n + nx * ny) * 4
    f0 = np.frombuffer(blob, dtype=np.float32, count=n, offset=hdr).copy()
    g0 = np.frombuffer(blob, dtype=np.float32, count=n, offset=hdr + 4 * n).copy()
    lib = L.load()
    cp = L.make_params(p, nx)
    dev = torch.device("cuda", 0)
    bufs = [torch.from_numpy(f0).to(dev), torch.from_numpy(g0).to(dev)]
    outs = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rho_avg = float(fields_for(p, nx, ny, 300)[0].sum() / (nx * ny))
    diag = np.zeros(len(L.DIAG_NAMES))
    torch.cuda.synchronize()
    for call in range(3):
        st = lib.lbm_step_noalloc(ctypes.byref(cp), nx, ny, L.FP32, ptr(bufs[0]), ptr(bufs[1]), ptr(outs[0]),
                                  ptr(outs[1]), 1 if call == 0 else 0, call, rho_avg,
                                  diag.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
        if st != 0:
            raise L.LbmError(st, "lbm_step_noalloc")
        rho_avg = diag[3]
        bufs, outs = outs, bufs
    return bufs[0].cpu().numpy()


def child_main(lib, out):
    from paper_2009_05264_gb300 import lbm as L

    L.load(path=lib)
    np.savez(out, **run_cases(L))


@pytest.fixture(scope="module")
def checked_run(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = B.build(bounds_check=True)
    out = str(tmp_path_factory.mktemp("bounds") / "checked.npz")
    code = ("import sys; sys.path[:0] = [{root!r}, {tests!r}]; import test_gpu_bounds as t; "
            "t.child_main({lib!r}, {out!r})").format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib, out=out)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(out))


def test_no_access_leaves_its_buffer_and_results_match_the_default_build(checked_run):
    from paper_2009_05264_gb300 import lbm as L

    ref = run_cases(L)
    assert set(ref) == set(checked_run)
    for key, want in ref.items():
        got = checked_run[key]
        if key.endswith(".kernel"):
            assert got[0] == want[0], key
            continue
        prec = "fp64" if "fp64" in key else "fp32"
        # storage-form FP32 populations are deviations from w_i rho_ref: the population scale is rho / 9
        scale = 5.95 / 9.0 if key.startswith("noalloc") else max(np.abs(want).max(), 1e-30)
        assert np.abs(got - want).max() <= ROUNDING[prec] * scale, key


PROBE = r'''
#define LBM_BOUNDS_CHECK
#include "lbm_kernels.cuh"
__global__ void probe(pplbm::InstState* st, int* out) {
  out[0] = pplbm::idx_ok(st, 0, 10);
  out[1] = pplbm::idx_ok(st, 9, 10);
  out[2] = pplbm::idx_ok(st, 10, 10);
  out[3] = pplbm::idx_ok(st, -1, 10);
  out[4] = pplbm::idx_ok(st, 1ll << 40, 10);
  out[5] = (int)st->status;
  out[6] = (int)st->bounds_hits;
}
extern "C" int run_probe(int* out) {
  pplbm::InstState* st = nullptr;
  if (cudaMalloc(&st, sizeof(pplbm::InstState)) != cudaSuccess) return -1;
  cudaMemset(st, 0, sizeof(pplbm::InstState));
  probe<<<1, 1>>>(st, out);
  const int e = (int)cudaDeviceSynchronize();
  cudaFree(st);
  return e;
}
'''


def test_the_check_rejects_and_counts_an_index_outside_its_buffer(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src, lib = tmp_path / "probe.cu", tmp_path / "libprobe.so"
    src.write_text(PROBE)
    subprocess.check_call([nvcc, "-shared", "-Xcompiler", "-fPIC", "-O3", "-std=c++17", "-gencode",
                           "arch=compute_103a,code=sm_103a", "-I", B.CSRC, "-I", os.path.join(ROOT, "include"),
                           "-o", str(lib), str(src)])
    P = ctypes.CDLL(str(lib))
    P.run_probe.argtypes = [ctypes.c_void_p]
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert P.run_probe(ctypes.c_void_p(out.data_ptr())) == 0
    got = out.cpu().numpy()
    assert list(got[:5]) == [1, 1, 0, 0, 0]  # the last element is in, one past it and below 0 are out
    assert got[5] == 4  # STATUS_BOUNDS
    assert got[6] == 3  # three rejected accesses counted
