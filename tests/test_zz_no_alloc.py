"""The allocation-free step (lbm_step_noalloc) against the context API.

lbm_step_noalloc serves callers that cannot allocate device memory: it runs the
same fused step on buffers the caller owns, with its scratch in a fixed array
inside the library.  Two consecutive calls must reproduce what a context's
lbm_step computes from the same state, within the parity tolerances of the
other GPU tests.  This file is collected last so that a run stopping at the first
failure has already run everything else; it also passes in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2009_05264_gb300 import inputs as I
from paper_2009_05264_gb300 import params as PP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def raw_state(lat, elt):
    """Storage-form populations (f, g) of a context, from its checkpoint blob
    (header, 9 planes of f, 9 of g, 1 of the density history)."""
    blob = lat.save_state()
    n = 9 * lat.nx * lat.ny
    hdr = len(blob) - (2 * n + lat.nx * lat.ny) * elt
    dt = np.float64 if elt == 8 else np.float32
    f = np.frombuffer(blob, dtype=dt, count=n, offset=hdr)
    g = np.frombuffer(blob, dtype=dt, count=n, offset=hdr + n * elt)
    return f.copy(), g.copy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_step_matches_context_step_twice(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05264_gb300 import lbm

    L = lbm.load()
    nx, ny = 257, 61  # several 120-column strips and bands, ragged in both directions
    p = PP.resolve(PP.default_params(geometry="channel", u_in=0.01, dTheat_R=0.08, heat_on_step=1, heater_x0=50,
                                     heater_len=30, g_a=2e-4), nx)
    Tc = oracle.Tc(p)
    fields = I.smooth_random(nx, ny, 5.95, 0.9 * Tc, seed=77, drho=0.002, du=0.005, dT=0.002)
    elt = 8 if prec == "fp64" else 4
    dt = torch.float64 if prec == "fp64" else torch.float32

    lat = lbm.Lattice(nx, ny, prec)
    lat.set_params(p)
    lat.init_fields(*fields)
    f0, g0 = raw_state(lat, elt)  # post-stream initial state in storage form
    rho_avg = float(np.ascontiguousarray(fields[0]).sum() / (nx * ny))

    cp = lbm.make_params(p, nx)
    prec_code = lbm.FP64 if prec == "fp64" else lbm.FP32
    dev = torch.device("cuda", 0)
    bufs = [torch.from_numpy(f0).to(dev), torch.from_numpy(g0).to(dev)]
    outs = [torch.empty(9 * nx * ny, dtype=dt, device=dev) for _ in range(2)]
    torch.cuda.synchronize()
    diag = np.zeros(len(lbm.DIAG_NAMES))
    for call in range(2):
        st = L.lbm_step_noalloc(ctypes.byref(cp), nx, ny, prec_code, ctypes.c_void_p(bufs[0].data_ptr()),
                                ctypes.c_void_p(bufs[1].data_ptr()), ctypes.c_void_p(outs[0].data_ptr()),
                                ctypes.c_void_p(outs[1].data_ptr()), 1 if call == 0 else 0, call, rho_avg,
                                diag.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
        assert st == 0, lbm.STATUS.get(st, st)
        lat.step(1)
        f_ref, g_ref = raw_state(lat, elt)
        f_got, g_got = outs[0].cpu().numpy(), outs[1].cpu().numpy()
        if prec == "fp64":
            scale_f, scale_g = np.abs(f_ref).max(), np.abs(g_ref).max()
        else:  # storage form is a deviation: compare against the full population scale
            scale_f, scale_g = p["rho_out"] / 9.0, 0.9 * Tc / 9.0
        assert np.abs(f_got - f_ref).max() < TOL[prec] * scale_f
        assert np.abs(g_got - g_ref).max() < TOL[prec] * scale_g
        d_ref = lat.diagnostics()
        assert diag[0] == d_ref["step"] == call
        assert diag[1] == pytest.approx(d_ref["mass"], rel=TOL[prec])
        assert diag[3] == pytest.approx(d_ref["rho_avg"], rel=TOL[prec])
        rho_avg = diag[3]
        bufs, outs = outs, bufs


def test_noalloc_rejects_oversized_and_aliased_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05264_gb300 import lbm

    L = lbm.load()
    p = PP.resolve(PP.default_params(geometry="channel"), 64)
    cp = lbm.make_params(p, 64)
    buf = torch.zeros(9 * 64 * 8, dtype=torch.float32, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    # output aliasing the input
    assert L.lbm_step_noalloc(ctypes.byref(cp), 64, 8, lbm.FP32, ptr, ptr, ptr, ptr, 1, 0, 5.95, None, None) == 1
    # more column strips than the scratch's tile table holds (checked before any device work)
    big = lbm.make_params(p, 1_000_000)
    assert L.lbm_step_noalloc(ctypes.byref(big), 1_000_000, 2, lbm.FP32, ptr, ptr, ctypes.c_void_p(1),
                              ctypes.c_void_p(1), 1, 0, 5.95, None, None) == 1
