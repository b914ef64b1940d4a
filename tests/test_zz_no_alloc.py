"""The allocation-free step (lbm_step_noalloc) against the context API.

lbm_step_noalloc serves callers that cannot allocate device memory: it runs the
same fused step on buffers the caller owns, with its scratch in a fixed array
inside the library.  Three consecutive calls must reproduce what a context's
lbm_step computes from the same state, within the parity tolerances of the
other GPU tests, on each step form the call can take (thermal channel; isothermal
periodic box without g buffers; channel with the bubble counters, which selects the
step's full form), every diagnostics slot included; and every call after the first must
leave the device's free memory unchanged (the first may load the library's module,
which places the scratch array).  This file is collected last so
that a run stopping at the first failure has already run everything else; it also
passes in a fresh process.
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


def case(form, nx):
    if form == "channel":
        return PP.resolve(PP.default_params(geometry="channel", u_in=0.01, dTheat_R=0.08, heat_on_step=1,
                                            heater_x0=50, heater_len=30, g_a=2e-4), nx)
    if form == "periodic_isothermal":
        return PP.resolve(PP.default_params(geometry="periodic", thermal=0, g_a=0.0, rho_out=5.95), nx)
    if form == "channel_bubbles":  # a vapour pocket on the heater so that the counters are non-zero
        return PP.resolve(PP.default_params(geometry="channel", u_in=0.01, dTheat_R=0.2, heat_on_step=0,
                                            heater_x0=40, heater_len=40, g_a=2e-4, bubble_stats=1,
                                            rho_vapor=5.0), nx)
    raise ValueError(form)


@pytest.mark.parametrize("form", ["channel", "periodic_isothermal", "channel_bubbles"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_step_matches_context_step(prec, form):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05264_gb300 import lbm

    L = lbm.load()
    nx, ny = 257, 61  # several 120-column strips and bands, ragged in both directions
    p = case(form, nx)
    thermal = p["thermal"] == 1
    Tc = oracle.Tc(p)
    fields = I.smooth_random(nx, ny, 5.95, 0.9 * Tc, seed=77, drho=0.002, du=0.005, dT=0.002)
    if form == "channel_bubbles":
        y, x = np.mgrid[0:ny, 0:nx]
        fields[0][(np.hypot(x - 60.0, y - 2.0) < 8.0)] = 3.0
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
    bufs = [torch.from_numpy(f0).to(dev), torch.from_numpy(g0).to(dev) if thermal else None]
    outs = [torch.empty(9 * nx * ny, dtype=dt, device=dev), torch.empty(9 * nx * ny, dtype=dt, device=dev)
            if thermal else None]
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    torch.cuda.synchronize()
    diag = np.zeros(len(lbm.DIAG_NAMES))
    for call in range(3):
        free_before = torch.cuda.mem_get_info(dev)[0]
        st = L.lbm_step_noalloc(ctypes.byref(cp), nx, ny, prec_code, ptr(bufs[0]), ptr(bufs[1]), ptr(outs[0]),
                                ptr(outs[1]), 1 if call == 0 else 0, call, rho_avg,
                                diag.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
        free_after = torch.cuda.mem_get_info(dev)[0]
        assert st == 0, lbm.STATUS.get(st, st)
        if call > 0:  # nothing allocated on the device by this call (the first may load the module)
            assert free_before == free_after, (call, free_before, free_after)
        lat.step(1)
        f_ref, g_ref = raw_state(lat, elt)
        f_got = outs[0].cpu().numpy()
        if prec == "fp64":
            scale_f, scale_g = np.abs(f_ref).max(), np.abs(g_ref).max()
        else:  # storage form is a deviation: compare against the full population scale
            scale_f, scale_g = p["rho_out"] / 9.0, 0.9 * Tc / 9.0
        assert np.abs(f_got - f_ref).max() < TOL[prec] * scale_f
        if thermal:
            g_got = outs[1].cpu().numpy()
            assert np.abs(g_got - g_ref).max() < TOL[prec] * scale_g
        d_ref = lat.diagnostics()
        assert diag[0] == d_ref["step"] == call
        for k, name in enumerate(lbm.DIAG_NAMES[1:], start=1):
            if name.endswith("vapor") or name == "vapor_area":  # node counts: exact in FP64, a few in FP32
                slack = 0 if prec == "fp64" else 3
                assert abs(diag[k] - d_ref[name]) <= slack, name
            else:
                assert diag[k] == pytest.approx(d_ref[name], rel=TOL[prec], abs=TOL[prec] * 1e-3), name
        if form == "channel_bubbles":
            assert diag[lbm.DIAG_NAMES.index("vapor_area")] > 0
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
    # more column strips than the scratch's tile table holds (8192 strips of 120 columns): an
    # isothermal periodic row of 983161 nodes, with real input and output buffers of full size,
    # so that every pointer handed over is valid for the lattice it describes
    nx = 983161
    big = lbm.make_params(PP.resolve(PP.default_params(geometry="periodic", thermal=0, g_a=0.0), nx), nx)
    f_in = torch.zeros(9 * nx, dtype=torch.float32, device="cuda")
    f_out = torch.zeros(9 * nx, dtype=torch.float32, device="cuda")
    assert L.lbm_step_noalloc(ctypes.byref(big), nx, 1, lbm.FP32, ctypes.c_void_p(f_in.data_ptr()), None,
                              ctypes.c_void_p(f_out.data_ptr()), None, 1, 0, 5.95, None, None) == 1
