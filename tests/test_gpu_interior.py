"""The step kernel's interior path against its general loop and against the oracle.

Tiles away from the open ends and from any wrap in x take a loop without per-node boundary
logic (LBM_KERNEL_INTERIOR, the default form).  It states the general loop's arithmetic
expression for expression, but it is compiled separately, so the compiler may fuse a few
multiply-adds differently: populations and diagnostics records must agree with the scalar
form to rounding (1e-12 of the population scale in FP64, 1e-6 in FP32, after 60 steps) on
every geometry it serves (channel, walls), for every column width and band height,
including the first step after an initialisation (post-stream input).  Against the oracle
it keeps the parity tolerances of the other GPU tests on lattices wide enough that most
tiles take the interior path.
"""
import numpy as np
import pytest

import oracle
from paper_2009_05264_gb300 import inputs as I
from paper_2009_05264_gb300 import params as PP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05264_gb300 import lbm as L

    return L


def case(nx, ny, geometry, thermal=1, **kw):
    base = dict(geometry=geometry, thermal=thermal, u_in=0.02, dTheat_R=0.1, heat_on_step=5, heater_x0=nx // 3,
                heater_len=nx // 6, g_a=2e-4)
    base.update(kw)
    p = PP.resolve(PP.default_params(**base), nx)
    fields = I.smooth_random(nx, ny, 5.95, 0.9 * oracle.Tc(p), seed=nx * 7 + ny, drho=0.003, du=0.005, dT=0.003)
    return p, fields


def advance(L, nx, ny, p, fields, precision, kernel, tiling, steps):
    lat = L.Lattice(nx, ny, precision)
    lat.set_params(p)
    lat.set_kernel(kernel)
    if tiling:
        lat.set_tiling(*tiling)
    lat.init_fields(*fields)
    lat.step(steps)
    assert lat.step_kernel == kernel
    out = lat.populations(), lat.diagnostics_range(0, steps)
    lat.close()
    return out


ROUNDING = {"fp64": 1e-12, "fp32": 1e-6}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("geometry,thermal,nx,ny,tiling", [
    ("channel", 1, 611, 41, (128, 0)),   # default band plan, ragged last strip
    ("channel", 1, 611, 41, (64, 5)),
    ("channel", 1, 900, 23, (256, 9)),
    ("walls", 1, 500, 30, (128, 7)),     # periodic in x: interior tiles never wrap
    ("channel", 0, 487, 33, (128, 6)),   # isothermal two-phase step
    ("channel", 1, 371, 2, (128, 4)),    # two rows: both wall rows in one band
])
def test_interior_path_agrees_with_general_loop(precision, geometry, thermal, nx, ny, tiling):
    L = lbm()
    p, fields = case(nx, ny, geometry, thermal)
    steps = 60
    (f_i, g_i), rec_i = advance(L, nx, ny, p, fields, precision, "interior", tiling, steps)
    (f_s, g_s), rec_s = advance(L, nx, ny, p, fields, precision, "scalar", tiling, steps)
    tol = ROUNDING[precision]
    assert np.abs(f_i - f_s).max() <= tol * np.abs(f_s).max()
    assert np.abs(g_i - g_s).max() <= tol * np.abs(g_s).max()
    assert np.array_equal(rec_i[:, 0], rec_s[:, 0])  # step numbers
    for j in range(1, rec_s.shape[1]):
        scale = max(np.abs(rec_s[:, j]).max(), 1e-300)
        assert np.abs(rec_i[:, j] - rec_s[:, j]).max() <= 100 * tol * scale, j


@pytest.mark.parametrize("precision,tol,steps", [("fp64", FP64_TOL, 1000), ("fp32", FP32_TOL, 1000)])
def test_interior_path_matches_oracle(precision, tol, steps):
    L = lbm()
    nx, ny = 600, 40
    p, fields = case(nx, ny, "channel", heat_on_step=100)
    lat = L.Lattice(nx, ny, precision)
    lat.set_params(p)
    assert lat.step_kernel == "interior"
    lat.init_fields(*fields)
    orc = oracle.Oracle(nx, ny, p)
    orc.init_fields(*fields)
    lat.step(steps)
    assert orc.step(steps) == 0
    got, ref = lat.fields(), orc.fields()
    scale_u = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
    for k in ("rho", "ux", "uy", "T"):
        scale = scale_u if k in ("ux", "uy") else np.abs(ref[k]).max()
        err = np.abs(got[k] - ref[k]).max() / scale
        print(f"{precision} {k}: max error {err:.3e} of its scale")
        assert err < tol, k
    d, od = lat.diagnostics(), orc.last_diag()
    for k in ("mass", "energy", "dtstar", "flux_in", "flux_out"):
        assert d[k] == pytest.approx(od[k], rel=tol, abs=tol), k
