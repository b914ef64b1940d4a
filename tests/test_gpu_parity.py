"""GPU parity: the fused CUDA step against the FP64 CPU oracle, element by element.

Tolerances: FP64 storage and arithmetic agree with the oracle to 1e-12
relative over 1000 steps (only rounding order and FMA contraction differ);
FP32 storage (deviations from the rest weights) and arithmetic agree to 1e-5
relative on rho and T and 1e-5 of the velocity scale on u.
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


def prm(nx, **kw):
    return PP.resolve(PP.default_params(**kw), nx)


def rel_err(got, ref, key):
    if key in ("ux", "uy"):
        scale = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max(), 1e-12)
    else:
        scale = np.abs(ref[key]).max()
    return np.abs(got[key] - ref[key]).max() / scale


def run_pair(nx, ny, p, fields, steps, precision="fp64", tiling=None, chunks=1, kernel="auto"):
    L = lbm()
    lat = L.Lattice(nx, ny, precision)
    lat.set_params(p)
    lat.set_kernel(kernel)
    if tiling:
        lat.set_tiling(*tiling)
    lat.init_fields(*fields)
    orc = oracle.Oracle(nx, ny, p)
    orc.init_fields(*fields)
    per = steps // chunks
    for _ in range(chunks):
        lat.step(per)
        assert orc.step(per) == 0
    return lat, orc


def channel_case(nx, ny, **kw):
    base = dict(geometry="channel", u_in=0.01, dTheat_R=0.08, heat_on_step=40, heater_x0=nx // 5,
                heater_len=max(3, nx // 10), g_a=2e-4)
    base.update(kw)
    p = prm(nx, **base)
    Tc = oracle.Tc(p)
    fields = I.smooth_random(nx, ny, 5.95, 0.9 * Tc, seed=nx * 131 + ny, drho=0.002, du=0.005, dT=0.002)
    return p, fields


@pytest.mark.parametrize("nx,ny,tiling", [(150, 37, (64, 5)), (150, 37, (128, 16)), (33, 17, (64, 4)),
                                          (6, 5, (64, 5))])
def test_fp64_channel_thermal_matches_oracle(nx, ny, tiling):
    p, fields = channel_case(nx, ny)
    lat, orc = run_pair(nx, ny, p, fields, 300, "fp64", tiling, chunks=3)
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < FP64_TOL, k
    fg, gg = lat.populations()
    fo, go = orc.populations()
    assert np.abs(fg - fo).max() < FP64_TOL * np.abs(fo).max()
    assert np.abs(gg - go).max() < FP64_TOL * np.abs(go).max()
    dg, do = lat.diagnostics(), orc.last_diag()
    for k in ("mass", "energy", "rho_avg", "flux_in", "flux_out"):
        assert dg[k] == pytest.approx(do[k], rel=1e-12, abs=1e-14), k
    assert dg["dp"] == pytest.approx(do["dp"], rel=1e-9, abs=1e-14)
    assert dg["dtstar"] == pytest.approx(do["dtstar"], rel=1e-9, abs=1e-12)
    assert dg["step"] == do["step"] == 299


def test_fp64_channel_1000_steps():
    nx, ny = 130, 24
    p, fields = channel_case(nx, ny, heat_on_step=300)
    lat, orc = run_pair(nx, ny, p, fields, 1000, "fp64", chunks=4)
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < FP64_TOL, k


def test_fp64_periodic_droplet_1000_steps():
    nx, ny = 70, 48
    p = prm(nx, geometry="periodic", thermal=0, g_a=0.0)
    T = 0.9 * oracle.Tc(p)
    rv, rl, _ = oracle.maxwell(p, T)
    fields = I.disk(nx, ny, 14, rl, rv, T, seed=2009052640, amp=1e-3)
    lat, orc = run_pair(nx, ny, p, fields, 1000, "fp64", (64, 8))
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy"):
        assert rel_err(got, ref, k) < FP64_TOL, k
    assert lat.diagnostics()["mass"] == pytest.approx(orc.last_diag()["mass"], rel=1e-13)


def test_fp64_walls_thermal_periodic_x():
    nx, ny = 90, 21
    p = prm(nx, geometry="walls", thermal=1, heat_on_step=10, heater_x0=80, heater_len=20, g_a=1e-4, rho_w=5.0,
            dTheat_R=0.1)
    Tc = oracle.Tc(p)
    fields = I.smooth_random(nx, ny, 5.95, 0.9 * Tc, seed=5, drho=0.002, du=0.005, dT=0.002)
    lat, orc = run_pair(nx, ny, p, fields, 200, "fp64", (64, 6))
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < FP64_TOL, k


def test_fp64_periodic_thermal_two_phase():
    nx, ny = 40, 40
    p = prm(nx, geometry="periodic", thermal=1, g_a=1e-4)
    T = 0.9 * oracle.Tc(p)
    rv, rl, _ = oracle.maxwell(p, T)
    fields = I.disk(nx, ny, 10, rl, rv, T, seed=9, amp=1e-3)
    lat, orc = run_pair(nx, ny, p, fields, 300, "fp64", (64, 7))
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < FP64_TOL, k


def test_fp64_single_phase_poiseuille():
    nx, ny = 100, 10
    p = prm(nx, geometry="channel", thermal=0, multiphase=0, g_a=0.0, u_in=0.016, rho_out=1.0)
    fields = I.uniform(nx, ny, 1.0, 0.0)
    lat, orc = run_pair(nx, ny, p, fields, 1000, "fp64")
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy"):
        assert rel_err(got, ref, k) < FP64_TOL, k


@pytest.mark.parametrize("kernel", ["paired", "scalar", "tma", "interior"])
@pytest.mark.parametrize("tiling", [(128, 16), (64, 4), (256, 37)])
def test_fp32_channel_thermal_1000_steps(tiling, kernel):
    nx, ny = 300, 37
    p, fields = channel_case(nx, ny, heat_on_step=200)
    lat, orc = run_pair(nx, ny, p, fields, 1000, "fp32", tiling, kernel=kernel)
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < FP32_TOL, k


def two_phase_errors(got, ref):
    """Pointwise errors of an FP32 two-phase field against the oracle, split into bulk nodes
    (density gradient below 1 % of its maximum) and interface nodes: density relative to its
    maximum, the interface displacement in lattice units (the density difference over the
    local gradient, regularised at the bulk edge), the relative L2 norms, and the velocity in
    lattice units (relative to the lattice speed dx/dt = 1) and relative to its own maximum."""
    gy, gx = np.gradient(ref["rho"])
    grad = np.hypot(gx, gy)
    bulk = grad < 0.01 * grad.max()
    diff = np.abs(got["rho"] - ref["rho"])
    du = np.maximum(np.abs(got["ux"] - ref["ux"]), np.abs(got["uy"] - ref["uy"]))
    u_max = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
    e = {"rho_bulk": diff[bulk].max() / np.abs(ref["rho"]).max(),
         "rho_interface": diff[~bulk].max() / np.abs(ref["rho"]).max(),
         "displacement": (diff[~bulk] / (grad[~bulk] + 0.1 * grad.max())).max(),
         "rho_L2": np.linalg.norm(got["rho"] - ref["rho"]) / np.linalg.norm(ref["rho"]),
         "rho_L2_shift": np.linalg.norm(got["rho"] - ref["rho"]) / np.linalg.norm(grad),
         "T": np.abs(got["T"] - ref["T"]).max() / np.abs(ref["T"]).max(),
         "T_L2": np.linalg.norm(got["T"] - ref["T"]) / np.linalg.norm(ref["T"]),
         "u_lattice": du.max(), "u_rel_max": du.max() / u_max, "u_max": u_max}
    print("FP32 two-phase errors: " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()))
    return e


def two_phase_fp32_checks(got, ref, lat_mass, orc_mass):
    """FP32 criteria where an interface is present: rounding noise moves an interface by a
    fraction of a lattice unit, and a pointwise difference there is that displacement times
    the density gradient; so bulk nodes keep the 1e-5 bound, interface nodes bound the
    displacement to 1e-3 lattice units, the density field differs in the L2 norm by no more
    than a rigid shift of the whole field by 1e-3 lattice units plus 1e-5 of the field, the
    temperature within 1e-5 in the relative L2 norm, and the velocity (in a drop only the
    spurious current) within 1e-5 in lattice units, i.e. relative to the lattice speed."""
    e = two_phase_errors(got, ref)
    assert e["rho_bulk"] < FP32_TOL
    assert e["displacement"] < 1e-3
    gy, gx = np.gradient(ref["rho"])
    assert (np.linalg.norm(got["rho"] - ref["rho"]) <
            1e-3 * np.linalg.norm(np.hypot(gx, gy)) + FP32_TOL * np.linalg.norm(ref["rho"]))
    assert e["T_L2"] < FP32_TOL
    assert e["u_lattice"] < FP32_TOL
    assert abs(lat_mass - orc_mass) < FP32_TOL * orc_mass
    return e


@pytest.mark.parametrize("kernel", ["paired", "scalar", "tma"])
def test_fp32_periodic_droplet_1000_steps(kernel):
    nx, ny = 64, 64
    p = prm(nx, geometry="periodic", thermal=0, g_a=0.0)
    T = 0.86 * oracle.Tc(p)
    p["T0_R"] = 0.86
    rv, rl, _ = oracle.maxwell(p, T)
    fields = I.disk(nx, ny, 25 * 64 / 128, rl, rv, T, seed=2009052640, amp=1e-3)
    p["init_rho_out"] = rl  # FP32 storage and pseudopotential reference: the liquid
    lat, orc = run_pair(nx, ny, p, fields, 1000, "fp32", kernel=kernel)
    got, ref = lat.fields(), orc.fields()
    two_phase_fp32_checks(got, ref, lat.diagnostics()["mass"], orc.last_diag()["mass"])


@pytest.mark.parametrize("kernel", ["paired", "scalar", "tma"])
def test_fp32_thermal_droplet_1000_steps(kernel):
    nx, ny = 40, 40
    p = prm(nx, geometry="periodic", thermal=1, g_a=1e-4)
    T = 0.9 * oracle.Tc(p)
    rv, rl, _ = oracle.maxwell(p, T)
    p["init_rho_out"] = rl
    fields = I.disk(nx, ny, 10, rl, rv, T, seed=9, amp=1e-3)
    lat, orc = run_pair(nx, ny, p, fields, 1000, "fp32", kernel=kernel)
    got, ref = lat.fields(), orc.fields()
    two_phase_fp32_checks(got, ref, lat.diagnostics()["mass"], orc.last_diag()["mass"])
    # flow here is buoyancy- and phase-change-driven, not only spurious currents
    for k in ("ux", "uy"):
        assert rel_err(got, ref, k) < 1e-4, k


@pytest.mark.parametrize("kernel", ["paired", "tma"])
@pytest.mark.parametrize("nx,ny,geometry,tiling", [(151, 37, "channel", (128, 16)), (57, 23, "channel", (64, 5)),
                                                   (63, 30, "walls", (128, 8)), (37, 41, "periodic", (64, 6)),
                                                   (245, 17, "walls", (128, 4)), (121, 30, "periodic", (128, 4)),
                                                   (3, 2, "channel", (128, 4))])
def test_fp32_kernel_odd_and_periodic_edges(nx, ny, geometry, tiling, kernel):
    """Edge cases of the paired and TMA step forms: an odd width (the last pair half
    outside the domain), open ends inside a pair or a staged box, wrap-around in
    periodic directions, a width that is an exact multiple of the 120-column tile
    plus a ragged tail, bands of 4 rows, and the smallest channel (3 x 2)."""
    if geometry == "channel":
        p, fields = channel_case(nx, ny, heat_on_step=20)
    else:
        p = prm(nx, geometry=geometry, thermal=1, g_a=1e-4, heater_x0=3, heater_len=7, heat_on_step=10)
        fields = I.smooth_random(nx, ny, 5.95, 0.9 * oracle.Tc(p), seed=nx + 7 * ny, drho=0.002, du=0.005, dT=0.002)
    lat, orc = run_pair(nx, ny, p, fields, 300, "fp32", tiling, kernel=kernel)
    if kernel == "tma" and tiling[0] == 128:
        assert lat.step_kernel == "tma"
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < FP32_TOL, k
    assert lat.diagnostics()["mass"] == pytest.approx(orc.last_diag()["mass"], rel=FP32_TOL)


def test_fp32_step_kernel_forms_agree():
    """The FP32 step forms compute the same update.  The TMA form does the scalar form's
    arithmetic in the same order within the same code (only the staging of the pulled
    populations differs), so their populations agree bit for bit; the paired form orders a
    few roundings differently and the interior path is compiled separately (the compiler
    may fuse a few multiply-adds differently), so after 200 steps they agree to ~1e-6."""
    L = lbm()
    nx, ny = 260, 41
    p, fields = channel_case(nx, ny, heat_on_step=10)
    pops = {}
    for kernel in ("paired", "scalar", "tma", "interior"):
        lat = L.Lattice(nx, ny, "fp32")
        lat.set_params(p)
        lat.set_kernel(kernel)
        assert lat.step_kernel == kernel
        lat.init_fields(*fields)
        lat.step(200)
        pops[kernel] = lat.populations()
    for a, b in zip(pops["paired"], pops["scalar"]):
        assert np.abs(a - b).max() < 1e-5 * np.abs(b).max()
    for a, b in zip(pops["tma"], pops["scalar"]):
        assert np.array_equal(a, b)
    for a, b in zip(pops["interior"], pops["scalar"]):
        assert np.abs(a - b).max() < 1e-5 * np.abs(b).max()
    assert L.load().lbm_set_kernel(lat._h, 7) == 1  # LBM_EINVAL


def test_step_kernel_resolution():
    """LBM_KERNEL_AUTO takes the interior form (the one-column kernel with its interior path)
    for the step's lean form and the scalar form for the full form; a TMA request takes the
    TMA form for a lean FP32 lattice on 128-column tiles and the scalar form where the TMA
    form does not apply."""
    L = lbm()
    nx, ny = 130, 20
    p, _ = channel_case(nx, ny)
    lat = L.Lattice(nx, ny, "fp32")
    lat.set_params(p)
    assert lat.step_kernel == "interior"
    lat.set_params(dict(p, bubble_stats=1))
    assert lat.step_kernel == "scalar"
    lat.set_params(p)
    lat.set_kernel("scalar")
    assert lat.step_kernel == "scalar"
    lat.set_kernel("tma")
    assert lat.step_kernel == "tma"
    lat.set_tiling(64, 8)
    assert lat.step_kernel == "scalar"
    assert lat.tiling == {"cols": 64, "tall_rows": 0, "tall_count": 0, "short_rows": 8}
    lat.set_tiling(128, 0)
    t = lat.tiling
    assert t["cols"] == 128 and t["tall_count"] * t["tall_rows"] < ny
    lat.set_params(dict(p, bubble_stats=1))  # full form
    assert lat.step_kernel == "scalar"
    lat.set_params(dict(p, source_model=1))
    assert lat.step_kernel == "scalar"
    lat.set_kernel("paired")
    assert lat.step_kernel == "scalar"  # no paired Hazi-Markus form
    lat.set_params(p)
    assert lat.step_kernel == "paired"
    lat64 = L.Lattice(nx, ny, "fp64")
    lat64.set_params(p)
    assert lat64.step_kernel == "interior"
    lat64.set_kernel("tma")
    assert lat64.step_kernel == "scalar"


@pytest.mark.parametrize("precision,slack", [("fp64", 1), ("fp32", 3)])
def test_bubble_diagnostics_match_oracle(precision, slack):
    """Vapour area and its wall / heater footprints of a heated sessile bubble, every
    50 steps, against the oracle's counts (node counts; FP32 may move a few interface
    nodes across the threshold)."""
    L = lbm()
    nx, ny, R = 90, 40, 14
    p = prm(nx, geometry="walls", thermal=1, g_a=5e-5, heater_x0=40, heater_len=10, heat_on_step=0, dTheat_R=0.3,
            bubble_stats=1)
    T = 0.9 * oracle.Tc(p)
    rv, rl, _ = oracle.maxwell(p, T)
    p["init_rho_out"] = rl
    fields = I.sessile(nx, ny, R, rv, rl, T)
    lat = L.Lattice(nx, ny, precision)
    lat.set_params(p)
    lat.init_fields(*fields)
    orc = oracle.Oracle(nx, ny, p)
    orc.init_fields(*fields)
    for _ in range(4):
        lat.step(25)
        assert orc.step(25) == 0
        got, ref = lat.diagnostics(), orc.last_diag()
        assert got["step"] == ref["step"]
        for k in ("vapor_area", "wall_vapor", "heater_vapor", "zone_vapor"):
            assert abs(got[k] - ref[k]) <= slack, (k, got[k], ref[k])
        assert ref["vapor_area"] > 250 and ref["heater_vapor"] > 0  # the bubble is still on the heater


def pool_case(nx, ny, seed=5, **kw):
    base = dict(geometry="pool", thermal=1, g_a=1e-4, heater_x0=nx // 2 - 3, heater_len=7, heat_on_step=20,
                dTheat_R=0.15, rho_out=5.9)
    base.update(kw)
    p = prm(nx, **base)
    p["init_rho_out"] = 5.9
    T = 0.9 * oracle.Tc(p)
    fields = I.smooth_random(nx, ny, 5.9, T, seed=seed, drho=0.002, du=0.005, dT=0.002)
    return p, fields


@pytest.mark.parametrize("tiling", [(128, 16), (64, 5)])
def test_fp64_pool_boiling_geometry_matches_oracle(tiling):
    """Sec. 2.D pool: periodic sides, heated bottom wall, constant-pressure top."""
    nx, ny = 130, 41
    p, fields = pool_case(nx, ny)
    lat, orc = run_pair(nx, ny, p, fields, 300, "fp64", tiling)
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "T"):
        assert rel_err(got, ref, k) < FP64_TOL, k
    # the pool's flow is weak (|u| < 1e-2, driven by the heater) and the top row's Zou-He is
    # solved in closed form here and as a moment system in the oracle: u agrees to a few
    # 1e-12 of its scale
    for k in ("ux", "uy"):
        assert rel_err(got, ref, k) < 5 * FP64_TOL, k
    d, r = lat.diagnostics(), orc.last_diag()
    assert d["mass"] == pytest.approx(r["mass"], rel=1e-13) and d["energy"] == pytest.approx(r["energy"], rel=1e-13)


@pytest.mark.parametrize("kernel", ["scalar", "paired"])
def test_fp32_pool_boiling_geometry_1000_steps(kernel):
    nx, ny = 121, 37
    p, fields = pool_case(nx, ny, seed=9)
    lat, orc = run_pair(nx, ny, p, fields, 1000, "fp32", (128, 12), kernel=kernel)
    got, ref = lat.fields(), orc.fields()
    # the heater thins the liquid to rho ~ 4.3 over a few nodes: the two-phase criteria apply
    two_phase_fp32_checks(got, ref, lat.diagnostics()["mass"], orc.last_diag()["mass"])
    for k in ("ux", "uy"):
        assert rel_err(got, ref, k) < 1e-4, k


@pytest.mark.parametrize("precision,steps,tol", [("fp64", 300, FP64_TOL), ("fp32", 1000, FP32_TOL)])
def test_hazi_markus_source_matches_oracle(precision, steps, tol):
    """First Eq. 19 with the temporal density gradient rho^n - rho^(n-1) (per-node history)."""
    nx, ny = 180, 37
    p, fields = channel_case(nx, ny, heat_on_step=30, source_model=1)
    lat, orc = run_pair(nx, ny, p, fields, steps, precision, (128, 12), kernel="paired")  # falls back to one column
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < tol, k
    # and it is not the Gong-Cheng result
    p0, _ = channel_case(nx, ny, heat_on_step=30)
    orc0 = oracle.Oracle(nx, ny, p0)
    orc0.init_fields(*fields)
    assert orc0.step(steps) == 0
    assert rel_err(orc0.fields(), ref, "T") > 100 * tol


def test_hazi_markus_checkpoint_resume_is_bitwise():
    L = lbm()
    nx, ny = 150, 30
    p, fields = channel_case(nx, ny, heat_on_step=10, source_model=1)
    lat = L.Lattice(nx, ny, "fp32")
    lat.set_params(p)
    lat.init_fields(*fields)
    lat.step(60)
    blob = lat.save_state()
    lat.step(40)
    a = lat.populations()
    lat.load_state(blob)
    lat.step(40)
    b = lat.populations()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_diagnostics_range_returns_every_step_record():
    L = lbm()
    nx, ny = 120, 30
    p, fields = channel_case(nx, ny, heat_on_step=5)
    lat = L.Lattice(nx, ny, "fp64")
    lat.set_params(p)
    lat.init_fields(*fields)
    orc = oracle.Oracle(nx, ny, p)
    orc.init_fields(*fields)
    ref = []
    for _ in range(40):
        assert orc.step(1) == 0
        ref.append(orc.last_diag())
    lat.step(40)
    rec = lat.diagnostics_range(0, 40)
    assert np.array_equal(rec[:, 0], np.arange(40))
    assert np.array_equal(rec[-1], np.array(list(lat.diagnostics().values())))
    names = L.DIAG_NAMES
    for k in ("mass", "energy", "dp", "dtstar", "flux_in", "flux_out"):
        got = rec[:, names.index(k)]
        want = np.array([r[k] for r in ref])
        assert np.abs(got - want).max() <= 1e-11 * max(np.abs(want).max(), 1e-300), k
    with pytest.raises(L.LbmError):
        lat.diagnostics_range(30, 20)  # step 49 not taken yet
    lat.step(1100)
    with pytest.raises(L.LbmError):
        lat.diagnostics_range(0, 10)  # older than the 1024-record ring
    assert lat.diagnostics_range(1140 - 1024, 1024).shape == (1024, len(names))


def test_tiling_does_not_change_results():
    """Per-node arithmetic does not depend on the band height: without buoyancy (no global
    sum in the update) every band height gives bit-identical populations for one column
    width.  Different column widths are separately compiled kernels and agree to rounding."""
    L = lbm()
    nx, ny = 200, 45
    p, fields = channel_case(nx, ny, g_a=0.0)
    runs = {}
    for tiling in [(128, 16), (128, 7), (128, 45), (64, 4), (64, 45), (256, 9)]:
        lat = L.Lattice(nx, ny, "fp32")
        lat.set_params(p)
        lat.set_tiling(*tiling)
        lat.init_fields(*fields)
        lat.step(100)
        runs[tiling] = lat.populations()
    for a, b in [((128, 16), (128, 7)), ((128, 16), (128, 45)), ((64, 4), (64, 45))]:
        assert np.array_equal(runs[a][0], runs[b][0]) and np.array_equal(runs[a][1], runs[b][1]), (a, b)
    ref = runs[(128, 16)]
    for t in [(64, 4), (256, 9)]:
        assert np.abs(runs[t][0] - ref[0]).max() < 1e-6 * np.abs(ref[0]).max()
        assert np.abs(runs[t][1] - ref[1]).max() < 1e-6 * np.abs(ref[1]).max()


def test_checkpoint_resume_is_bitwise():
    L = lbm()
    nx, ny = 90, 20
    for prec in ("fp32", "fp64"):
        p, fields = channel_case(nx, ny, heat_on_step=30)
        a = L.Lattice(nx, ny, prec)
        a.set_params(p)
        a.init_fields(*fields)
        a.step(60)
        blob = a.save_state()
        a.step(40)
        b = L.Lattice(nx, ny, prec)
        b.set_params(p)
        b.load_state(blob)
        assert b.step_count == 60
        b.step(40)
        fa, ga = a.populations()
        fb, gb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_set_populations_roundtrip_and_oracle_state_injection():
    """A state taken from the oracle mid-run, injected with its step and buoyancy mean,
    continues exactly like the oracle."""
    L = lbm()
    nx, ny = 64, 19
    p, fields = channel_case(nx, ny, heat_on_step=25)
    orc = oracle.Oracle(nx, ny, p)
    orc.init_fields(*fields)
    orc.step(20)
    f, g = orc.populations()
    lat = L.Lattice(nx, ny, "fp64")
    lat.set_params(p)
    lat.set_populations(f, g, step=orc.step_count, rho_avg_prev=orc.rho_avg_prev)
    f2, g2 = lat.populations()
    assert np.array_equal(f2, f) and np.array_equal(g2, g)
    lat.step(30)
    orc.step(30)
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < FP64_TOL, k


def test_builtin_disk_init_matches_input_generator():
    L = lbm()
    nx, ny = 100, 64
    p = prm(nx, geometry="periodic", thermal=0, g_a=0.0, init_kind=1, init_rho_in=5.88, init_rho_out=0.59,
            init_radius=20.0, init_width=2.0, perturb_amp=1e-3, seed=2009052640)
    lat = L.Lattice(nx, ny, "fp64")
    lat.set_params(p)
    rho = lat.fields()["rho"]
    T0 = p["T0_R"] * oracle.Tc(p)
    ref = I.disk(nx, ny, 20.0, 5.88, 0.59, T0, width=2.0, seed=2009052640, amp=1e-3)[0]
    assert np.abs(rho - ref).max() < 1e-13 * ref.max()


def test_unstable_state_is_reported_not_trapped():
    L = lbm()
    nx, ny = 40, 10
    p, fields = channel_case(nx, ny)
    rho = fields[0].copy()
    rho[5, 20] = 11.0  # beyond 1/b = 10.5: outside the Peng-Robinson domain
    lat = L.Lattice(nx, ny, "fp64")
    lat.set_params(p)
    lat.init_fields(rho, fields[1], fields[2], fields[3])
    with pytest.raises(L.LbmError) as e:
        lat.step(1)
    assert e.value.status == 3
    # the context stays usable
    lat.init_fields(*fields)
    lat.step(2)


def test_bad_arguments_are_rejected():
    L = lbm()
    lat = L.Lattice(20, 10, "fp32")
    with pytest.raises(L.LbmError):
        lat.step(1)  # no parameters yet
    p = prm(20, geometry="channel", tau_f=0.4)
    with pytest.raises(L.LbmError):
        lat.set_params(p)
    with pytest.raises(L.LbmError):
        lat.set_tiling(96, 8)
    small = L.Lattice(2, 10, "fp32")
    with pytest.raises(L.LbmError):
        small.set_params(prm(2, geometry="channel"))


@pytest.mark.parametrize("precision,steps,tol", [("fp32", 20, FP32_TOL), ("fp64", 10, FP64_TOL)])
def test_full_size_channel_against_oracle(precision, steps, tol):
    """8000 x 800 thermal channel in the benchmark's launch configuration (the default
    two-level band plan, the interior path on every tile away from the open ends, all steps in
    one overlapped persistent launch, tiles of consecutive steps in flight at once): 20 FP32 or
    10 FP64 fused steps compared with the oracle over every node, and every step's diagnostics
    record (the tiles' fixed-point totals) against the oracle's."""
    import os

    L = lbm()
    nx, ny = 8000, 800
    p = prm(nx, geometry="channel", u_in=0.03, dTheat_R=0.08, heater_x0=1600, heater_len=40, heat_on_step=1,
            rho_out=5.95)
    Tc = oracle.Tc(p)
    fields = I.smooth_random(nx, ny, 5.95, 0.9 * Tc, seed=2009052643, drho=0.002, du=0.005, dT=0.002)
    lat = L.Lattice(nx, ny, precision)
    lat.set_params(p)
    t = lat.tiling
    assert t["cols"] == 128 and t["tall_count"] > 0  # the two-level plan
    assert lat.step_kernel == "interior" and lat.step_loop == "overlapped"
    lat.init_fields(*fields)
    lat.step(steps)
    rec = lat.diagnostics_range(0, steps)
    col = {k: L.DIAG_NAMES.index(k) for k in ("step", "mass", "energy", "flux_in", "flux_out")}
    orc = oracle.Oracle(nx, ny, p, threads=os.cpu_count() or 1)
    orc.init_fields(*fields)
    flux_scale = p["rho_out"] * p["u_in"] * ny  # the inflow once developed; early records are small sums
    for n in range(steps):
        assert orc.step(1) == 0
        od = orc.last_diag()
        assert rec[n, col["step"]] == n
        for k in ("mass", "energy"):
            assert rec[n, col[k]] == pytest.approx(od[k], rel=tol), k
        for k in ("flux_in", "flux_out"):
            assert abs(rec[n, col[k]] - od[k]) < tol * flux_scale, k
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < tol, k


def test_fields_into_caller_arrays():
    """fields(out=...) fills the caller's arrays (here pinned host memory) with the same values
    as a fresh read, reads only the keys given, and rejects arrays of the wrong shape or type."""
    L = lbm()
    nx, ny = 70, 20
    p, fields = channel_case(nx, ny)
    lat = L.Lattice(nx, ny, "fp32")
    lat.set_params(p)
    lat.init_fields(*fields)
    lat.step(20)
    ref = lat.fields()
    pinned = {k: torch.empty((ny, nx), dtype=torch.float64).pin_memory().numpy() for k in ("rho", "T")}
    got = lat.fields(out=pinned)
    assert got is pinned and set(got) == {"rho", "T"}
    for k in got:
        assert np.array_equal(got[k], ref[k])
    with pytest.raises(ValueError):
        lat.fields(out={"rho": np.empty((nx, ny))})
    with pytest.raises(ValueError):
        lat.fields(out={"ux": np.empty((ny, nx), dtype=np.float32)})


def test_autotune_keeps_a_valid_tiling():
    """lbm_autotune times the candidate tilings, keeps the fastest and leaves a lattice that
    still steps in parity with the oracle after re-initialisation."""
    L = lbm()
    nx, ny = 150, 37
    p, fields = channel_case(nx, ny)
    lat = L.Lattice(nx, ny, "fp32")
    lat.set_params(p)
    lat.init_fields(*fields)
    cols, rows = lat.autotune(trial_steps=3)
    t = lat.tiling
    assert cols in (64, 128, 256) and t["cols"] == cols
    assert rows == 0 or (t["tall_count"] == 0 and t["short_rows"] == min(rows, ny))
    lat.init_fields(*fields)
    lat.step(200)
    orc = oracle.Oracle(nx, ny, p)
    orc.init_fields(*fields)
    assert orc.step(200) == 0
    got, ref = lat.fields(), orc.fields()
    for k in ("rho", "ux", "uy", "T"):
        assert rel_err(got, ref, k) < FP32_TOL, k


def test_fixed_point_totals_at_full_width():
    """The step's totals are 64-bit fixed point with 52 - ceil(log2 m) fraction bits, m the nodes
    feeding a total (nx ny for mass and energy, ny for the inlet and outlet fluxes).  On a
    4000 x 800 FP64 channel (30 and 42 fraction bits) the record of step n equals the exact sums
    over the fields the step starts from, within one grid step per tile plus FP64 rounding."""
    import math

    L = lbm()
    nx, ny = 4000, 800
    p, fields = channel_case(nx, ny)
    lat = L.Lattice(nx, ny, "fp64")
    lat.set_params(p)
    lat.init_fields(*fields)
    lat.step(5)
    f = lat.fields()
    lat.step(1)
    d = lat.diagnostics()
    assert d["step"] == 5
    ntiles_max = -(-nx // 56) * -(-ny // 4)  # the narrowest, shortest tiling

    def bound(m, size):
        frac_bits = 52 - math.ceil(math.log2(m))
        return ntiles_max * 2.0 ** -(frac_bits + 1) + 1e-14 * size

    mass, energy = math.fsum(f["rho"].ravel()), math.fsum(f["T"].ravel())
    assert abs(d["mass"] - mass) <= bound(nx * ny, mass)
    assert abs(d["energy"] - energy) <= bound(nx * ny, energy)
    for key, col in (("flux_in", 0), ("flux_out", nx - 1)):
        q = f["rho"][:, col] * f["ux"][:, col]
        want = math.fsum(q)
        assert abs(d[key] - want) <= bound(ny, float(np.abs(q).sum())), key
    lat.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_repeated_runs_are_bit_identical(precision):
    """The per-tile sums enter integer fixed-point totals, so the order in which the tiles of a
    launch finish (which varies from run to run) cannot change a record or, through the buoyancy
    mean, a population: two runs of the same lattice with the same tiling agree bit for bit."""
    L = lbm()
    nx, ny = 1000, 200
    p, fields = channel_case(nx, ny, heat_on_step=10)
    runs = []
    for _ in range(2):
        lat = L.Lattice(nx, ny, precision)
        lat.set_params(p)
        lat.set_tiling(64, 4)  # many small tiles: 18 strips x 50 bands = 900 per launch
        lat.init_fields(*fields)
        lat.step(60)
        f, g = lat.populations()
        runs.append((f, g, lat.diagnostics_range(0, 60)))
        lat.close()
    (f0, g0, r0), (f1, g1, r1) = runs
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    assert np.array_equal(r0, r1)
