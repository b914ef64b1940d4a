"""Bounded device waits.  The persistent step loop: one cooperative launch per call, a
bounded grid barrier between steps, tiles drawn from a per-step counter; and the TMA step
form's bounded waits on its bulk-copied rows.

It runs the step kernel's tile body, so it must agree with one launch per step to rounding
(the two are compiled separately) and with the oracle at the parity tolerances, both where
every CTA holds one tile per step (a small channel, the case it is chosen for) and where the
CTAs draw several tiles per step.  Its barrier waits are bounded: with the poll limit set to
one poll, the first CTA to reach a barrier gives up while the others still work, the call
reports LBM_ETIMEOUT, nothing faults, and the context is usable again after a fresh
initialisation.
"""
import numpy as np
import pytest

import oracle
from paper_2009_05264_gb300 import inputs as I
from paper_2009_05264_gb300 import params as PP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
ROUNDING = {"fp64": 1e-12, "fp32": 1e-6}


def lbm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05264_gb300 import lbm as L

    return L


def channel(nx, ny, **kw):
    base = dict(geometry="channel", u_in=0.03, dTheat_R=0.08, heater_x0=nx // 5, heater_len=max(5, nx // 25),
                heat_on_step=20, g_a=5e-5)
    base.update(kw)
    p = PP.resolve(PP.default_params(**base), nx)
    fields = I.smooth_random(nx, ny, 5.95, 0.9 * oracle.Tc(p), seed=nx + ny, drho=0.002, du=0.005, dT=0.002)
    return p, fields


def run(L, nx, ny, p, fields, precision, loop, steps, tiling=None, calls=1):
    lat = L.Lattice(nx, ny, precision)
    lat.set_params(p)
    lat.set_step_loop(loop)
    if tiling:
        lat.set_tiling(*tiling)
    lat.init_fields(*fields)
    launches0 = lat.launches
    for _ in range(calls):
        lat.step(steps // calls)
    return lat, lat.launches - launches0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("nx,ny,tiling", [(400, 60, None), (1000, 100, (64, 4)), (2000, 160, (64, 4))])
def test_persistent_loop_agrees_with_one_launch_per_step(precision, nx, ny, tiling):
    L = lbm()
    p, fields = channel(nx, ny)
    steps = 120
    per, n_per = run(L, nx, ny, p, fields, precision, "persistent", steps, tiling, calls=3)
    ref, n_ref = run(L, nx, ny, p, fields, precision, "launches", steps, tiling)
    assert n_per == 3 and n_ref == steps  # one launch per call against one per step
    assert per.step_count == ref.step_count == steps
    f_p, g_p = per.populations()
    f_r, g_r = ref.populations()
    tol = ROUNDING[precision]
    assert np.abs(f_p - f_r).max() <= tol * np.abs(f_r).max()
    assert np.abs(g_p - g_r).max() <= tol * np.abs(g_r).max()
    rec_p, rec_r = per.diagnostics_range(0, steps), ref.diagnostics_range(0, steps)
    assert np.array_equal(rec_p[:, 0], rec_r[:, 0])
    for j in (1, 2, 3, 5, 6, 7):
        scale = max(np.abs(rec_r[:, j]).max(), 1e-300)
        assert np.abs(rec_p[:, j] - rec_r[:, j]).max() <= 100 * tol * scale, j


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_persistent_loop_matches_oracle(precision):
    L = lbm()
    nx, ny, steps = 300, 50, 1000
    p, fields = channel(nx, ny)
    lat = L.Lattice(nx, ny, precision)
    lat.set_params(p)
    lat.init_fields(*fields)
    assert lat.step_loop == "persistent"  # a small lattice: one wave of the persistent kernel
    lat.step(steps)
    orc = oracle.Oracle(nx, ny, p)
    orc.init_fields(*fields)
    assert orc.step(steps) == 0
    got, ref = lat.fields(), orc.fields()
    scale_u = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
    for k in ("rho", "ux", "uy", "T"):
        scale = scale_u if k in ("ux", "uy") else np.abs(ref[k]).max()
        assert np.abs(got[k] - ref[k]).max() < TOL[precision] * scale, k
    d, od = lat.diagnostics(), orc.last_diag()
    for k in ("mass", "energy", "flux_in", "flux_out"):
        assert d[k] == pytest.approx(od[k], rel=TOL[precision]), k


def test_barrier_timeout_is_reported_and_the_context_recovers():
    L = lbm()
    nx, ny = 1000, 100
    p, fields = channel(nx, ny)
    lat = L.Lattice(nx, ny, "fp32")
    lat.set_params(p)
    lat.set_step_loop("persistent")
    lat.set_tiling(64, 4)  # hundreds of CTAs: the first at a barrier cannot find all the others there
    lat.init_fields(*fields)
    lat.set_wait_limit(1)
    with pytest.raises(L.LbmError) as err:
        lat.step(20)
    assert err.value.status == 4  # LBM_ETIMEOUT
    # the device is still usable: the same context, initialised again, reproduces a fresh run
    lat.set_wait_limit(0)
    lat.init_fields(*fields)
    lat.step(30)
    fresh, _ = run(L, nx, ny, p, fields, "fp32", "persistent", 30, (64, 4))
    for a, b in zip(lat.populations(), fresh.populations()):
        assert np.array_equal(a, b)
    assert lat.diagnostics()["mass"] == fresh.diagnostics()["mass"]
    with pytest.raises(L.LbmError):
        lat.set_wait_limit(-1)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_persistent_batch_agrees_with_graph_replayed_launches(precision):
    """A batch of uneven channels advanced by one cooperative launch per call agrees with the
    same batch advanced by graph-replayed launches, member by member, to rounding."""
    L = lbm()
    sizes = [(300, 40), (170, 64), (520, 33)]
    runs = {}
    for loop in ("persistent", "launches"):
        b = L.Batch(precision, thermal=True)
        b.set_step_loop(loop)
        members = []
        for k, (nx, ny) in enumerate(sizes):
            p, fields = channel(nx, ny, u_in=0.01 + 0.01 * k)
            m = b.add(nx, ny, p)
            m.init_fields(*fields)
            members.append(m)
        assert b.step_loop == loop
        b.step(40)
        runs[loop] = [m.populations() for m in members]
        assert all(m.step_count == 40 for m in members)
        b.close()
    tol = ROUNDING[precision]
    for (fp, gp), (fr, gr) in zip(runs["persistent"], runs["launches"]):
        assert np.abs(fp - fr).max() <= tol * np.abs(fr).max()
        assert np.abs(gp - gr).max() <= tol * np.abs(gr).max()


def test_tma_row_wait_timeout_is_reported_and_the_context_recovers():
    """The TMA step form waits on mbarriers for its bulk-copied rows, each wait bounded.  With
    the poll limit at one poll a wait gives up while its row's copies are still in flight; the
    CTA lets them (and the next row's) land before it ends, the call reports LBM_ETIMEOUT, and
    the context, initialised again, reproduces a fresh run bit for bit."""
    L = lbm()
    nx, ny = 1000, 100
    p, fields = channel(nx, ny)

    def tma_lattice():
        lat = L.Lattice(nx, ny, "fp32")
        lat.set_params(p)
        lat.set_kernel("tma")
        lat.set_step_loop("launches")
        lat.set_tiling(128, 0)
        lat.init_fields(*fields)
        assert lat.step_kernel == "tma"
        return lat

    lat = tma_lattice()
    lat.step(1)  # the first step after an initialisation reads its own populations: no bulk copies
    lat.set_wait_limit(1)
    with pytest.raises(L.LbmError) as err:
        lat.step(5)
    assert err.value.status == 4  # LBM_ETIMEOUT
    lat.set_wait_limit(0)
    lat.init_fields(*fields)
    lat.step(20)
    fresh = tma_lattice()
    fresh.step(20)
    for a, b in zip(lat.populations(), fresh.populations()):
        assert np.array_equal(a, b)


# The overlapped form: tilings with more tiles than the persistent launch's CTAs (608 of the
# FP32 one-column kernel, 304 in FP64, on 152 SMs), 120-column strips of 4-row bands.
OVERLAP_CASES = [("channel", 3000, 160), ("walls", 2600, 120), ("periodic", 2500, 124)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("geometry,nx,ny", OVERLAP_CASES)
def test_overlapped_loop_agrees_with_one_launch_per_step(precision, geometry, nx, ny):
    """Tiles of consecutive steps in flight at once agree with one launch per step to rounding
    (the buoyancy mean differs by the rounding of one collision), records included."""
    L = lbm()
    p, fields = channel(nx, ny, geometry=geometry)
    steps = 120
    per, n_per = run(L, nx, ny, p, fields, precision, "persistent", steps, (128, 4), calls=3)
    assert per.step_loop == "overlapped"
    ref, n_ref = run(L, nx, ny, p, fields, precision, "launches", steps, (128, 4))
    assert n_per == 3 and n_ref == steps
    assert per.step_count == ref.step_count == steps
    tol = ROUNDING[precision]
    for a, b in zip(per.populations(), ref.populations()):
        assert np.abs(a - b).max() <= tol * np.abs(b).max()
    rec_p, rec_r = per.diagnostics_range(0, steps), ref.diagnostics_range(0, steps)
    assert np.array_equal(rec_p[:, 0], rec_r[:, 0])
    for j in (1, 2, 3, 4, 5, 6, 7):
        scale = max(np.abs(rec_r[:, j]).max(), 1e-300)
        assert np.abs(rec_p[:, j] - rec_r[:, j]).max() <= 100 * tol * scale, j


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_overlapped_loop_matches_oracle(precision):
    L = lbm()
    nx, ny, steps = 3000, 100, 400
    p, fields = channel(nx, ny)
    lat = L.Lattice(nx, ny, precision)
    lat.set_params(p)
    lat.set_step_loop("persistent")
    lat.set_tiling(128, 4)  # 625 tiles
    lat.init_fields(*fields)
    assert lat.step_loop == "overlapped"
    for _ in range(4):
        lat.step(steps // 4)
    orc = oracle.Oracle(nx, ny, p, threads=8)
    orc.init_fields(*fields)
    assert orc.step(steps) == 0
    got, ref = lat.fields(), orc.fields()
    scale_u = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
    for k in ("rho", "ux", "uy", "T"):
        scale = scale_u if k in ("ux", "uy") else np.abs(ref[k]).max()
        assert np.abs(got[k] - ref[k]).max() < TOL[precision] * scale, k
    d, od = lat.diagnostics(), orc.last_diag()
    for k in ("mass", "energy", "rho_avg", "dp", "flux_in", "flux_out"):
        assert d[k] == pytest.approx(od[k], rel=TOL[precision], abs=TOL[precision] * 1e-3), k


def test_overlapped_loop_timeout_is_reported_and_the_context_recovers():
    """With the poll limit at one poll the first tile that has to wait gives up; the launch
    ends without a fault, the call reports LBM_ETIMEOUT, and the context, initialised again,
    reproduces a fresh overlapped run bit for bit (the overlapped loop is deterministic)."""
    L = lbm()
    nx, ny = 3000, 160
    p, fields = channel(nx, ny)
    lat = L.Lattice(nx, ny, "fp32")
    lat.set_params(p)
    lat.set_step_loop("persistent")
    lat.set_tiling(128, 4)
    lat.init_fields(*fields)
    assert lat.step_loop == "overlapped"
    lat.set_wait_limit(1)
    with pytest.raises(L.LbmError) as err:
        lat.step(20)
    assert err.value.status == 4  # LBM_ETIMEOUT
    lat.set_wait_limit(0)
    lat.init_fields(*fields)
    lat.step(30)
    fresh, _ = run(L, nx, ny, p, fields, "fp32", "persistent", 30, (128, 4))
    for a, b in zip(lat.populations(), fresh.populations()):
        assert np.array_equal(a, b)
    assert lat.diagnostics()["mass"] == fresh.diagnostics()["mass"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_overlapped_batch_agrees_with_launches_and_the_oracle(precision):
    """A batch whose tiling needs several waves of CTAs (three channels and a walls lattice of
    uneven size, 120-column strips of 4-row bands) advanced by overlapped persistent launches
    agrees member by member with graph-replayed launches to rounding, and its first member with
    the oracle at the parity tolerance; members keep their own step counts."""
    L = lbm()
    sizes = [(2000, 160, "channel"), (1500, 120, "channel"), (1800, 90, "walls"), (1300, 140, "channel")]
    steps = 90
    runs = {}
    for loop in ("persistent", "launches"):
        b = L.Batch(precision, thermal=True)
        b.set_step_loop(loop)
        b.set_tiling(128, 4)
        members, cases = [], []
        for k, (nx, ny, geo) in enumerate(sizes):
            p, fields = channel(nx, ny, geometry=geo, u_in=0.01 + 0.005 * k)
            m = b.add(nx, ny, p)
            m.init_fields(*fields)
            members.append(m)
            cases.append((p, fields))
        if loop == "persistent":
            assert b.step_loop == "overlapped"
        for _ in range(3):
            b.step(steps // 3)
        runs[loop] = [(m.populations(), m.diagnostics_range(0, steps)) for m in members]
        assert all(m.step_count == steps for m in members)
        if loop == "persistent":
            nx, ny, _ = sizes[0]
            orc = oracle.Oracle(nx, ny, cases[0][0], threads=8)
            orc.init_fields(*cases[0][1])
            assert orc.step(steps) == 0
            got, ref = members[0].fields(), orc.fields()
            scale_u = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
            for key in ("rho", "ux", "uy", "T"):
                scale = scale_u if key in ("ux", "uy") else np.abs(ref[key]).max()
                assert np.abs(got[key] - ref[key]).max() < TOL[precision] * scale, key
        b.close()
    tol = ROUNDING[precision]
    for ((fp, gp), rp), ((fr, gr), rr) in zip(runs["persistent"], runs["launches"]):
        assert np.abs(fp - fr).max() <= tol * np.abs(fr).max()
        assert np.abs(gp - gr).max() <= tol * np.abs(gr).max()
        assert np.array_equal(rp[:, 0], rr[:, 0])
        for j in (1, 2, 3, 6, 7):
            scale = max(np.abs(rr[:, j]).max(), 1e-300)
            assert np.abs(rp[:, j] - rr[:, j]).max() <= 100 * tol * scale, j
