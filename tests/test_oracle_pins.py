"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/paper_values.json), closed forms (critical point,
Poiseuille flow, steady conduction), conservation laws, symmetry and the
continuum limit of the interaction force.  None needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2009_05264_gb300 import inputs as I
from paper_2009_05264_gb300 import params as PP

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def prm(nx=64, **kw):
    return PP.resolve(PP.default_params(**kw), nx)


def test_paper_constants_are_the_defaults():
    p = PP.default_params()
    for key in ("beta", "c0", "a", "b"):
        assert p[key] == pytest.approx(GOLD[key]["value"], rel=1e-15)
    assert p["omega"] == GOLD["omega_R134a"]["value"]
    assert p["T0_R"] == GOLD["T0_R"]["value"]
    # Eq. 10: g1 = 4 g2 with g1 = 2G, g2 = G/2 -> the wetting strength 18 G reproduces it with w_i
    assert (2.0 * p["G"]) / (0.5 * p["G"]) == GOLD["g1_over_g2"]["value"]


def test_critical_point_of_eq12():
    """At T = Tc the PR isotherm has (to the rounding of 0.0778 and 0.45724) a
    horizontal inflection at p_c = 0.0778 R Tc / b; a loop just below, none above."""
    p = prm()
    Tc = oracle.Tc(p)
    rho = np.linspace(0.05, 0.9 / p["b"], 20001)

    def slope(T):
        pr = np.array([oracle.pressure(p, r, T) for r in rho])
        return np.gradient(pr, rho), pr

    s, pr = slope(Tc)
    k = int(np.argmin(s))
    assert abs(s[k]) < 2e-3 * pr[k] / rho[k]          # dp/drho ~ 0 at the inflection
    pc = 0.0778 * p["R"] * Tc / p["b"]
    assert pr[k] == pytest.approx(pc, rel=2e-3)
    assert pr[k] / (rho[k] * p["R"] * Tc) == pytest.approx(0.3074, abs=3e-3)  # PR critical compressibility
    assert slope(0.98 * Tc)[0].min() < 0
    assert slope(1.02 * Tc)[0].min() > 0


def test_dpdT_matches_temperature_derivative():
    p = prm()
    Tc = oracle.Tc(p)
    for rho in (0.3, 0.59, 2.0, 5.9, 7.5):
        for TR in (0.7, 0.9, 1.2):
            T = TR * Tc
            h = 1e-6 * T
            num = (oracle.pressure(p, rho, T + h) - oracle.pressure(p, rho, T - h)) / (2 * h)
            assert oracle.dpdT(p, rho, T) == pytest.approx(num, rel=1e-7)


def test_psi_inverts_to_eos_pressure():
    """Eq. 11: the pseudopotential pressure c_s^2 rho + c0 g psi^2 / 2 is the EOS pressure."""
    p = prm()
    T = 0.9 * oracle.Tc(p)
    for rho in (0.2, 0.59, 3.0, 5.95, 8.0):
        psi = oracle.psi(p, rho, T)
        assert rho / 3 + p["c0"] * p["G"] * psi ** 2 / 2 == pytest.approx(oracle.pressure(p, rho, T), rel=1e-12)


@pytest.mark.parametrize("TR", [0.7, 0.8, 0.86, 0.9, 0.95])
def test_maxwell_equal_area(TR):
    """Coexistence: equal pressure and zero area of (p - p_sat) over specific volume,
    checked with an independent adaptive quadrature."""
    p = prm()
    T = TR * oracle.Tc(p)
    rv, rl, ps = oracle.maxwell(p, T)
    assert oracle.pressure(p, rv, T) == pytest.approx(ps, rel=1e-9)
    assert oracle.pressure(p, rl, T) == pytest.approx(ps, rel=1e-9)
    area, _ = integrate.quad(lambda v: oracle.pressure(p, 1.0 / v, T) - ps, 1.0 / rl, 1.0 / rv,
                             limit=400, epsabs=1e-14)
    scale = ps * (1.0 / rv - 1.0 / rl)
    assert abs(area) < 1e-6 * scale
    assert rv < rl


def test_maxwell_densities_match_paper_at_09Tc():
    p = prm()
    rv, rl, _ = oracle.maxwell(p, 0.9 * oracle.Tc(p))
    assert rl == pytest.approx(GOLD["rho_liquid_at_0.9Tc"]["value"], rel=0.02)
    assert rv == pytest.approx(GOLD["rho_vapour_at_0.9Tc"]["value"], rel=0.02)


def test_shan_chen_force_continuum_limit():
    """Eqs. 8-11: for a smooth density field the discrete force tends to
    -grad(p_EOS - c_s^2 rho) (the leading order is independent of beta)."""
    nx, ny = 256, 3
    p = prm(nx, geometry="periodic", thermal=0, g_a=0.0)
    T = 0.9 * oracle.Tc(p)
    x = np.arange(nx)
    k = 2 * np.pi / nx
    rho_x = 3.0 * (1.0 + 0.05 * np.sin(k * x))
    rho = np.tile(rho_x, (ny, 1))
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(rho, np.zeros_like(rho), np.zeros_like(rho), np.full_like(rho, T))
    F = O.fields()
    h = 1e-6
    dp_drho = np.array([(oracle.pressure(p, r + h, T) - oracle.pressure(p, r - h, T)) / (2 * h) for r in rho_x])
    expect = -(dp_drho - 1.0 / 3.0) * 3.0 * 0.05 * k * np.cos(k * x)
    err = np.abs(F["Fx"][1] - expect).max() / np.abs(expect).max()
    assert err < 5e-3
    assert np.abs(F["Fy"]).max() < 1e-15


def test_wetting_force_neutral_wall():
    """Eq. 15 with G_wet = 18 G and psi_w = psi(rho_w): with beta = 1 a wall whose
    false density equals the fluid's exerts exactly the force a fluid row would,
    so a uniform fluid feels no net force at the wall rows."""
    nx, ny = 8, 6
    rho0 = 2.5
    p = prm(nx, geometry="walls", thermal=0, g_a=0.0, beta=1.0, rho_w=rho0)
    T = p["T0_R"] * oracle.Tc(p)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.uniform(nx, ny, rho0, T))
    F = O.fields()
    assert np.abs(F["Fx"]).max() < 1e-14 and np.abs(F["Fy"]).max() < 1e-14
    # a denser false wall attracts the fluid (G < 0): force toward the bottom wall at row 0
    p2 = prm(nx, geometry="walls", thermal=0, g_a=0.0, beta=1.0, rho_w=4.0)
    O.set_params(p2)
    F2 = O.fields()
    assert (F2["Fy"][0] < 0).all() and (F2["Fy"][-1] > 0).all()


def test_uniform_rest_state_is_steady():
    nx, ny = 12, 10
    p = prm(nx, geometry="periodic", thermal=1)
    T = p["T0_R"] * oracle.Tc(p)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.uniform(nx, ny, 5.9, T))
    f0, g0 = O.populations()
    assert O.step(50) == 0
    f1, g1 = O.populations()
    assert np.abs(f1 - f0).max() < 1e-14 and np.abs(g1 - g0).max() < 1e-15


def _total_momentum(f):
    return (f * CX[:, None, None]).sum(), (f * CY[:, None, None]).sum()


def test_mass_and_momentum_conservation_periodic():
    """Streaming and BGK conserve mass; the exact-difference term adds F to the
    momentum and the total Shan-Chen, buoyancy (with the lagged mean) force of a
    periodic domain sums to zero, so total momentum is conserved too."""
    nx, ny = 48, 40
    p = prm(nx, geometry="periodic", thermal=0, g_a=1e-4)
    T = 0.9 * oracle.Tc(p)
    rv, rl, _ = oracle.maxwell(p, T)
    O = oracle.Oracle(nx, ny, p)
    rho, ux, uy, TT = I.disk(nx, ny, 12, rl, rv, T, seed=3, amp=1e-3)
    ux = 0.01 * I.unit_noise(nx, ny, 5)
    O.init_fields(rho, ux, uy, TT)
    f0, _ = O.populations()
    m0 = f0.sum()
    px0, py0 = _total_momentum(f0)
    assert O.step(400) == 0
    f1, _ = O.populations()
    assert abs(f1.sum() - m0) / m0 < 1e-13
    px1, py1 = _total_momentum(f1)
    assert abs(px1 - px0) < 1e-11 * m0 and abs(py1 - py0) < 1e-11 * m0
    d = O.last_diag()
    assert d["mass"] == pytest.approx(m0, rel=1e-13)


@pytest.mark.parametrize("source_model", [0, 1])
def test_energy_budget_equals_source(source_model):
    """Eq. 16 conserves sum g except for the source: in a periodic domain
    sum T^{n+1} - sum T^n = sum phi^n (either Eq. 19)."""
    nx, ny = 32, 24
    p = prm(nx, geometry="periodic", thermal=1, g_a=0.0, source_model=source_model)
    T = 0.9 * oracle.Tc(p)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.smooth_random(nx, ny, 5.5, T, seed=7, drho=0.02, du=0.02, dT=0.01))
    assert O.step(1) == 0
    for _ in range(20):
        e0 = O.last_diag()
        assert O.step(1) == 0
        e1 = O.last_diag()
        assert abs(e1["energy"] - e0["energy"] - e0["source"]) < 1e-13 * e0["energy"]
    assert abs(e0["source"]) > 1e-9  # the budget test is not vacuous


def test_hazi_markus_source_reduces_to_t_div_u_without_density_change():
    """First Eq. 19: phi = T/(rho^2 c_v) (dp/dT)_rho drho/dt + T div u.  On the first step
    after a state is injected rho^(n-1) = rho^n, so phi = T div u, which the second Eq. 19
    also gives when c_v -> infinity; once the density moves the two differ."""
    nx, ny = 30, 20
    fields = None
    out = {}
    for name, kw in (("hm", dict(source_model=1)), ("gc_inf", dict(source_model=0, c_v=1e300))):
        p = prm(nx, geometry="periodic", thermal=1, g_a=0.0, **kw)
        T = 0.9 * oracle.Tc(p)
        fields = I.smooth_random(nx, ny, 5.5, T, seed=21, drho=0.02, du=0.02, dT=0.01)
        O = oracle.Oracle(nx, ny, p)
        O.init_fields(*fields)
        assert O.step(1) == 0
        out[name] = (O.last_diag()["source"], O.populations())
        assert O.step(1) == 0
        out[name + "2"] = O.last_diag()["source"]
    # (rho^0 = sum f^eq(rho) equals the input density only to rounding, ~1e-16)
    assert out["hm"][0] == pytest.approx(out["gc_inf"][0], rel=1e-10)
    np.testing.assert_allclose(out["hm"][1][1], out["gc_inf"][1][1], rtol=1e-13, atol=1e-17)
    assert abs(out["hm2"] - out["gc_inf2"]) > 1e-6 * abs(out["gc_inf2"])  # drho/dt now acts


def test_both_sources_give_the_same_compression_heating_in_a_sound_wave():
    """The two Eq. 19 forms are one energy equation (with continuity, drho/dt = -rho div u
    to first order in a small-amplitude wave, where u . grad rho is second order): in a
    standing sound wave they heat and cool the liquid alike, and far more than T div u
    alone would."""
    nx, ny = 64, 4
    res = {}
    for name, kw in (("gc", dict(source_model=0)), ("hm", dict(source_model=1)),
                     ("no_work", dict(source_model=0, c_v=1e300))):
        p = prm(nx, geometry="periodic", thermal=1, g_a=0.0, **kw)
        T0 = 0.9 * oracle.Tc(p)
        x = np.arange(nx)[None, :] * np.ones((ny, 1))
        rho = 5.5 * (1 + 0.002 * np.sin(2 * np.pi * x / nx))
        O = oracle.Oracle(nx, ny, p)
        O.init_fields(rho, np.zeros_like(rho), np.zeros_like(rho), np.full_like(rho, T0))
        assert O.step(80) == 0
        res[name] = O.fields()["T"][0] - T0
    gc, hm = res["gc"], res["hm"]
    assert np.corrcoef(gc, hm)[0, 1] > 0.999
    assert np.linalg.norm(hm - gc) < 0.05 * np.linalg.norm(gc)
    assert np.abs(gc).max() > 10 * np.abs(res["no_work"]).max()


def test_poiseuille_profile():
    """Sec. 2.D, Fig. 4(a): single-phase duct flow at Re_in = 0.96 is parabolic with
    peak 1.5 times the mean at x = 8H; halfway bounce-back puts the walls at y = -1/2, H - 1/2."""
    H, nx = 10, 100
    tau = 1.0
    Re = GOLD["poiseuille_Re_in"]["value"]
    u_in = Re * ((tau - 0.5) / 3.0) / H
    p = prm(nx, geometry="channel", thermal=0, multiphase=0, g_a=0.0, u_in=u_in, rho_out=1.0, tau_f=tau)
    O = oracle.Oracle(nx, H, p)
    O.init_fields(*I.uniform(nx, H, 1.0, 0.0))
    assert O.step(4000) == 0
    F = O.fields()
    u = F["ux"][:, 8 * H]
    y = np.arange(H) + 0.5                      # node centres; walls at y = 0 and y = H
    shape = y * (H - y)                         # parabola vanishing at both halfway walls
    # the continuum peak-to-mean ratio 1.5, seen through sampling at H node centres
    sampled_ratio = GOLD["poiseuille_peak_to_mean"]["value"] * (shape.max() / (H * H / 4)) / (shape.mean() / (H * H / 6))
    assert u.max() / u.mean() == pytest.approx(sampled_ratio, rel=0.005)
    A = u.sum() / shape.sum()
    assert np.abs(u - A * shape).max() < 0.01 * u.max()
    # steady mass flux through the section equals the inflow
    flux_in = (F["rho"][:, 0] * F["ux"][:, 0]).sum()
    assert (F["rho"][:, 8 * H] * u).sum() == pytest.approx(flux_in, rel=1e-3)
    # developed-flow pressure gradient of plane Poiseuille flow: dp/dx = -12 mu u_mean / H^2
    pr = F["rho"][H // 2] / 3.0
    x0, x1 = 4 * H, 9 * H
    grad = (pr[x1] - pr[x0]) / (x1 - x0)
    mu = F["rho"][H // 2, (x0 + x1) // 2] * (tau - 0.5) / 3.0
    assert grad == pytest.approx(-12 * mu * u.mean() / H ** 2, rel=0.03)


def test_open_boundary_moments():
    """Zou-He (Sec. 2.C): after every step the inlet nodes carry velocity (u_in, 0)
    and the outlet nodes density rho_out with no transverse momentum, corners included."""
    nx, ny = 20, 9
    p = prm(nx, geometry="channel", thermal=1, u_in=0.03, rho_out=5.9)
    T = p["T0_R"] * oracle.Tc(p)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.smooth_random(nx, ny, 5.9, T, seed=11, drho=0.01, du=0.01, dT=0.01))
    for _ in range(3):
        assert O.step(1) == 0
        f, _ = O.populations()
        rho = f.sum(axis=0)
        jx = (f * CX[:, None, None]).sum(axis=0)
        jy = (f * CY[:, None, None]).sum(axis=0)
        np.testing.assert_allclose(jx[:, 0] / rho[:, 0], 0.03, rtol=0, atol=1e-14)
        np.testing.assert_allclose(jy[:, 0], 0.0, atol=1e-13)
        np.testing.assert_allclose(rho[:, -1], 5.9, rtol=1e-14)
        np.testing.assert_allclose(jy[:, -1], 0.0, atol=1e-13)
        # zero temperature gradient at the exit plane: T(nx-1) = T(nx-2) on every row
        Tn = O.populations()[1].sum(axis=0)
        np.testing.assert_allclose(Tn[:, -1], Tn[:, -2], rtol=1e-15)
        assert np.ptp(Tn[:, -2]) > 1e-6  # the outlet column is not uniform: the check has teeth


def test_source_divergence_is_exact_for_a_linear_velocity_field():
    """The source of the second Eq. 19 needs div u_act.  For u = (0, a (y - y_m)) between
    walls every row, the two next to the walls included, must see div u = a exactly, so
    with an ideal-gas EOS ((dp/dT)_rho = 0, phi = T div u) the step's total source is
    a T nx ny."""
    nx, ny, a = 6, 12, 1e-3
    p = prm(nx, geometry="walls", thermal=1, multiphase=0, g_a=0.0, heater_len=0)
    T = 0.9 * oracle.Tc(p)
    rho, ux, uy, TT = I.uniform(nx, ny, 1.0, T)
    uy = a * (np.arange(ny, dtype=np.float64)[:, None] - 0.5 * (ny - 1)) * np.ones((1, nx))
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(rho, ux, uy, TT)
    assert O.step(1) == 0
    assert O.last_diag()["source"] == pytest.approx(a * T * nx * ny, rel=1e-12)


def test_thermal_liquid_between_walls_is_quiet():
    """A saturated liquid at rest between isothermal walls (Sec. 2.C) with a small seeded
    perturbation relaxes: its velocity decays instead of growing into a wall mode."""
    nx, ny = 8, 40
    p = prm(nx, geometry="walls", thermal=1, g_a=0.0, heater_len=0)
    Tc = oracle.Tc(p)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.smooth_random(nx, ny, 5.95, 0.9 * Tc, seed=7, drho=0.002, du=0.005, dT=0.002))
    amp = []
    for _ in range(3):
        assert O.step(2000) == 0
        amp.append(np.abs(O.fields()["uy"]).max())
    assert amp[2] < amp[1] < amp[0] < 1e-6


def test_vapour_diagnostics_count_the_bubble():
    """Bubble area, its footprint on the bottom wall and over the heater (Sec. 3.A,
    Figs. 7-8) are node counts of rho < rho_vapor; the first step's record counts the
    moments of the initial state, i.e. exactly the input field."""
    nx, ny, R = 60, 30, 11
    p = prm(nx, geometry="walls", thermal=1, g_a=0.0, heater_x0=25, heater_len=7, heat_on_step=0)
    T = 0.9 * oracle.Tc(p)
    rv, rl, _ = oracle.maxwell(p, T)
    fields = list(I.sessile(nx, ny, R, rv, rl, T))  # a vapour half-disk on the bottom wall
    fields[0] = fields[0].copy()
    fields[0][1, 2:5] = rv  # vapour on the second row only, away from the heater: wall rows differ
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*fields)
    assert O.step(1) == 0
    d = O.last_diag()
    vap = fields[0] < p["rho_vapor"]
    assert d["vapor_area"] == vap.sum() and d["wall_vapor"] == vap[0].sum() != vap[1].sum()
    assert d["heater_vapor"] == vap[0, 25:32].sum()
    assert d["zone_vapor"] == vap[:, 18:39].sum()
    assert 0.4 * np.pi * R * R < d["vapor_area"] < 0.6 * np.pi * R * R and d["heater_vapor"] == 7


def test_steady_conduction_between_walls():
    """With u = 0 anti-bounce-back (Sec. 2.C) and g^eq (Eq. 18) reduce to pure
    diffusion: the steady profile between a heated bottom wall at y = -1/2 and the
    top wall at y = ny - 1/2 is linear."""
    nx, ny = 4, 16
    p = prm(nx, geometry="walls", thermal=1, multiphase=0, g_a=0.0, heater_x0=0, heater_len=nx,
            heat_on_step=0, dTheat_R=0.1, tau_g=0.8)
    Tc = oracle.Tc(p)
    Tin, Th = p["Tin_R"] * Tc, (p["Tin_R"] + p["dTheat_R"]) * Tc
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.uniform(nx, ny, 1.0, Tin))
    assert O.step(12000) == 0
    T = O.fields()["T"][:, 0]
    y = np.arange(ny) + 0.5
    expect = Th + (Tin - Th) * y / ny
    assert np.abs(T - expect).max() < 1e-9 * (Th - Tin)


def test_heater_switch_on_timing():
    """The heater superheat enters the boundary condition of step heat_on_step,
    so the row above it warms first in the state after that step."""
    nx, ny = 6, 5
    p = prm(nx, geometry="walls", thermal=1, multiphase=0, g_a=0.0, heater_x0=0, heater_len=nx,
            heat_on_step=5, dTheat_R=0.1)
    Tin = p["Tin_R"] * oracle.Tc(p)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.uniform(nx, ny, 1.0, Tin))
    O.step(5)
    assert np.abs(O.fields()["T"] - Tin).max() < 1e-15
    O.step(1)
    T = O.fields()["T"]
    assert (T[0] > Tin + 1e-6).all() and np.abs(T[1:] - Tin).max() < 1e-15


def test_flat_interface_coexistence():
    """Sec. 2.D, Fig. 4(b): flat-interface densities follow the Maxwell
    construction for T_R >= 0.7 (within a few per cent for this force scheme)."""
    nx, ny = 4, 96
    p = prm(nx, geometry="periodic", thermal=0, g_a=0.0)
    T = 0.9 * oracle.Tc(p)
    rv, rl, _ = oracle.maxwell(p, T)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.slab(nx, ny, 24, rl, rv, T))
    assert O.step(12000) == 0
    rho = O.fields()["rho"][:, 0]
    assert rho.max() == pytest.approx(rl, rel=0.04)
    assert rho.min() == pytest.approx(rv, rel=0.04)
    assert rho.max() == pytest.approx(GOLD["rho_liquid_at_0.9Tc"]["value"], rel=0.04)
    assert rho.min() == pytest.approx(GOLD["rho_vapour_at_0.9Tc"]["value"], rel=0.04)


@pytest.mark.slow
def test_laplace_law():
    """Static droplets: the pressure jump is linear in 1/R with vanishing intercept."""
    nx = ny = 64
    p = prm(nx, geometry="periodic", thermal=0, g_a=0.0)
    T = 0.9 * oracle.Tc(p)
    rv, rl, _ = oracle.maxwell(p, T)
    inv_r, dps = [], []
    for R in (10.0, 13.0, 16.0, 20.0):
        O = oracle.Oracle(nx, ny, p)
        O.init_fields(*I.disk(nx, ny, R, rl, rv, T))
        assert O.step(3000) == 0
        rho = O.fields()["rho"]
        p_in = oracle.pressure(p, rho[ny // 2, nx // 2], T)
        p_out = oracle.pressure(p, rho[0, 0], T)
        # effective radius from the liquid area
        area = ((rho - rho.min()) / (rho.max() - rho.min())).sum()
        inv_r.append(1.0 / math.sqrt(area / math.pi))
        dps.append(p_in - p_out)
    slope, icpt = np.polyfit(inv_r, dps, 1)
    fit = np.polyval([slope, icpt], inv_r)
    assert slope > 0
    assert np.abs(fit - dps).max() < 0.03 * max(dps)
    assert abs(icpt) < 0.1 * max(dps)


@pytest.mark.slow
def test_bubble_rises_under_buoyancy():
    """Eq. 14: with gravity along -y the lighter vapour bubble moves up
    (a bubble well above the critical size of a closed box, so it neither condenses nor drifts)."""
    nx, ny = 48, 80
    p = prm(nx, geometry="periodic", thermal=0, g_a=2e-4)
    T = 0.9 * oracle.Tc(p)
    rv, rl, _ = oracle.maxwell(p, T)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.disk(nx, ny, 14, rv, rl, T))

    def centroid():
        rho = O.fields()["rho"]
        vap = rho < 0.5 * (rl + rv)
        return (np.arange(ny)[:, None] * np.ones((1, nx)))[vap].mean(), vap.sum()

    assert O.step(400) == 0
    y0, n0 = centroid()
    assert O.step(1200) == 0
    y1, n1 = centroid()
    assert n1 > 0.8 * n0
    assert y1 > y0 + 1.5


def test_pool_top_is_a_constant_pressure_surface():
    """Pool boiling domain (Sec. 2.D): periodic sides, heated bottom wall, and a top read
    as a free surface, i.e. a constant-pressure boundary: after every step the top row
    has rho = rho_out and no tangential momentum (Zou-He), and the temperature of the row
    below (zero gradient)."""
    nx, ny = 24, 12
    p = prm(nx, geometry="pool", thermal=1, g_a=1e-4, heater_x0=9, heater_len=5, heat_on_step=0, dTheat_R=0.15,
            rho_out=5.9)
    T = 0.9 * oracle.Tc(p)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.smooth_random(nx, ny, 5.9, T, seed=3, drho=0.01, du=0.01, dT=0.01))
    for _ in range(3):
        assert O.step(5) == 0
        f, g = O.populations()
        np.testing.assert_allclose(f[:, -1, :].sum(axis=0), 5.9, rtol=1e-14)
        np.testing.assert_allclose((f[:, -1, :] * CX[:, None]).sum(axis=0), 0.0, atol=1e-13)
        np.testing.assert_array_equal(g[:, -1, :], g[:, -2, :])
    assert np.ptp(g[:, -2, :].sum(axis=0)) > 0  # the temperature is not trivially uniform


def test_pool_bubble_is_lifted_by_buoyancy():
    """Eq. 14 in the pool: with gravity the vapour moves up; without, it does not.
    (An unheated bubble in liquid held at the saturation pressure is a critical nucleus and
    condenses over ~10^3 steps, so the test compares early rise velocities.)"""
    nx, ny = 48, 80
    rise = {}
    for ga in (0.0, 1e-4):
        p = prm(nx, geometry="pool", thermal=0, g_a=ga, heater_len=0)
        T = 0.9 * oracle.Tc(p)
        rv, rl, _ = oracle.maxwell(p, T)
        p["rho_out"] = rl
        O = oracle.Oracle(nx, ny, p)
        O.init_fields(*I.disk(nx, ny, 14, rv, rl, T, cy=30.0))
        assert O.step(150) == 0
        F = O.fields()
        vap = F["rho"] < 0.5 * (rl + rv)
        assert vap.sum() > 400
        rise[ga] = F["uy"][vap].mean()
    assert abs(rise[0.0]) < 0.005 and rise[1e-4] > rise[0.0] + 0.02


@pytest.mark.slow
def test_contact_angle_decreases_with_wall_density():
    """Sec. 3.E, Fig. 15: a false wall density nearer the liquid value wets more
    (smaller contact angle); nearer the vapour value wets less."""
    nx, ny = 72, 36
    thetas = []
    for rho_w in (1.5, 3.0, 4.5):
        p = prm(nx, geometry="walls", thermal=0, g_a=0.0, rho_w=rho_w)
        T = 0.9 * oracle.Tc(p)
        rv, rl, _ = oracle.maxwell(p, T)
        O = oracle.Oracle(nx, ny, p)
        O.init_fields(*I.sessile(nx, ny, 14, rl, rv, T))
        assert O.step(3000) == 0
        liquid = O.fields()["rho"] > 0.5 * (rl + rv)
        base = liquid[0].sum()
        height = liquid.any(axis=1).sum()
        thetas.append(PP.contact_angle_from_cap(height, base))
    assert thetas[0] > thetas[1] > thetas[2]


def test_centreline_pressure_drop():
    """Delta p (Sec. 3.B, Fig. 12b): the pressure at (1, ny/2) minus that at (nx-2, ny/2), taken from
    the moments the step starts from.  Without the pseudopotential the fluid is the lattice ideal
    gas p = c_s^2 rho = rho/3 (Sec. 2.A), so a density varying in x and y gives the two probes'
    density difference over 3 (a wrong probe row or column, or a flipped sign, misses it); a liquid
    and a vapour at Maxwell coexistence (Sec. 2.D) have equal pressures and unequal densities, so
    Delta p vanishes there while a density difference would not."""
    nx, ny = 24, 9
    xs, ys = np.arange(nx)[None, :], np.arange(ny)[:, None]
    zero = np.zeros((ny, nx))
    p = prm(nx, geometry="channel", thermal=0, multiphase=0, g_a=0.0, u_in=0.0, rho_out=1.0)
    rho = 1.0 + 0.01 * xs * (1.0 + 0.05 * ys ** 2)  # the x-difference depends on the row
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(rho, zero, zero)
    assert O.step(1) == 0
    d = O.last_diag()
    assert d["step"] == 0
    assert d["dp"] == pytest.approx((rho[ny // 2, 1] - rho[ny // 2, nx - 2]) / 3.0, rel=1e-13)

    p2 = prm(nx, geometry="channel", thermal=0, g_a=0.0, u_in=0.0)
    T = p2["T0_R"] * oracle.Tc(p2)
    rv, rl, ps = oracle.maxwell(p2, T)
    assert rl - rv > 1.0
    two = np.where(xs < nx // 2, rl, rv) + 0.0 * zero
    O2 = oracle.Oracle(nx, ny, dict(p2, rho_out=rv))
    O2.init_fields(two, zero, zero)
    O2.step(1)
    d2 = O2.last_diag()
    assert abs(d2["dp"]) < 1e-9 * ps


def test_heater_temperature_contrast():
    """delta T* (Sec. 3.B, Fig. 12c) = (T_w - T_nb) / (T_w - T_bulk): T_nb the mean temperature over
    the heater columns of the row next to the heater, T_bulk the domain mean, T_w the heater
    temperature once it is on.  A uniform field away from T_w gives exactly 1 (bulk and
    heater-adjacent row agree; a bulk taken from T_in instead would not); the heater-adjacent
    nodes at T_w give exactly 0 (a neighbouring row or column in T_nb would not); with the heater
    off it is 0 by definition."""
    nx, ny = 20, 8
    x0, nh = 6, 5
    zero = np.zeros((ny, nx))
    base = dict(geometry="channel", thermal=1, multiphase=0, g_a=0.0, u_in=0.0, rho_out=1.0, heater_x0=x0,
                heater_len=nh, dTheat_R=0.3)
    p = prm(nx, heat_on_step=0, **base)
    Tc = oracle.Tc(p)
    Tw = (p["Tin_R"] + p["dTheat_R"]) * Tc
    T1 = (p["Tin_R"] + 0.05) * Tc
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(1.0 + zero, zero, zero, T1 + zero)
    O.step(1)
    assert O.last_diag()["dtstar"] == pytest.approx(1.0, abs=1e-13)

    T = T1 + zero
    T[0, x0:x0 + nh] = Tw
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(1.0 + zero, zero, zero, T)
    O.step(1)
    assert abs(O.last_diag()["dtstar"]) < 1e-13

    O = oracle.Oracle(nx, ny, prm(nx, heat_on_step=10, **base))
    O.init_fields(1.0 + zero, zero, zero, T)
    O.step(1)
    assert O.last_diag()["dtstar"] == 0.0


def test_inlet_and_outlet_flux_diagnostics():
    """The flux records are sums over the rows of rho u_x at x = 0 and x = nx - 1.  From a fluid at
    rest (rho = 1, no force) the first step starts from the initialised populations (no boundary
    fill yet): both are 0.  The next step's inlet and outlet nodes pull rest populations, so Zou-He
    gives closed forms per row: rho u_x = u_in / (1 - u_in) at the velocity inlet and 1 - rho_out at
    the pressure outlet, while the neighbouring columns are still at rest."""
    nx, ny = 16, 7
    u_in, rho_out = 0.02, 1.01
    p = prm(nx, geometry="channel", thermal=0, multiphase=0, g_a=0.0, u_in=u_in, rho_out=rho_out)
    zero = np.zeros((ny, nx))
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(1.0 + zero, zero, zero)
    O.step(1)
    d = O.last_diag()
    assert d["flux_in"] == 0.0 and d["flux_out"] == 0.0
    O.step(1)
    d = O.last_diag()
    assert d["step"] == 1
    assert d["flux_in"] == pytest.approx(ny * u_in / (1.0 - u_in), rel=1e-13)
    assert d["flux_out"] == pytest.approx(ny * (1.0 - rho_out), rel=1e-12)


def test_inlet_temperature_is_a_fixed_point_at_rest():
    """The inlet's anti-bounce-back (Sec. 2.C) imposes T_in on the links that streaming leaves
    unknown; with the fluid at rest and uniformly at T_in the incoming populations are exactly
    g^eq(T_in, 0), so the field stays at T_in to rounding.  T_in differs from the initial-state T0
    here, so an inlet that imposed T0 (or anything else) would move the inlet column."""
    nx, ny = 20, 9
    p = prm(nx, geometry="channel", thermal=1, multiphase=0, g_a=0.0, u_in=0.0, rho_out=1.0, Tin_R=0.95,
            T0_R=0.9, heater_len=0)
    Tin = p["Tin_R"] * oracle.Tc(p)
    zero = np.zeros((ny, nx))
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(1.0 + zero, zero, zero, Tin + zero)
    assert O.step(20) == 0
    assert np.abs(O.fields()["T"] - Tin).max() < 1e-14


def test_zou_he_non_equilibrium_bounce_back():
    """Zou-He (Sec. 2.C) closes the open boundaries by bouncing back the non-equilibrium part normal
    to them, f_1 - f_1^eq = f_3 - f_3^eq; the odd part of the equilibrium (Eq. 3) then gives
    f_1 - f_3 = (2/3) rho u_x on every inlet and outlet node off the corners.  Imposing only the
    moments (an equilibrium f_1, say) would keep rho and u right and break this."""
    nx, ny = 20, 9
    p = prm(nx, geometry="channel", thermal=1, u_in=0.03, rho_out=5.9)
    T = p["T0_R"] * oracle.Tc(p)
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(*I.smooth_random(nx, ny, 5.9, T, seed=12, drho=0.01, du=0.01, dT=0.01))
    for _ in range(3):
        assert O.step(1) == 0
        f, _ = O.populations()
        rho = f.sum(axis=0)
        jx = (f * CX[:, None, None]).sum(axis=0)
        for x in (0, nx - 1):
            lhs = f[1, 1:-1, x] - f[3, 1:-1, x]
            np.testing.assert_allclose(lhs, (2.0 / 3.0) * jx[1:-1, x], rtol=0, atol=1e-13)
        assert np.abs(jx[1:-1, -1]).max() > 1e-4  # the outlet carries flow: the check has teeth


def test_buoyancy_uses_the_previous_steps_mean():
    """Eq. 14 with its one-step lag: F_y = -(rho - rho_avg) g_a, rho_avg the mean density of the
    previous step's state, so summed over the nodes the buoyancy is -g_a (M_n - M_(n-1)), the mass
    change over the last step.  A closed box keeps its mass and cannot tell; a channel whose outlet
    density exceeds the fluid's gains mass every step, so a mean of the current step (sum zero) or
    a stale one (the sum since the start) misses it."""
    nx, ny, ga = 20, 9, 1e-3
    p = prm(nx, geometry="channel", thermal=0, multiphase=0, g_a=ga, u_in=0.01, rho_out=1.02)
    zero = np.zeros((ny, nx))
    O = oracle.Oracle(nx, ny, p)
    O.init_fields(1.0 + zero, zero, zero)
    for _ in range(4):
        assert O.step(1) == 0
        F = O.fields()
        m_now, m_prev = math.fsum(F["rho"].ravel()), O.last_diag()["mass"]
        assert m_now - m_prev > 0.1
        assert math.fsum(F["Fy"].ravel()) == pytest.approx(-ga * (m_now - m_prev), rel=1e-9)
