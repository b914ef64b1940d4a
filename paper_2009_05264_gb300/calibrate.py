"""Contact-angle calibration of the wetting parameter (Eq. 15, Sec. 3.E, Fig. 15).

The paper sets wettability through the wall's false density rho_w but gives no
map from rho_w to a contact angle.  This module measures one: isothermal sessile
drops, one per rho_w, on the bottom wall of a periodic-in-x box, all advanced
together as one ``lbm.Batch`` (one fused launch per step), then the static angle
from each cap's height and base width.  ``rho_w_for_angle`` inverts the measured
table (the angle falls monotonically as rho_w rises towards the liquid density).

Drops start as half-disks of the coexisting liquid in its vapour; the coexistence
densities come from Maxwell's equal-area rule on the Peng-Robinson isotherm
(Eq. 12), computed here with numpy/scipy.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs as I
from . import params as PP


def pressure(p: dict, rho, T):
    """Peng-Robinson pressure of Eq. 12 with alpha(T) = [1 + kappa (1 - sqrt(T/Tc))]^2."""
    w = p["omega"]
    kappa = 0.37464 + 1.54226 * w - 0.26992 * w * w
    alpha = (1.0 + kappa * (1.0 - math.sqrt(T / PP.Tc(p)))) ** 2
    a, b, R = p["a"], p["b"], p["R"]
    rho = np.asarray(rho, dtype=np.float64)
    return rho * R * T / (1.0 - b * rho) - a * alpha * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho)


def coexistence(p: dict, T: float):
    """(rho_v, rho_l, p_sat) of the isotherm T < Tc by Maxwell's equal-area rule:
    equal pressures and equal integrals of dp / rho (equal chemical potential)."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    b = p["b"]
    grid = np.linspace(1e-4, 0.999 / b, 40001)
    pg = pressure(p, grid, T)
    dp = np.diff(pg)
    turns = np.nonzero(np.sign(dp[1:]) != np.sign(dp[:-1]))[0] + 1
    if len(turns) < 2:
        raise ValueError("isotherm has no van der Waals loop (T >= Tc?)")
    r_max, r_min = grid[turns[0]], grid[turns[1]]  # local maximum, then local minimum of p

    def branch(ps, lo, hi):
        return brentq(lambda r: float(pressure(p, r, T)) - ps, lo, hi, xtol=1e-14)

    def mismatch(ps):
        rv = branch(ps, 1e-12, r_max)
        rl = branch(ps, r_min, 0.9999 / b)
        # integral of (p - ps) / rho^2 d rho from rv to rl vanishes at coexistence
        val, _ = quad(lambda r: (float(pressure(p, r, T)) - ps) / (r * r), rv, rl, points=[r_max, r_min],
                      epsabs=1e-14, epsrel=1e-12, limit=200)
        return val

    p_lo = max(float(pressure(p, r_min, T)), 1e-10)
    p_hi = float(pressure(p, r_max, T))
    ps = brentq(mismatch, p_lo * (1 + 1e-9), p_hi * (1 - 1e-9), xtol=1e-16)
    return branch(ps, 1e-12, r_max), branch(ps, r_min, 0.9999 / b), ps


def cap_angle(rho: np.ndarray, rho_l: float, rho_v: float) -> tuple[float, int, int]:
    """(angle in degrees, base width, height) of the liquid cap on the bottom wall:
    liquid where rho exceeds the mid density; the wall lies half a row below row 0."""
    liquid = rho > 0.5 * (rho_l + rho_v)
    base = int(liquid[0].sum())
    height = int(liquid.any(axis=1).sum())
    if base == 0:
        return 180.0, base, height
    return PP.contact_angle_from_cap(height, base), base, height


def contact_angles(rho_w_values, nx: int = 100, ny: int = 50, radius: float = 18.0, steps: int = 6000,
                   T_R: float = 0.9, precision: str = "fp32", device: int = 0, tiling=None):
    """Measured static contact angle for each wall density, one batched run.

    Returns a list of dicts {rho_w, theta, base, height}."""
    from . import lbm

    base = PP.resolve(PP.default_params(geometry="walls", thermal=0, g_a=0.0, T0_R=T_R, Tin_R=T_R), nx)
    T = T_R * PP.Tc(base)
    rho_v, rho_l, _ = coexistence(base, T)
    fields = I.sessile(nx, ny, radius, rho_l, rho_v, T)
    batch = lbm.Batch(precision, thermal=False, device=device)
    try:
        if tiling:
            batch.set_tiling(*tiling)
        members = []
        for rw in rho_w_values:
            p = dict(base, rho_w=float(rw), init_rho_out=rho_l)
            m = batch.add(nx, ny, p)
            m.init_fields(*fields)
            members.append((float(rw), m))
        batch.step(steps)
        out = []
        for rw, m in members:
            theta, w, h = cap_angle(m.fields()["rho"], rho_l, rho_v)
            out.append({"rho_w": rw, "theta": theta, "base": w, "height": h})
        return out
    finally:
        batch.close()


def rho_w_for_angle(theta: float, table) -> float:
    """Wall density giving contact angle theta (degrees), interpolated linearly in a
    measured table (from contact_angles) on its monotone part."""
    pts = sorted(((r["rho_w"], r["theta"]) for r in table if 0.0 < r["theta"] < 180.0), key=lambda t: t[0])
    if len(pts) < 2:
        raise ValueError("need at least two measured angles strictly between 0 and 180 degrees")
    rw = np.array([t[0] for t in pts])
    th = np.array([t[1] for t in pts])
    if not np.all(np.diff(th) < 0):
        raise ValueError("measured angles do not fall monotonically with rho_w")
    if not th[-1] <= theta <= th[0]:
        raise ValueError(f"theta {theta} outside the measured range [{th[-1]:.1f}, {th[0]:.1f}]")
    return float(np.interp(theta, th[::-1], rw[::-1]))
