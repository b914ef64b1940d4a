"""Pool boiling: bubble departure diameter against gravity (Sec. 2.D, Fig. 5).

The paper validates its model on a pool: saturated liquid at T_R = 0.9 in a domain of
aspect ratio 4 with periodic sides, a free-surface top and an isothermal bottom wall at
the saturation temperature, with a heated segment at the centre of the bottom wall; the
departure diameter regresses as D_d = 0.246 g^-0.49 against the lattice gravity g (Fritz's
correlation gives the exponent 0.5).  ``departure_diameters`` runs one lattice per g as a
single batch (one fused launch per step), tracks departures from density snapshots
(``bubbles.DepartureTracker``: a vapour region that leaves the heater) and averages the
diameter of the departures after the start-up; ``fit_power_law`` regresses D_d = C g^n.

Readings (the paper gives neither tau_g, c_v nor the wettability of the pool): the
domain is 4 times taller than wide (128 x 512 by default); the heater is 10 nodes at
0.3 Tc superheat (with the paper's 5 nodes at T_R = 1.05 and the library defaults
tau_g = 0.6, c_v = 6, no bubble departs within 1.5e5 steps); rho_w = 3.0.
"""
from __future__ import annotations

import math

import numpy as np

from . import bubbles as B
from . import calibrate as CAL
from . import inputs as I
from . import params as PP


def pool_params(g_a: float, nx: int, heater_len: int = 10, dTheat_R: float = 0.3, rho_w: float = 3.0,
                T_R: float = 0.9) -> tuple[dict, float, float]:
    """(library parameters, rho_l, rho_v) of a pool at T_R with the heater centred on the
    bottom wall, switched on from the start; the top holds the saturated liquid density."""
    base = PP.default_params()
    T = T_R * PP.Tc(base)
    rho_v, rho_l, _ = CAL.coexistence(PP.resolve(base, nx), T)
    p = PP.resolve(PP.default_params(geometry="pool", g_a=g_a, heater_x0=nx // 2 - heater_len // 2,
                                     heater_len=heater_len, dTheat_R=dTheat_R, heat_on_step=0, rho_out=rho_l,
                                     init_rho_out=rho_l, rho_vapor=0.5 * (rho_l + rho_v), rho_w=rho_w, u_in=0.0,
                                     T0_R=T_R, Tin_R=T_R), nx)
    return p, rho_l, rho_v


def departure_diameters(g_values, nx: int = 128, ny: int = 512, steps: int = 100000, every: int = 100,
                        skip: int = 2, n_mean: int = 5, heater_len: int = 10, dTheat_R: float = 0.3,
                        rho_w: float = 3.0, precision: str = "fp32", device: int = 0) -> list[dict]:
    """One pool per g, advanced together for `steps` steps; per g the departure events and
    the mean diameter and period of the n_mean departures after the first `skip` (None
    where fewer departures occurred)."""
    from . import lbm

    batch = lbm.Batch(precision, thermal=True, device=device)
    try:
        runs = []
        for g in g_values:
            p, rho_l, rho_v = pool_params(g, nx, heater_len, dTheat_R, rho_w)
            m = batch.add(nx, ny, p)
            m.init_fields(*I.uniform(nx, ny, rho_l, p["T0_R"] * PP.Tc(p)))
            runs.append((float(g), m, B.DepartureTracker(p["rho_vapor"], p["heater_x0"], heater_len,
                                                         min_area=10, periodic_x=True)))
        for k in range(steps // every):
            batch.step(every)
            for _, m, tr in runs:
                tr.update(m.fields()["rho"], (k + 1) * every)
        out = []
        for g, _, tr in runs:
            st = B.event_statistics(tr.events, skip=skip, n_diameter=n_mean, n_period=n_mean - 1)
            out.append({"g": g, "departures": len(tr.events), "diameter": st["diameter"], "period": st["period"],
                        "events": tr.events})
        return out
    finally:
        batch.close()


def fit_power_law(g, d) -> tuple[float, float]:
    """Least-squares fit of log d = log C + n log g; returns (C, n)."""
    lg, ld = np.log(np.asarray(g, dtype=np.float64)), np.log(np.asarray(d, dtype=np.float64))
    n, logc = np.polyfit(lg, ld, 1)
    return float(math.exp(logc)), float(n)
