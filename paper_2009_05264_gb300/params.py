"""Problem parameters of the flow-boiling channel (all lattice units).

Field names follow the paper's symbols (Sec. 2; Eq. numbers in comments).
Values the paper fixes are the defaults; values it leaves open are defaults of
this library, marked as such.  The same mapping feeds the CUDA library's
``lbm_params`` struct and, in the tests, the oracle's.
"""
from __future__ import annotations

import math

GEOMETRY = {"periodic": 0, "channel": 1, "walls": 2, "pool": 3}


def default_params(**overrides) -> dict:
    p = dict(
        geometry="channel",  # Sec. 2.C: inlet x=0, outlet x=nx-1, walls at y=-1 and y=ny
        thermal=1,           # evolve g (Eq. 16)
        multiphase=1,        # Shan-Chen + wetting forces (Eqs. 9, 15)
        tau_f=1.0,           # not stated in the paper (library default)
        tau_g=0.6,           # not stated in the paper; 0.6 keeps the anti-bounce-back walls stable
        a=2.0 / 49.0,        # Eq. 12, Sec. 2.A
        b=2.0 / 21.0,        # Eq. 12
        R=1.0,               # Eq. 12
        omega=0.32,          # acentric factor of R134a (Sec. 2.A)
        beta=1.16,           # Eq. 8
        c0=6.0,              # Eq. 11
        G=-1.0,              # interaction strength g of Eqs. 10-11 (sign fixed by Eq. 11 needing p - rho/3 < 0)
        T0_R=0.9,            # initial saturated liquid at T_R = 0.9 (Sec. 2.C)
        Tin_R=0.9,           # inlet and wall temperature (Sec. 2.C)
        dTheat_R=0.3,        # heater superheat 0.3 Tc (Sec. 3)
        u_in=0.01,           # inlet velocity (library default)
        rho_out=5.95,        # outlet density: liquid density at 0.9 Tc printed in Sec. 3.D
        rho_w=5.95,          # false wall density of Eq. 15 (sets the contact angle; library default)
        G_wet=None,          # Eq. 15 strength; None -> 9 (1 + beta) G: a wall whose false density equals
                             # the fluid's then exerts no net force on uniform fluid under the beta-mixed Eq. 9
        g_a=5e-5,            # lattice gravity printed for the pool-boiling check (Sec. 2.D)
        c_v=6.0,             # specific heat of Eq. 19 (not stated in the paper; library default)
        heater_x0=-1,        # -1 -> nx/5 (microheater at one fifth of the length, Sec. 2.C)
        heater_len=5,        # five heated nodes (Sec. 2.C)
        heat_on_step=10000,  # heater switched on after 10000 steps (Sec. 2.C)
        source_model=0,      # energy source: 0 Gong-Cheng (second Eq. 19, the paper's), 1 Hazi-Markus (first)
        reserved0=0,
        bubble_stats=0,      # 1: the library counts vapour nodes every step (bubble diagnostics)
        rho_vapor=3.2,       # vapour below this density in the bubble diagnostics: about the
                             # midpoint of the coexisting densities (0.59, 5.88) at 0.9 Tc
        init_kind=0,         # 0 uniform, 1 disk
        init_rho_in=5.95,
        init_rho_out=5.95,
        init_radius=0.0,
        init_width=2.0,
        perturb_amp=0.0,
        seed=0,
    )
    p.update(overrides)
    if p["G_wet"] is None:
        p["G_wet"] = 9.0 * (1.0 + p["beta"]) * p["G"]
    return p


def resolve(p: dict, nx: int) -> dict:
    """Fill the size-dependent defaults (heater position)."""
    q = dict(p)
    if isinstance(q["geometry"], str):
        q["geometry"] = GEOMETRY[q["geometry"]]
    if q["heater_x0"] is None or q["heater_x0"] < 0:
        q["heater_x0"] = nx // 5
    if q["G_wet"] is None:
        q["G_wet"] = 9.0 * (1.0 + q["beta"]) * q["G"]
    return q


def Tc(p: dict) -> float:
    """Critical temperature implied by a and b of Eq. 12: Tc = 0.0778 a / (0.45724 b R)."""
    return 0.0778 * p["a"] / (0.45724 * p["b"] * p["R"])


def tau_from_viscosity(nu: float) -> float:
    """nu = c_s^2 (tau - 1/2) (Sec. 2.A) solved for tau."""
    return 3.0 * nu + 0.5


def reynolds(u: float, H: float, tau_f: float) -> float:
    """Re_in = u H / nu with nu = (tau_f - 1/2)/3."""
    return u * H / ((tau_f - 0.5) / 3.0)


def contact_angle_from_cap(height: float, base: float) -> float:
    """Circular-cap contact angle in degrees from cap height h and base width w: 2 atan(2h/w)."""
    return math.degrees(2.0 * math.atan2(2.0 * height, base))
