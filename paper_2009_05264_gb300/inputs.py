"""Seeded synthetic inputs for the lattice: initial macroscopic fields only.

This module holds none of the method's arithmetic.  It produces the initial
density, velocity and temperature fields (numpy float64, shape (ny, nx),
row-major) that both the CUDA library and the CPU oracle are started from, and
the parameter sets of the channel workloads.  Random numbers come from
splitmix64 used as a counter-based hash (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the value for node k of
instance m under seed s is splitmix64(s ^ (m << 40) ^ k), mapped to [-1, 1).
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """splitmix64 output function applied elementwise to uint64 counters."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
    return z ^ (z >> np.uint64(31))


def unit_noise(nx: int, ny: int, seed: int, instance: int = 0):
    """xi in [-1, 1) per node, (ny, nx): 53 high bits of the hash scaled to [0, 1), times 2, minus 1."""
    k = np.arange(nx * ny, dtype=np.uint64)
    key = np.uint64(seed) ^ (np.uint64(instance) << np.uint64(40)) ^ k
    z = splitmix64(key)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (2.0 * u - 1.0).reshape(ny, nx)


def uniform(nx: int, ny: int, rho: float, T: float):
    """Quiescent uniform state: (rho, ux, uy, T) arrays."""
    return (np.full((ny, nx), float(rho)), np.zeros((ny, nx)), np.zeros((ny, nx)),
            np.full((ny, nx), float(T)))


def disk(nx: int, ny: int, radius: float, rho_in: float, rho_out: float, T: float,
         width: float = 2.0, cx: float | None = None, cy: float | None = None,
         seed: int = 0, amp: float = 0.0, instance: int = 0):
    """Disk of density rho_in (droplet: liquid; bubble: vapour) in rho_out, tanh
    interface of the given width, times (1 + amp * xi) with seeded noise xi."""
    cx = (nx - 1) / 2.0 if cx is None else cx
    cy = (ny - 1) / 2.0 if cy is None else cy
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    rho = 0.5 * (rho_in + rho_out) - 0.5 * (rho_in - rho_out) * np.tanh(2.0 * (r - radius) / width)
    if amp != 0.0:
        rho = rho * (1.0 + amp * unit_noise(nx, ny, seed, instance))
    return rho, np.zeros((ny, nx)), np.zeros((ny, nx)), np.full((ny, nx), float(T))


def slab(nx: int, ny: int, half_width: float, rho_in: float, rho_out: float, T: float,
         width: float = 2.0):
    """Flat liquid layer |y - yc| < half_width (two flat interfaces), periodic in x."""
    yc = (ny - 1) / 2.0
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    d = np.abs(y - yc) - half_width
    rho = 0.5 * (rho_in + rho_out) - 0.5 * (rho_in - rho_out) * np.tanh(2.0 * d / width)
    return rho, np.zeros((ny, nx)), np.zeros((ny, nx)), np.full((ny, nx), float(T))


def sessile(nx: int, ny: int, radius: float, rho_l: float, rho_v: float, T: float,
            width: float = 2.0):
    """Half-disk of liquid resting on the bottom wall (centre at the wall, y = -1/2)."""
    return disk(nx, ny, radius, rho_l, rho_v, T, width=width, cx=(nx - 1) / 2.0, cy=-0.5)


def smooth_random(nx: int, ny: int, rho0: float, T0: float, seed: int, drho: float = 0.05,
                  du: float = 0.01, dT: float = 0.0, instance: int = 0):
    """Smooth seeded perturbation of a uniform state (sum of a few Fourier modes
    with seeded phases) plus small node noise: a generic input for parity runs."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    ph = unit_noise(8, 1, seed, instance).ravel() * np.pi
    sx, sy = 2 * np.pi / max(nx, 1), 2 * np.pi / max(ny, 1)
    noise = unit_noise(nx, ny, seed + 1, instance)
    rho = rho0 * (1.0 + drho * (np.sin(sx * x + ph[0]) * np.cos(sy * y + ph[1]) + 0.1 * noise))
    ux = du * np.sin(sy * y + ph[2]) * np.cos(sx * x + ph[3])
    uy = du * np.sin(sx * x + ph[4]) * np.sin(sy * y + ph[5])
    T = T0 * (1.0 + dT * np.cos(sx * x + ph[6]) * np.sin(sy * y + ph[7]))
    return rho, ux, uy, T


def sweep_draws(n: int, seed: int, nx_range=(400, 2000), ny_range=(50, 200), u_range=(0.01, 0.05),
                dT_range=(0.03, 0.12), rho_w_range=(2.2, 4.0)):
    """Seeded parameter draws of a channel sweep: lattice size (uniform integers,
    inclusive), inlet velocity, heater superheat (in units of T_c) and wall density
    rho_w (the wetting parameter of Eq. 15), each uniform in its range.  Returns a
    list of dicts.  The default rho_w range gives static contact angles of about
    137 to 46 degrees (isothermal sessile drops at 0.9 T_c, 100 x 50 lattice)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        out.append(dict(nx=int(rng.integers(nx_range[0], nx_range[1] + 1)),
                        ny=int(rng.integers(ny_range[0], ny_range[1] + 1)),
                        u_in=float(rng.uniform(*u_range)), dTheat_R=float(rng.uniform(*dT_range)),
                        rho_w=float(rng.uniform(*rho_w_range))))
    return out
