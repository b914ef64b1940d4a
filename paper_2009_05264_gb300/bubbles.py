"""Bubble statistics from the per-step diagnostics records (Sec. 3.A-3.C; Figs. 8,
12, 13, 17).

The fused step records, every step, the vapour area (nodes with rho < rho_vapor),
the vapour footprint on the row next to the bottom wall, the footprint over the
heater sites and the vapour in the columns around the heater (x_h - n_h <= x <
x_h + 2 n_h).  From those series:

* a bubble sits on the heater while the heater footprint is non-zero, and departs
  at the first step whose heater footprint is zero after such a run;
* its departure diameter is that of the circle with the area of the vapour around
  the heater at that step, D = 2 sqrt(A / pi) (2D bubbles), and the departure
  period is the time between successive departures; the paper averages the
  diameter over five departures and the period over four;
* the contact-line extent L_t(t) is the wall footprint (the length of wall under
  vapour, in lattice units, in 2D); its oscillation is summarised by a fitted sine.

Where a thin vapour film stays on the heater while bubbles rise from it, the heater
footprint never returns to zero; ``detachments`` then finds departures from field
snapshots instead: a departure is a connected vapour region that no longer touches the
heater sites and overlaps the vapour that was attached to the heater one snapshot
earlier (and is not the continuation of an already detached bubble).
"""
from __future__ import annotations

import math

import numpy as np

COLUMNS = ("step", "mass", "energy", "rho_avg", "dp", "dtstar", "flux_in", "flux_out", "vapor_area",
           "wall_vapor", "heater_vapor", "zone_vapor")


def _col(series: np.ndarray, name: str) -> np.ndarray:
    return np.asarray(series)[:, COLUMNS.index(name)]


def departures(series: np.ndarray, min_attached: int = 1) -> list[dict]:
    """Departure events of a (steps, len(COLUMNS)) diagnostics array, in step order:
    dicts with the step, the vapour area around the heater and the diameter."""
    step = _col(series, "step")
    on = _col(series, "heater_vapor") > 0
    zone = _col(series, "zone_vapor")
    out = []
    run = 0
    for k in range(len(step)):
        if on[k]:
            run += 1
            continue
        if run >= min_attached and k > 0:
            a = float(zone[k])
            out.append({"step": int(step[k]), "area": a, "diameter": 2.0 * math.sqrt(a / math.pi)})
        run = 0
    return out


def departure_statistics(series: np.ndarray, n_diameter: int = 5, n_period: int = 4,
                         min_attached: int = 1) -> dict:
    """Mean departure diameter over the first n_diameter departures and mean period over
    the first n_period intervals between them (None where too few departures)."""
    ev = departures(series, min_attached)
    d = [e["diameter"] for e in ev[:n_diameter]]
    t = [e["step"] for e in ev[: n_period + 1]]
    return {"departures": len(ev),
            "diameter": float(np.mean(d)) if len(d) == n_diameter else None,
            "period": float(np.mean(np.diff(t))) if len(t) == n_period + 1 else None,
            "events": ev}


def fit_sine(t: np.ndarray, y: np.ndarray) -> dict:
    """Least-squares fit y ~ c + A sin(2 pi t / P + phi), started from the strongest
    non-zero frequency of the series; returns c, A (>= 0), P and phi."""
    from scipy.optimize import curve_fit

    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    dt = float(np.median(np.diff(t)))
    spec = np.abs(np.fft.rfft(y - y.mean()))
    freq = np.fft.rfftfreq(len(y), d=dt)
    k = int(np.argmax(spec[1:]) + 1)
    p0 = [y.mean(), math.sqrt(2.0) * y.std(), 1.0 / freq[k], 0.0]
    # phase start: best of a few trial phases
    best = None
    for ph in np.linspace(0, 2 * math.pi, 8, endpoint=False):
        r = np.sum((y - (p0[0] + p0[1] * np.sin(2 * math.pi * t / p0[2] + ph))) ** 2)
        if best is None or r < best[0]:
            best = (r, ph)
    p0[3] = best[1]
    f = lambda tt, c, A, P, phi: c + A * np.sin(2 * math.pi * tt / P + phi)  # noqa: E731
    (c, A, P, phi), _ = curve_fit(f, t, y, p0=p0, maxfev=20000)
    if A < 0:
        A, phi = -A, phi + math.pi
    return {"offset": float(c), "amplitude": float(A), "period": float(P), "phase": float(phi % (2 * math.pi))}


def record(lattice, steps: int, chunk: int = 1000) -> np.ndarray:
    """Advance a lattice by `steps` steps and return every step's diagnostics record
    (read back every `chunk` <= 1024 steps, before the ring overwrites them).  The
    vapour columns are counted only for lattices created with bubble_stats = 1."""
    if not 1 <= chunk <= 1024:
        raise ValueError("chunk must be within the 1024-record ring")
    rows = []
    done = 0
    lattice.sync()  # the step count below must include every step already enqueued
    while done < steps:
        n = min(chunk, steps - done)
        first = lattice.step_count
        lattice.step(n)
        rows.append(lattice.diagnostics_range(first, n))
        done += n
    return np.concatenate(rows) if rows else np.empty((0, len(COLUMNS)))


def vapour_components(rho: np.ndarray, rho_vapor: float, periodic_x: bool = False):
    """Labels (0 = liquid) of the 4-connected vapour regions rho < rho_vapor of a (ny, nx)
    field, joined across x = 0 / x = nx - 1 when periodic_x; returns (labels, count)."""
    from scipy import ndimage

    vap = np.asarray(rho) < rho_vapor
    lab, n = ndimage.label(vap)
    if periodic_x and n > 1:
        parent = list(range(n + 1))

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        for a, b in zip(lab[:, 0], lab[:, -1]):
            if a and b:
                ra, rb = find(int(a)), find(int(b))
                if ra != rb:
                    parent[max(ra, rb)] = min(ra, rb)
        roots = np.array([find(k) for k in range(n + 1)])
        uniq, lab = np.unique(roots[lab], return_inverse=True)
        lab = lab.reshape(vap.shape)
        n = len(uniq) - 1  # root 0 is the liquid
    return lab, n


class DepartureTracker:
    """Online form of ``detachments``: feed snapshots in step order with update(); the
    departure events accumulate in .events (only the previous snapshot's masks are kept)."""

    def __init__(self, rho_vapor: float, heater_x0: int, heater_len: int, min_area: int = 20,
                 periodic_x: bool = False):
        self.rho_vapor, self.heater_x0, self.heater_len = rho_vapor, heater_x0, heater_len
        self.min_area, self.periodic_x = min_area, periodic_x
        self.events: list[dict] = []
        self._att = self._det = None

    def update(self, rho: np.ndarray, step: int):
        lab, n = vapour_components(rho, self.rho_vapor, self.periodic_x)
        nx = lab.shape[1]
        x0, hl = self.heater_x0, self.heater_len
        cols = np.arange(x0, x0 + hl) % nx if self.periodic_x else np.arange(max(x0, 0), min(x0 + hl, nx))
        on_heater = set(int(v) for v in lab[0, cols]) - {0}
        area = np.bincount(lab.ravel(), minlength=n + 1)
        attached = np.isin(lab, sorted(on_heater)) if on_heater else np.zeros(lab.shape, dtype=bool)
        detached = np.zeros(lab.shape, dtype=bool)
        for c in range(1, n + 1):
            if c in on_heater or area[c] < self.min_area:
                continue
            comp = lab == c
            detached |= comp
            if self._att is not None and (comp & self._att).any() and not (comp & self._det).any():
                a = float(area[c])
                self.events.append({"step": int(step), "area": a, "diameter": 2.0 * math.sqrt(a / math.pi)})
        self._att, self._det = attached, detached


def detachments(frames, steps, rho_vapor: float, heater_x0: int, heater_len: int, min_area: int = 20,
                periodic_x: bool = False) -> list[dict]:
    """Departure events from a sequence of density snapshots (ny, nx) taken at `steps`:
    a vapour region of at least min_area nodes that touches none of the heater sites
    (row 0, columns heater_x0 .. heater_x0 + heater_len - 1), overlaps the vapour attached
    to the heater in the previous snapshot and overlaps no region that was already
    detached there.  Each event: step, area (nodes) and diameter 2 sqrt(area / pi)."""
    tr = DepartureTracker(rho_vapor, heater_x0, heater_len, min_area, periodic_x)
    for rho, step in zip(frames, steps):
        tr.update(rho, step)
    return tr.events


def event_statistics(events: list[dict], skip: int = 0, n_diameter: int = 5, n_period: int = 4) -> dict:
    """Mean diameter over n_diameter departures and mean period over n_period intervals,
    after dropping the first `skip` departures (the start-up transient); None where there
    are too few."""
    ev = events[skip:]
    d = [e["diameter"] for e in ev[:n_diameter]]
    t = [e["step"] for e in ev[: n_period + 1]]
    return {"departures": len(events),
            "diameter": float(np.mean(d)) if len(d) == n_diameter else None,
            "period": float(np.mean(np.diff(t))) if len(t) == n_period + 1 else None}


def snapshots(lattice, steps: int, every: int):
    """Advance a lattice by `steps` steps, returning (density snapshots, their steps) taken
    every `every` steps."""
    frames, at = [], []
    lattice.sync()
    for _ in range(steps // every):
        lattice.step(every)
        frames.append(lattice.fields()["rho"].copy())
        at.append(lattice.step_count)
    return frames, at
