"""Bubble statistics from diagnostics series (departure detection, averages, sine fit)."""
import math

import numpy as np
import pytest

from paper_2009_05264_gb300 import bubbles as B


def series_with_departures(dep_steps, areas, n=4000):
    s = np.zeros((n, len(B.COLUMNS)))
    s[:, 0] = np.arange(n)
    attached = np.zeros(n, dtype=bool)
    zone = np.zeros(n)
    prev = 0
    for d, a in zip(dep_steps, areas):
        start = prev + (d - prev) // 3  # nucleation a while after the previous departure
        attached[start:d] = True
        zone[start:d] = np.linspace(1, a * 0.9, d - start)
        zone[d] = a
        zone[d + 1:d + 30] = a  # the departed bubble still near the heater for a while
        prev = d
    s[:, B.COLUMNS.index("heater_vapor")] = np.where(attached, 3.0, 0.0)
    s[:, B.COLUMNS.index("zone_vapor")] = zone
    return s


def test_departures_are_found_with_their_areas():
    deps = [500, 1100, 1690, 2300, 2880, 3500]
    areas = [300.0, 320.0, 310.0, 305.0, 315.0, 330.0]
    ev = B.departures(series_with_departures(deps, areas))
    assert [e["step"] for e in ev] == deps
    assert [e["area"] for e in ev] == areas
    assert ev[0]["diameter"] == pytest.approx(2 * math.sqrt(300 / math.pi))


def test_departure_statistics_average_five_diameters_and_four_periods():
    deps = [500, 1100, 1690, 2300, 2880, 3500]
    areas = [300.0, 320.0, 310.0, 305.0, 315.0, 330.0]
    st = B.departure_statistics(series_with_departures(deps, areas))
    assert st["departures"] == 6
    assert st["diameter"] == pytest.approx(np.mean([2 * math.sqrt(a / math.pi) for a in areas[:5]]))
    assert st["period"] == pytest.approx(np.mean(np.diff(deps[:5])))
    few = B.departure_statistics(series_with_departures(deps[:3], areas[:3]))
    assert few["diameter"] is None and few["period"] is None


def test_sine_fit_recovers_contact_line_oscillation():
    t = np.arange(0, 6000, 10.0)
    y = 40 + 12 * np.sin(2 * math.pi * t / 750 + 1.1) + np.random.default_rng(1).normal(0, 0.5, t.size)
    fit = B.fit_sine(t, y)
    assert fit["period"] == pytest.approx(750, rel=0.01)
    assert fit["amplitude"] == pytest.approx(12, rel=0.03)
    assert fit["offset"] == pytest.approx(40, abs=0.2)
