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


def _disk(mask_shape, cx, cy, r):
    y, x = np.mgrid[0:mask_shape[0], 0:mask_shape[1]]
    return (x - cx) ** 2 + (y - cy) ** 2 <= r * r


def synthetic_cycles(n_cycles=5, period=10, nx=60, ny=90, rho_l=6.0, rho_v=0.6):
    """Density snapshots of bubbles growing on a heater (columns 25-34), pinching off above a
    vapour film that stays on the heater, and rising; returns frames, steps and the expected
    departure events (frame step, area)."""
    frames, steps, expected = [], [], []
    risers = []  # (cy, r) of detached bubbles
    film = np.zeros((ny, nx), dtype=bool)
    film[0, 27:33] = True
    for c in range(n_cycles):
        for k in range(period):
            vap = film.copy()
            r = 3 + k if k <= 5 else 0
            if k <= 5:
                vap |= _disk(vap.shape, 30, r - 1, r)  # attached: reaches row 0
            if k == 6:
                risers.append([9.0, 6])
            for b in risers:
                vap |= _disk(vap.shape, 30, b[0], b[1])
            rho = np.where(vap, rho_v, rho_l)
            step = (c * period + k + 1) * 100
            if k == 6:
                lab = _disk(vap.shape, 30, 9.0, 6)
                expected.append((step, float(lab.sum())))
            frames.append(rho)
            steps.append(step)
            for b in risers:
                b[0] += 4.0
            risers = [b for b in risers if b[0] - b[1] < ny]
    return frames, steps, expected


def test_snapshot_detachments_over_a_residual_film():
    frames, steps, expected = synthetic_cycles()
    ev = B.detachments(frames, steps, 3.2, heater_x0=25, heater_len=10, min_area=20)
    assert [(e["step"], e["area"]) for e in ev] == expected
    st = B.event_statistics(ev)
    assert st["departures"] == 5
    assert st["period"] == pytest.approx(1000.0)
    assert st["diameter"] == pytest.approx(2 * math.sqrt(expected[0][1] / math.pi))
    # skipping the first departure as start-up leaves four: too few for the five-departure
    # diameter and the four-interval period
    late = B.event_statistics(ev, skip=1)
    assert late["diameter"] is None and late["period"] is None


def test_small_fragments_and_risers_are_not_departures():
    frames, steps, expected = synthetic_cycles(n_cycles=2)
    ev = B.detachments(frames, steps, 3.2, heater_x0=25, heater_len=10, min_area=200)
    assert ev == []  # the 113-node bubbles are below this min_area
    ev = B.detachments(frames[7:], steps[7:], 3.2, heater_x0=25, heater_len=10, min_area=20)
    assert [e["step"] for e in ev] == [expected[1][0]]  # the first riser was already detached


def test_vapour_components_join_across_a_periodic_edge():
    rho = np.full((10, 20), 6.0)
    rho[4:7, 0:3] = 0.5
    rho[4:7, 17:20] = 0.5
    rho[1, 9] = 0.5
    lab, n = B.vapour_components(rho, 3.2, periodic_x=False)
    assert n == 3
    lab, n = B.vapour_components(rho, 3.2, periodic_x=True)
    assert n == 2
    assert lab[5, 0] == lab[5, 19] != lab[1, 9]
    assert np.bincount(lab.ravel())[lab[5, 0]] == 18


def test_detachment_rule_edge_cases():
    """The departure rule's clauses one at a time, on hand-made frames (60 x 40, heater columns
    25-34): a bubble lifted one row off the heater departs (row 0 decides what is attached); a
    rising bubble that grows into where the previous frame's attached vapour was is not counted
    again (it overlaps a region already detached); a blob that appears away from the heater is
    not a departure (it overlaps no attached vapour); and 4-connectivity keeps regions that touch
    only at a corner apart."""
    ny, nx, rho_l, rho_v = 40, 60, 6.0, 0.6

    def frame(*disks):
        vap = np.zeros((ny, nx), dtype=bool)
        for cx, cy, r in disks:
            vap |= _disk(vap.shape, cx, cy, r)
        return np.where(vap, rho_v, rho_l)

    det = lambda fr: B.detachments(fr, [100 * (k + 1) for k in range(len(fr))], 3.2, heater_x0=25,  # noqa: E731
                                   heater_len=10, min_area=20)
    lifted = [frame((30, 5, 5)), frame((30, 6, 5))]  # rows 0-10, then rows 1-11
    assert [e["step"] for e in det(lifted)] == [200]
    grow = [frame((30, 5, 6)),                    # attached, rows 0-11
            frame((30, 3, 4), (30, 14, 5)),       # new attached bubble rows 0-7; riser rows 9-19 departs
            frame((30, 2, 2), (30, 15, 8))]       # the riser grows into rows 7-23: overlaps both
    assert [e["step"] for e in det(grow)] == [200]
    appear = [frame((30, 5, 6)), frame((30, 5, 6), (8, 25, 5))]
    assert det(appear) == []
    rho = np.full((10, 10), rho_l)
    rho[2:5, 2:5] = rho_v
    rho[5:8, 5:8] = rho_v  # touches the first block only at the corner (4, 4)-(5, 5)
    assert B.vapour_components(rho, 3.2)[1] == 2
