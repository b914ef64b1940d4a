"""Long-run bubble departures of the FP32 and FP64 GPU steps against the oracle's.

Over tens of thousands of steps the boiling fields decorrelate pointwise, so the FP32
criterion there is statistical: the departure diameter averaged over five departures
and the departure period averaged over four (Sec. 3.B) within 2 % of the FP64 CPU
oracle's, on a heated channel (600 x 80, heater of 40 nodes at 0.3 Tc superheat,
u_in = 0.005) whose bubbles depart periodically.  The oracle's departures are stored
in tests/golden/departures_channel_600x80.json, written by make_departures.py beside it.
"""
import json
import os

import pytest

from paper_2009_05264_gb300 import bubbles as B
from paper_2009_05264_gb300 import inputs as I
from paper_2009_05264_gb300 import params as PP

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "departures_channel_600x80.json")))
TOL = 0.02


def library_params():
    g = GOLD["params"]
    p = PP.resolve(PP.default_params(**{k: v for k, v in g.items() if k != "geometry"}, geometry="channel",
                                     init_rho_out=GOLD["rho_l"]), GOLD["nx"])
    for k, v in g.items():
        assert p[k] == v, k  # the lattice runs exactly the oracle's parameters
    return p


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_long_run_departures_match_the_oracle(precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05264_gb300 import lbm

    nx, ny = GOLD["nx"], GOLD["ny"]
    lat = lbm.Lattice(nx, ny, precision)
    lat.set_params(library_params())
    lat.init_fields(*I.uniform(nx, ny, GOLD["rho_l"], GOLD["T"]))
    frames, at = B.snapshots(lat, GOLD["steps"], GOLD["snapshot_every"])
    g = GOLD["params"]
    ev = B.detachments(frames, at, g["rho_vapor"], g["heater_x0"], g["heater_len"], min_area=GOLD["min_area"])
    st = B.event_statistics(ev, skip=GOLD["skip"])
    assert len(ev) >= GOLD["skip"] + 5, ev
    assert st["diameter"] == pytest.approx(GOLD["mean_diameter"], rel=TOL)
    assert st["period"] == pytest.approx(GOLD["mean_period"], rel=TOL)


def test_per_step_counters_oscillate_with_the_departure_period():
    """The per-step vapour counters of the same channel (bubble_stats = 1) carry the ebullition
    cycle: the vapour around the heater and the contact-line extent L_t (wall footprint, Fig. 17)
    oscillate with the oracle's departure period, while a vapour film keeps the heater covered
    (so departures need the snapshot rule, not the heater footprint)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05264_gb300 import lbm

    nx, ny = GOLD["nx"], GOLD["ny"]
    lat = lbm.Lattice(nx, ny, "fp32")
    lat.set_params(dict(library_params(), bubble_stats=1))
    lat.init_fields(*I.uniform(nx, ny, GOLD["rho_l"], GOLD["T"]))
    s = B.record(lat, GOLD["steps"])
    t = s[:, B.COLUMNS.index("step")]
    late = t >= 12000  # after the start-up departures
    heater = s[late, B.COLUMNS.index("heater_vapor")]
    assert heater.min() == GOLD["params"]["heater_len"]  # the film never leaves the heater
    zone = B.fit_sine(t[late], s[late, B.COLUMNS.index("zone_vapor")])
    wall = B.fit_sine(t[late], s[late, B.COLUMNS.index("wall_vapor")])
    assert zone["period"] == pytest.approx(GOLD["mean_period"], rel=TOL)
    assert wall["period"] == pytest.approx(GOLD["mean_period"], rel=0.03) and wall["amplitude"] > 0.5
