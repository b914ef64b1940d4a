"""Writes departures_channel_600x80.json: the bubble departures of a heated channel
computed by the FP64 CPU oracle alone, the long-run reference of the GPU steps.

Sec. 3.B reports the departure diameter averaged over five departures and the
departure period averaged over four.  A departure here is a connected vapour region
(rho below the mid density of the coexisting phases, 4-connected) that touches none
of the heater sites, overlaps the vapour attached to the heater one snapshot earlier
and overlaps no region that was already detached there; its diameter is that of the
circle of its area, 2 sqrt(A / pi).  This script implements that rule itself (with
scipy's connected-component labelling as the one library primitive), independently of
the package's bubble module, which the GPU test uses.

Run from the repository root (about ten minutes on one core):
    python tests/golden/make_departures.py
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2009_05264_gb300 import inputs  # noqa: E402  (seeded input generators only)

NX, NY, STEPS, EVERY, MIN_AREA, SKIP = 600, 80, 40000, 25, 20, 3
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "departures_channel_600x80.json")


def channel_params(rho_l: float, rho_v: float) -> dict:
    """The oracle's parameters: the paper's fluid and forcing constants (Sec. 2.A), a
    channel with inlet, outlet and walls (Sec. 2.C), heater 40 nodes at x = 120 switched
    on from the start at 0.3 Tc superheat (Sec. 3.A), u_in = 0.005, g = 2e-4, rho_w = 3.0."""
    beta, G = 1.16, -1.0
    return dict(geometry=1, thermal=1, multiphase=1, tau_f=1.0, tau_g=0.6, a=2.0 / 49.0, b=2.0 / 21.0, R=1.0,
                omega=0.32, beta=beta, c0=6.0, G=G, T0_R=0.9, Tin_R=0.9, dTheat_R=0.3, u_in=0.005, rho_out=rho_l,
                rho_w=3.0, G_wet=9.0 * (1.0 + beta) * G, g_a=2e-4, c_v=6.0, heater_x0=120, heater_len=40,
                heat_on_step=0, rho_vapor=0.5 * (rho_l + rho_v), source_model=0, reserved0=0)


def departures(frames, steps, thr, x0, n):
    from scipy import ndimage

    events, prev_att, prev_det = [], None, None
    for rho, step in zip(frames, steps):
        lab, count = ndimage.label(rho < thr)
        heater = set(int(v) for v in lab[0, x0:x0 + n]) - {0}
        area = np.bincount(lab.ravel(), minlength=count + 1)
        att = np.isin(lab, sorted(heater))
        det = np.zeros_like(att)
        for c in range(1, count + 1):
            if c in heater or area[c] < MIN_AREA:
                continue
            comp = lab == c
            det |= comp
            if prev_att is not None and (comp & prev_att).any() and not (comp & prev_det).any():
                events.append({"step": int(step), "area": int(area[c])})
        prev_att, prev_det = att, det
    return events


def main():
    probe = channel_params(1.0, 0.1)
    Tc = oracle.Tc(probe)
    T = 0.9 * Tc
    rho_v, rho_l, _ = oracle.maxwell(probe, T)
    p = channel_params(rho_l, rho_v)
    orc = oracle.Oracle(NX, NY, p)
    orc.init_fields(*inputs.uniform(NX, NY, rho_l, T))
    frames, at = [], []
    t0 = time.time()
    for k in range(STEPS // EVERY):
        st = orc.step(EVERY)
        if st != 0:
            raise RuntimeError(f"oracle unstable at step {orc.step_count}")
        frames.append(orc.fields()["rho"].astype(np.float32))
        at.append(orc.step_count)
    ev = departures(frames, at, p["rho_vapor"], p["heater_x0"], p["heater_len"])
    use = ev[SKIP:]
    diam = [2.0 * math.sqrt(e["area"] / math.pi) for e in use[:5]]
    steps = [e["step"] for e in use[:5]]
    doc = {
        "_about": "Bubble departures of a heated channel from the FP64 CPU oracle (written by "
                  "tests/golden/make_departures.py, which calls only oracle/ and the seeded inputs). "
                  "Sec. 3.B averages the departure diameter over five departures and the period over four.",
        "nx": NX, "ny": NY, "steps": STEPS, "snapshot_every": EVERY, "min_area": MIN_AREA, "skip": SKIP,
        "rho_l": rho_l, "rho_v": rho_v, "T": T, "params": p, "events": ev,
        "mean_diameter": float(np.mean(diam)), "mean_period": float(np.mean(np.diff(steps))),
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps({k: doc[k] for k in ("mean_diameter", "mean_period", "oracle_seconds")}), len(ev), "events")


if __name__ == "__main__":
    main()
