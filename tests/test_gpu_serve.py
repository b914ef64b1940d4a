"""Serving on the GPU: requests that arrive while others run share the batch, and each
result is the same as the lattice solved alone (same tiling), to FP32 rounding: the batch
and a lattice alone run separately compiled instantiations of the same tile code, whose
multiply-add fusion may differ (1e-6 of each field's scale, inside the 1e-5 parity
tolerance)."""
import numpy as np
import pytest

import oracle
from paper_2009_05264_gb300 import inputs as I
from paper_2009_05264_gb300 import params as PP
from paper_2009_05264_gb300.serve import FakeClock, Request, Server

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_results_alone_and_in_the_mix_agree():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_05264_gb300 import lbm

    rng = np.random.default_rng(2009052644)
    reqs = []
    for k in range(5):
        nx, ny = int(rng.integers(120, 400)), int(rng.integers(40, 90))
        p = PP.resolve(PP.default_params(geometry="channel", u_in=float(rng.uniform(0.01, 0.04)),
                                         dTheat_R=float(rng.uniform(0.03, 0.12)), heat_on_step=10, heater_len=10,
                                         g_a=1e-4), nx)
        Tc = oracle.Tc(p)
        fields = I.smooth_random(nx, ny, 5.95, 0.9 * Tc, seed=500 + k, drho=0.002, du=0.005, dT=0.002)
        reqs.append(Request(k, nx, ny, p, fields, steps=int(rng.integers(40, 120)), arrival=3.0 * k))
    clock = FakeClock(tick=1.0)
    srv = Server("fp32", chunk=16, clock=clock, tiling=(128, 16))
    for r in reqs:
        srv.submit(r)
    done = {r.rid: r for r in srv.run()}
    assert all(done[k].status == "done" for k in range(5))
    assert srv.batch.launches > 0 and len(srv.batch) == 0
    overlapped = sum(1 for a in done.values() for b in done.values()
                     if a.rid < b.rid and b.admitted < a.done)
    assert overlapped >= 2  # later requests joined while earlier ones were running
    for r in reqs:
        lat = lbm.Lattice(r.nx, r.ny, "fp32")
        lat.set_params(r.params)
        lat.set_tiling(128, 16)
        lat.init_fields(*r.fields)
        lat.step(r.steps)
        alone = lat.fields()
        for key in ("rho", "ux", "uy", "T"):
            scale = np.abs(alone[key]).max() if key in ("rho", "T") else max(np.abs(alone["ux"]).max(),
                                                                          np.abs(alone["uy"]).max())
            err = np.abs(done[r.rid].result[key] - alone[key]).max() / scale
            assert err <= 1e-6, (r.rid, key, err)
        assert done[r.rid].result["diagnostics"]["step"] == r.steps - 1
