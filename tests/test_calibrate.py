"""Contact-angle calibration: Maxwell coexistence on the host, the table inversion,
and (GPU) the batched sessile-drop measurement against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2009_05264_gb300 import calibrate as C
from paper_2009_05264_gb300 import inputs as I
from paper_2009_05264_gb300 import params as PP


@pytest.mark.parametrize("TR", [0.7, 0.86, 0.9, 0.95])
def test_coexistence_matches_the_oracle_maxwell_construction(TR):
    p = PP.resolve(PP.default_params(geometry="walls", thermal=0), 64)
    T = TR * PP.Tc(p)
    rv, rl, ps = C.coexistence(p, T)
    orv, orl, ops = oracle.maxwell(p, T)
    assert rv == pytest.approx(orv, rel=1e-8) and rl == pytest.approx(orl, rel=1e-9)
    assert ps == pytest.approx(ops, rel=1e-8)
    assert C.pressure(p, rv, T) == pytest.approx(ps, rel=1e-9)


def test_rho_w_for_angle_interpolates_the_monotone_table():
    table = [{"rho_w": 2.0, "theta": 180.0}, {"rho_w": 2.5, "theta": 110.0}, {"rho_w": 3.0, "theta": 83.0},
             {"rho_w": 4.0, "theta": 46.0}, {"rho_w": 5.0, "theta": 0.0}]
    assert C.rho_w_for_angle(110.0, table) == pytest.approx(2.5)
    assert C.rho_w_for_angle(64.5, table) == pytest.approx(3.5)
    with pytest.raises(ValueError):
        C.rho_w_for_angle(130.0, table)
    with pytest.raises(ValueError):
        C.rho_w_for_angle(90.0, [{"rho_w": 2.0, "theta": 50.0}, {"rho_w": 3.0, "theta": 80.0}])


def test_cap_angle_of_a_half_disk_is_ninety_degrees():
    nx, ny, R = 101, 50, 20
    rho = I.sessile(nx, ny, R, 6.0, 0.6, 0.065, width=0.5)[0]
    theta, base, height = C.cap_angle(rho, 6.0, 0.6)
    assert abs(base - 2 * R) <= 1 and abs(height - R) <= 1
    assert theta == pytest.approx(90.0, abs=4.0)


@pytest.mark.gpu
def test_batched_calibration_matches_oracle_drops():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nx, ny, R, steps = 72, 36, 14, 3000
    rho_ws = (1.5, 3.0, 4.5)
    table = C.contact_angles(rho_ws, nx=nx, ny=ny, radius=R, steps=steps)
    assert [r["rho_w"] for r in table] == list(rho_ws)
    thetas = [r["theta"] for r in table]
    assert thetas[0] > thetas[1] > thetas[2]
    p0 = PP.resolve(PP.default_params(geometry="walls", thermal=0, g_a=0.0), nx)
    T = 0.9 * PP.Tc(p0)
    rv, rl, _ = oracle.maxwell(p0, T)
    for r in table:
        O = oracle.Oracle(nx, ny, dict(p0, rho_w=r["rho_w"]))
        O.init_fields(*I.sessile(nx, ny, R, rl, rv, T))
        assert O.step(steps) == 0
        _, base, height = C.cap_angle(O.fields()["rho"], rl, rv)
        assert abs(r["base"] - base) <= 1 and abs(r["height"] - height) <= 1, (r, base, height)
