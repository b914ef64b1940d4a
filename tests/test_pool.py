"""Pool-boiling helpers on the CPU: the power-law regression and the pool's parameters."""
import math

import numpy as np
import pytest

from paper_2009_05264_gb300 import pool


def test_power_law_fit_recovers_the_papers_regression():
    g = np.array([5e-5, 1e-4, 2e-4, 5e-4, 1e-3])
    c, n = pool.fit_power_law(g, 0.246 * g ** -0.49)  # Sec. 2.D: D_d = 0.246 g^-0.49
    assert c == pytest.approx(0.246, rel=1e-10) and n == pytest.approx(-0.49, abs=1e-12)
    noisy = 0.246 * g ** -0.49 * np.exp(np.random.default_rng(3).normal(0, 0.01, g.size))
    c, n = pool.fit_power_law(g, noisy)
    assert n == pytest.approx(-0.49, abs=0.03)


def test_pool_parameters():
    p, rho_l, rho_v = pool.pool_params(2e-4, nx=128, heater_len=10)
    assert p["geometry"] == 3 and p["g_a"] == 2e-4 and p["heat_on_step"] == 0
    assert p["heater_x0"] == 59 and p["heater_len"] == 10  # centred on the bottom wall
    assert rho_l == pytest.approx(5.8812, abs=1e-3) and rho_v == pytest.approx(0.5902, abs=1e-3)
    assert p["rho_out"] == rho_l and p["rho_vapor"] == pytest.approx(0.5 * (rho_l + rho_v))
    assert p["T0_R"] == p["Tin_R"] == 0.9
