"""The default step tiling (host logic of the library; no GPU needed)."""
import pytest

from paper_2009_05264_gb300 import lbm


def model_cost(nx, ny, cols, slots, plan):
    """Row-iterations per CTA slot in the documented model: every tile costs its rows plus 4
    halo rows plus one row of fixed cost, spread over the slots, plus half a tile of the
    class dispatched last."""
    strips = -(-nx // (cols - 8))
    work, y = 0.0, 0
    for _ in range(plan["tall_count"]):
        work += strips * (plan["tall_rows"] + 5)
        y += plan["tall_rows"]
    while y < ny:
        work += strips * (min(plan["short_rows"], ny - y) + 5)
        y += plan["short_rows"]
    return work / slots + 0.5 * (plan["short_rows"] + 5)


def rows_covered(ny, plan):
    bands = [plan["tall_rows"]] * plan["tall_count"]
    y = plan["tall_count"] * plan["tall_rows"]
    while y < ny:
        bands.append(min(plan["short_rows"], ny - y))
        y += plan["short_rows"]
    return bands


def test_benchmark_channel_plan():
    # 8000 x 800, 128-column CTAs, 152 SMs x 5 CTAs: 14 bands of 40 rows, then 20-row bands
    assert lbm.default_band_plan(8000, 800, 128, 760) == {"tall_rows": 40, "tall_count": 14, "short_rows": 20}


@pytest.mark.parametrize("nx,ny", [(8000, 800), (4000, 800), (2000, 800), (4000, 400), (16000, 1600), (1200, 125),
                                   (300, 37), (1000, 100), (6, 5), (3, 2), (130, 4)])
@pytest.mark.parametrize("cols,slots", [(128, 760), (64, 1520), (256, 304), (128, 64)])
def test_plan_covers_every_row_and_is_the_cheapest_candidate(nx, ny, cols, slots):
    plan = lbm.default_band_plan(nx, ny, cols, slots)
    bands = rows_covered(ny, plan)
    assert sum(bands) == ny and all(b >= 1 for b in bands)
    assert plan["short_rows"] >= min(4, ny)
    strips = -(-nx // (cols - 8))
    ks = -(-slots // strips)
    if plan["tall_count"]:
        h = plan["short_rows"]
        assert plan["tall_rows"] == 2 * h and (ks + 2) * h <= ny
    # no candidate of the model is cheaper: uniform bands of the balanced heights ceil(ny / b)
    # >= 4 rows, every band charged that height, and two-level plans with h >= 4
    best = model_cost(nx, ny, cols, slots, plan)
    if plan["tall_count"] == 0:  # a uniform plan is charged as the library charges uniform bands
        r = plan["short_rows"]
        best = strips * -(-ny // r) * (r + 5) / slots + 0.5 * (r + 5)
    heights = {ny} if ny <= 4 else {-(-ny // b) for b in range(1, ny + 1) if -(-ny // b) >= 4}
    for r in heights:
        assert best <= strips * -(-ny // r) * (r + 5) / slots + 0.5 * (r + 5) + 1e-9
    h = 4
    while (ks + 2) * h <= ny:
        cand = {"tall_rows": 2 * h, "tall_count": (ny - ks * h) // (2 * h), "short_rows": h}
        assert best <= model_cost(nx, ny, cols, slots, cand) + 1e-9
        h += 1


def test_plan_rejects_invalid_arguments():
    for args in [(0, 10, 128, 760), (10, 0, 128, 760), (100, 100, 96, 760), (100, 100, 128, 0)]:
        with pytest.raises(lbm.LbmError):
            lbm.default_band_plan(*args)
