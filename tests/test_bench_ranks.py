"""The benchmark's multi-rank bookkeeping on CPU: world_size-2 gloo ranks (replicas,
no data-path collective; only the timing reduction and the whole-job aggregate)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        slowest = bench.max_over_ranks(1.0 + rank, w)  # rank 1 is slower
        q.put((r, w, slowest, bench.whole_job_mlups(1000, 10, w, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_whole_job_rate():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 2.0 for o in out)  # both ranks see the slower rank's time
    assert all(o[3] == pytest.approx(1000 * 10 * 2 / 2.0 / 1e6) for o in out)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_mlups(6_400_000, 300, 1, 0.08) == pytest.approx(24000.0)


def test_fp64_pipe_figure_is_consistent_with_the_flop_figure():
    """DADD + DMUL + DFMA instructions per node lie between half the flops (all DFMA) and the flops
    (no DFMA); both figures come from the same committed summary, or neither does."""
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    flops = bench.profiled_fp64_flops_per_node()
    inst = bench.profiled_fp64_figure("fp64-pipe-inst-per-node")
    assert (flops is None) == (inst is None)
    if flops is not None:
        assert flops / 2 <= inst <= flops


def test_issue_roofline_arithmetic_and_profile_figures():
    """The issue figure is warp-instructions per node x nodes / launch time against 4 per SM per
    clock; the committed per-node counts come from the same summaries as the traffic figures."""
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    r = bench.issue_roofline(30.0, 1_000_000, 1e-3, 100, 2000.0)
    assert r["achieved"] == pytest.approx(30.0)      # 3e7 warp-instructions in 1 ms
    assert r["peak"] == pytest.approx(800.0)         # 100 SMs x 4 x 2 GHz
    assert r["frac"] == pytest.approx(30.0 / 800.0)
    for kernel in ("scalar", "tma"):
        ipn = bench.profiled_inst_per_node(kernel)
        tpn, _ = bench.profiled_traffic_per_node(kernel)
        assert (ipn is None) == (tpn is None)
        if ipn is not None:
            assert 10.0 < ipn < 60.0
    assert bench.profiled_inst_per_node("paired") is None
