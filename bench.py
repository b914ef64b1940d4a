"""Benchmark of the fused pseudopotential thermal LB step (MLUPS, fraction of HBM roofline).

Default workload: one flow-boiling channel of 8000 x 800 nodes (6.4 M), FP32
populations stored as deviations from the rest weights, thermal field on, the
microheater switched on, all Sec. 2.C boundary conditions.  One "step" is one
fused kernel launch updating every node's f and g.  Inputs are synthetic
(seeded smooth perturbation of saturated liquid at T_R = 0.9).

Under torchrun each rank advances its own independent channel (replicas; no
data-path collective), so `value` is the total node updates of all ranks per
second ("weak" scaling).

Three sub-measurements ride on the same JSON line (rank 0, single process only):
"fp64", the same channel in FP64; "batch", a seeded sweep of 64 channels of
uneven size and parameters advanced together (one fused launch per step, CUDA
graph replay, autotuned tiles) against the same 64 solved one at a time; and
"serve", Poisson arrivals of channel solves through the continuous-batching
server with p50/p99 time-to-result.

--impl reference times the FP64 CPU oracle (the plain restatement of the
paper used by the tests) on the host cores, on a bounded sample of the same
channel: a 1000 x 800 band of it per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX, NY = 8000, 800  # the 6.4 M-node roofline channel; --nx/--ny shrink it for profiling captures
SEED = 2009052642
WORKLOAD = "single flow-boiling channel 8000x800 D2Q9 + thermal g, FP32 SoA populations"


def workload_params(precision: str):
    from paper_2009_05264_gb300 import params as PP

    return PP.resolve(PP.default_params(geometry="channel", u_in=0.03, dTheat_R=0.08, heater_x0=NX // 5,
                                        heater_len=40, heat_on_step=0, rho_out=5.95), NX)


def bytes_per_node(precision: str, thermal: bool = True) -> int:
    """Algorithmic HBM bytes per node update: every stored population read once and written once."""
    elt = 8 if precision == "fp64" else 4
    return (18 if thermal else 9) * 2 * elt


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in d:
                    v = d[key]
                    return float(v if not isinstance(v, dict) else v.get("value")), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def channel_params(nx: int, u_in: float, dTheat_R: float, rho_w: float | None = None):
    from paper_2009_05264_gb300 import params as PP

    kw = dict(geometry="channel", u_in=u_in, dTheat_R=dTheat_R, heater_len=40, heat_on_step=0, rho_out=5.95)
    if rho_w is not None:
        kw["rho_w"] = rho_w
    return PP.resolve(PP.default_params(**kw), nx)


def channel_fields(nx: int, ny: int, Tc: float, seed: int, instance: int = 0):
    from paper_2009_05264_gb300 import inputs as I

    return I.smooth_random(nx, ny, 5.95, 0.9 * Tc, seed=seed, drho=0.002, du=0.005, dT=0.002, instance=instance)


def run_fp64(steps: int):
    """The same 8000 x 800 channel with FP64 populations: MLUPS and roofline fraction."""
    import torch

    from paper_2009_05264_gb300 import lbm

    p = workload_params("fp64")
    lat = lbm.Lattice(NX, NY, "fp64")
    lat.set_params(p)
    fields = channel_fields(NX, NY, lbm.critical_temperature(p), SEED)
    lat.init_fields(*fields)
    t0 = time.perf_counter()
    tuned = lat.autotune(trial_steps=4)
    tune_s = time.perf_counter() - t0
    lat.init_fields(*fields)  # the trials advanced the lattice
    lat.step(3)
    st = lat.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    lat.step_async(steps)
    e1.record(st)
    lat.sync()
    ms = e0.elapsed_time(e1)
    nodes = NX * NY
    peak, kind = read_peaks()
    gbs = bytes_per_node("fp64") * nodes * steps / (ms * 1e-3) / 1e9
    out = {"value": nodes * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "steps": steps, "ms_per_step": ms / steps,
           "tiling": f"autotuned {tuned[0]}x{tuned[1] or 'default plan'}", "autotune_s": tune_s,
           "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                   "peak_source": f"{kind} HBM copy bandwidth", "algorithmic_bytes_per_node": bytes_per_node("fp64")}}
    fpn = profiled_fp64_flops_per_node()
    peak_tf, peak_src = fp64_peak_tflops()
    out["fp64_fma_peak"] = {"value": peak_tf, "unit": "TFLOP/s", "source": peak_src}
    if fpn:  # FP64 arithmetic, not HBM, bounds this form on GB300
        tf = fpn * nodes * steps / (ms * 1e-3) / 1e12
        out["roofline"] = {"bound": "alu", "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s",
                           "frac": tf / peak_tf, "flops_per_node": fpn, "peak_source": peak_src,
                           "flops_source": f"ncu DADD + DMUL + 2 DFMA per node ({FP64_PROFILE})"}
        ipn = profiled_fp64_figure("fp64-pipe-inst-per-node")
        if ipn:  # DADD and DMUL take an issue slot of the FP64 pipe as a DFMA does, for half its flops
            ti = ipn * nodes * steps / (ms * 1e-3) / 1e12
            slots = peak_tf / 2.0
            out["roofline"]["pipe"] = {"achieved": ti, "peak": slots, "unit": "T FP64 thread-instructions/s",
                                       "frac": ti / slots, "inst_per_node": ipn,
                                       "peak_source": peak_src + " / 2 flops per DFMA"}
    else:
        out["roofline"] = dict(out["hbm"], bound="hbm")
    lat.close()
    return out


def fp64_peak_tflops():
    """FP64 FMA rate of this GPU, measured by the library's probe (independent DFMA chains, CUDA
    events), with the nominal datasheet figure only as a fallback."""
    try:
        from paper_2009_05264_gb300 import lbm

        best = max(lbm.probe_fma_rate("fp64", 1 << 16) for _ in range(3))
        return best / 1e12, "measured: FP64 FMA probe (independent DFMA chains, best of 3, CUDA events)"
    except Exception as exc:  # reporting only
        return FP64_NOMINAL_TFLOPS, f"nominal GB300 FP64 (non-tensor) rate; probe failed: {exc!r}"


def fp32_alu_roofline(kernel: str, nodes: int, step_s: float) -> dict | None:
    """FP32 arithmetic of the FP32 step against the FP32 rate this GPU sustains: the step's FP32
    thread-instructions per node (ncu, committed summary) per second over the probed FFMA rate
    (independent FFMA chains, one instruction per issue slot); None without a current figure."""
    import re

    if kernel not in PROFILES:
        return None
    path = os.path.join(ROOT, PROFILES[kernel])
    if not os.path.exists(path):
        return None
    m = re.search(r"fp32-inst-per-node:\s*([0-9.]+)\s*\(source digest ([0-9a-f]+)", open(path).read())
    if not m or m.group(2) != step_source_digest(kernel):
        return None
    try:
        from paper_2009_05264_gb300 import lbm

        ffma = max(lbm.probe_fma_rate("fp32", 1 << 16) for _ in range(3)) / 2.0  # FFMA per second
    except Exception as exc:  # reporting only
        return {"unavailable": repr(exc)}
    ipn = float(m.group(1))
    achieved = ipn * nodes / step_s
    return {"achieved": achieved / 1e12, "peak": ffma / 1e12, "unit": "T FP32 thread-instructions/s",
            "frac": achieved / ffma, "inst_per_node": ipn,
            "peak_source": "measured: FP32 FMA probe (independent FFMA chains, best of 3, CUDA events)"}


def run_c2(steps: int = 2000, nx: int = 1000, ny: int = 100):
    """The 1000 x 100 channel (heater of 40 nodes at nx/5, u_in = 0.03, superheat 0.08 Tc, as the
    large channel) in FP32 and FP64: MLUPS of each.  Its state (14-29 MB) stays in L2, so no HBM
    fraction is reported for it."""
    import torch

    from paper_2009_05264_gb300 import lbm
    from paper_2009_05264_gb300 import params as PP

    out = {"workload": f"flow-boiling channel {nx}x{ny}, heater 40 nodes at x = {nx // 5}", "steps": steps,
           "note": "state resident in L2: MLUPS only"}
    for prec in ("fp32", "fp64"):
        p = PP.resolve(PP.default_params(geometry="channel", u_in=0.03, dTheat_R=0.08, heater_x0=nx // 5,
                                         heater_len=40, heat_on_step=0, rho_out=5.95), nx)
        lat = lbm.Lattice(nx, ny, prec)
        lat.set_params(p)
        fields = channel_fields(nx, ny, lbm.critical_temperature(p), SEED + 1)
        lat.init_fields(*fields)
        t0 = time.perf_counter()
        tuned = lat.autotune(trial_steps=50 if prec == "fp32" else 10)
        tune_s = time.perf_counter() - t0
        lat.init_fields(*fields)  # the trials advanced the lattice
        lat.step(10)
        st = lat.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = steps if prec == "fp32" else max(100, steps // 10)
        e0.record(st)
        lat.step_async(n)
        e1.record(st)
        lat.sync()
        ms = e0.elapsed_time(e1)
        out[prec] = {"value": nx * ny * n / (ms * 1e-3) / 1e6, "unit": "MLUPS", "steps": n, "ms_per_step": ms / n,
                     "kernel": lat.step_kernel, "tiling": f"autotuned {tuned[0]}x{tuned[1] or 'default plan'}",
                     "autotune_s": tune_s}
        lat.close()
    return out


def run_batch(steps: int, trial_steps: int = 4, n: int = 64, seed: int = SEED + 4):
    """64 seeded channels (Nx U{400..2000}, Ny U{50..200}, u_in U[0.01,0.05], superheat U[0.03,0.12] Tc,
    rho_w U[2.2,4.0] i.e. contact angles of about 137 to 46 degrees), FP32: one batch (autotuned tiles, the
    library's default loop) against one at a time."""
    import torch

    from paper_2009_05264_gb300 import inputs as I
    from paper_2009_05264_gb300 import lbm

    draws = I.sweep_draws(n, seed)
    b = lbm.Batch("fp32", thermal=True)
    members = []
    for k, d in enumerate(draws):
        p = channel_params(d["nx"], d["u_in"], d["dTheat_R"], d["rho_w"])
        m = b.add(d["nx"], d["ny"], p)
        m.init_fields(*channel_fields(d["nx"], d["ny"], lbm.critical_temperature(p), seed, instance=k))
        members.append(m)
    nodes = sum(d["nx"] * d["ny"] for d in draws)
    t0 = time.perf_counter()
    cols, rows = b.autotune(trial_steps=trial_steps)
    tune_s = time.perf_counter() - t0
    b.step(3)
    loop = b.step_loop
    st = b.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = b.launches
    e0.record(st)
    b.step_async(steps)
    e1.record(st)
    b.sync()
    ms_b = e0.elapsed_time(e1)
    launches = b.launches - l0
    # the same lattices one at a time through the single-lattice call (each on its own default tiling)
    e0.record(st)
    for m in members:
        m.step_async(steps)
    e1.record(st)
    for m in members:
        m.sync()
    ms_s = e0.elapsed_time(e1)
    member_ok = [bool(np.isfinite(m.fields()["rho"]).all()) for m in members]
    ok = all(member_ok)
    b.close()
    batched = nodes * steps / (ms_b * 1e-3) / 1e6
    seq = nodes * steps / (ms_s * 1e-3) / 1e6
    peak, kind = read_peaks()
    gbs = bytes_per_node("fp32") * nodes * steps / (ms_b * 1e-3) / 1e9
    return {"workload": f"{n} channels, seeded sweep (seed {seed}), {nodes} nodes in total, FP32", "instances": n,
            "nodes": nodes, "steps": steps, "value": batched, "unit": "MLUPS", "ms_per_step": ms_b / steps,
            "sequential": {"value": seq, "unit": "MLUPS", "ms_per_step": ms_s / steps,
                           "how": "each lattice alone through lbm_step_async, one after another"},
            "speedup_vs_sequential": batched / seq, "tiling": f"{cols}x{rows}", "loop": loop, "autotune_s": tune_s,
            "gpu_launches": launches, "launches_sequential": n * steps, "finite": bool(ok),
            "members_finite": sum(member_ok), "members": len(member_ok),
            "solves_per_hour_50k_steps": n * 3600.0 / (50000 * ms_b * 1e-3 / steps),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_source": f"{kind} HBM copy bandwidth"}}


def run_serve(n_requests: int, steps: int, rate: float = 2.0, seed: int = SEED + 5, tiling=None,
              hbm_budget: int = 32 << 30, chunk: int = 500):
    """Poisson arrivals (rate per second) of channel solves, 80 % sweep draws and 20 % 4000 x 400,
    through the continuous-batching server on the wall clock."""
    from paper_2009_05264_gb300 import inputs as I
    from paper_2009_05264_gb300 import lbm
    from paper_2009_05264_gb300.serve import Request, Server, poisson_arrivals

    rng = np.random.default_rng(seed)
    arrivals = poisson_arrivals(n_requests, rate, seed)
    draws = I.sweep_draws(n_requests, seed + 1)
    reqs = []
    for k in range(n_requests):
        d = draws[k]
        if rng.random() < 0.2:
            d = dict(d, nx=4000, ny=400)
        p = channel_params(d["nx"], d["u_in"], d["dTheat_R"], d["rho_w"])
        fields = channel_fields(d["nx"], d["ny"], lbm.critical_temperature(p), seed, instance=k)
        reqs.append(Request(k, d["nx"], d["ny"], p, fields, steps, float(arrivals[k])))
    srv = Server("fp32", hbm_budget=hbm_budget, chunk=chunk, tiling=tiling)
    t0 = time.monotonic()
    for r in reqs:
        r.arrival += t0
        srv.submit(r)
    done = srv.run()
    wall = max(r.done for r in done if r.done is not None) - t0
    st = srv.stats()
    finite = all(np.isfinite(r.result["rho"]).all() for r in done if r.status == "done")
    peak_resident = srv.peak_resident
    srv.batch.close()
    return {"workload": f"{n_requests} Poisson arrivals at {rate}/s (seed {seed}): 80 % sweep draws, "
                        f"20 % 4000x400; {steps} steps each; FP32", "requests": n_requests, "steps_each": steps,
            "completed": st["completed"], "failed": st["failed"], "rejected": st["rejected"],
            "p50_s": st["p50_s"], "p99_s": st["p99_s"], "unit_latency": "s (arrival to fields on the host)",
            "value": st["node_updates"] / wall / 1e6, "unit": "MLUPS", "wall_s": wall,
            "gpu_busy_frac": st["gpu_busy_s"] / wall, "offered_mlups": float(
                sum(r.nx * r.ny for r in reqs) * steps * rate / n_requests / 1e6),
            "solves_per_hour": st["completed"] * 3600.0 / wall, "peak_resident": peak_resident,
            "hbm_budget_bytes": hbm_budget, "chunk_steps": chunk, "finite": bool(finite)}


_CSRC = "paper_2009_05264_gb300/csrc/"
# sources of each step-kernel form (scalar: also the FP64 step) and its ncu summary
STEP_SOURCES = {"scalar": (_CSRC + "lbm_kernels.cuh", _CSRC + "lbm_internal.h"),
                "interior": (_CSRC + "lbm_kernels.cuh", _CSRC + "lbm_internal.h"),
                "tma": (_CSRC + "lbm_kernels.cuh", _CSRC + "lbm_internal.h", _CSRC + "lbm_tma.cuh")}
PROFILES = {"interior": "profiles/lbm_fused_step_fp32_channel.md", "tma": "profiles/lbm_tma_step_fp32_channel.md"}
KERNEL_LABELS = {"scalar": "lbm_fused_kernel (MODE_STEP)",
                 "interior": "lbm_fused_kernel (MODE_STEP, interior path on tiles away from the open ends)",
                 "paired": "lbm_pair_kernel (two columns per thread, packed FP32)",
                 "tma": "lbm_tma_kernel (MODE_STEP, rows staged by bulk tensor copies)"}


def step_source_digest(kernel: str = "scalar") -> str:
    """Digest of a step kernel's sources: ties a profiled DRAM traffic figure to the
    code it was measured on."""
    import hashlib

    h = hashlib.sha256()
    for rel in STEP_SOURCES[kernel]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


FP64_PROFILE = "profiles/lbm_fused_step_fp64_channel.md"
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (non-tensor) nominal rate: the fallback when the probe cannot run


def profiled_fp64_flops_per_node():
    """FP64 floating-point operations per node update of the step kernel (DADD + DMUL + 2 DFMA,
    counted by ncu), or None when the summary was taken on other kernel sources."""
    return profiled_fp64_figure("fp64-flops-per-node")


def profiled_fp64_figure(key: str):
    """A per-node figure of the FP64 step kernel's committed ncu summary ("fp64-flops-per-node",
    "fp64-pipe-inst-per-node": DADD + DMUL + DFMA thread instructions), or None when the summary
    was taken on other kernel sources."""
    import re

    path = os.path.join(ROOT, FP64_PROFILE)
    if not os.path.exists(path):
        return None
    m = re.search(re.escape(key) + r":\s*([0-9.]+)\s*\(source digest ([0-9a-f]+)", open(path).read())
    if not m or m.group(2) != step_source_digest():
        return None
    return float(m.group(1))


def profiled_traffic_per_node(kernel: str):
    """DRAM bytes per node update of a step kernel form from its committed ncu summary, or
    (None, reason) when there is none or it was taken on other kernel sources."""
    import re

    if kernel not in PROFILES:
        return None, "not profiled"
    path = os.path.join(ROOT, PROFILES[kernel])
    if not os.path.exists(path):
        return None, "no profile summary"
    m = re.search(r"traffic-per-node:\s*([0-9.]+)\s*B\s*\(source digest ([0-9a-f]+)", open(path).read())
    if not m:
        return None, "profile summary has no traffic line"
    if m.group(2) != step_source_digest(kernel):
        return None, "kernel sources changed since the profile"
    return float(m.group(1)), f"ncu dram__bytes_read+write per node ({PROFILES[kernel]})"


def profiled_inst_per_node(kernel: str):
    """Warp-instructions per node update of a step kernel form from its committed ncu summary
    (smsp__inst_executed.sum over the output nodes, halo work included), or None when there is
    none or it was taken on other kernel sources."""
    import re

    if kernel not in PROFILES:
        return None
    path = os.path.join(ROOT, PROFILES[kernel])
    if not os.path.exists(path):
        return None
    m = re.search(r"inst-per-node:\s*([0-9.]+)\s*\(source digest ([0-9a-f]+)", open(path).read())
    if not m or m.group(2) != step_source_digest(kernel):
        return None
    return float(m.group(1))


def issue_roofline(inst_per_node: float, nodes: int, launch_s: float, sms: int, sm_mhz: float) -> dict:
    """Instruction issue of a step launch against the issue peak: every SM issues at most one
    warp-instruction per clock from each of its four schedulers."""
    achieved = inst_per_node * nodes / launch_s / 1e9
    peak = sms * 4 * sm_mhz * 1e6 / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "G warp-instructions/s", "frac": achieved / peak,
            "inst_per_node": inst_per_node,
            "peak_source": f"{sms} SMs x 4 schedulers x the sampled {sm_mhz:.0f} MHz SM clock"}


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of every rank's value (the slowest rank's time); the value itself on one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Node updates of all ranks per second (weak scaling: every rank advances its own lattice)."""
    return nodes_per_rank * steps * world / seconds / 1e6


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_rate(steps: int, nx: int, threads: int):
    """MLUPS of the oracle as it stands on `threads` host threads: `steps` steps of a nx x NY band
    of the benchmark channel (its rows spread over the threads; same results at any count)."""
    import oracle
    from paper_2009_05264_gb300 import inputs as I

    p = workload_params("fp64")
    Tc = oracle.Tc(p)
    fields = I.smooth_random(nx, NY, 5.95, 0.9 * Tc, seed=SEED, drho=0.002, du=0.005, dT=0.002)
    orc = oracle.Oracle(nx, NY, p, threads=threads)
    orc.init_fields(*fields)
    t0 = time.perf_counter()
    st = orc.step(steps)
    dt = time.perf_counter() - t0
    if st != 0:
        raise RuntimeError("oracle unstable on the baseline sample")
    return nx * NY * steps / dt / 1e6, dt


def cpu_baseline(steps: int = 60, nx: int = 1000):
    """The oracle as it stands on the host: all cores (OpenMP over rows, serial fixed-order sums)
    on `steps` steps of a nx x 800 band of the channel, and one core on a third of them
    (about 10-20 s of CPU work in all)."""
    cores = os.cpu_count() or 1
    v_all, dt_all = oracle_rate(steps, nx, cores)
    s1 = max(steps // 3, 5)
    v_one, dt_one = oracle_rate(s1, nx, 1)
    return {"value": v_all, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps of a {nx}x{NY} band of the channel (same physics), FP64, "
                      f"{cores} threads (OpenMP over rows)", "seconds": dt_all, "cpu_model": cpu_model(),
            "single_core": {"value": v_one, "unit": "MLUPS", "cores": 1, "seconds": dt_one,
                            "sample": f"{s1} steps of the same band, one thread"}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle  # noqa: F401

    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_rate(1, 200, cores)
    t0 = time.perf_counter()
    per = []
    for _ in range(args.steps):
        per.append(oracle_rate(1, 2000, cores)[1])
    total = time.perf_counter() - t0
    value = 2000 * NY * args.steps / sum(per) / 1e6
    line = {"impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY,
                       "sample": f"each step: one oracle step on a 2000x{NY} band"},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"one step of a 2000x{NY} band per timed step, {cores} threads (OpenMP "
                                       f"over rows)", "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2009_05264_gb300 import inputs as I
    from paper_2009_05264_gb300 import lbm

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = args.precision
    p = workload_params(prec)
    Tc = lbm.critical_temperature(p)
    fields = I.smooth_random(NX, NY, 5.95, 0.9 * Tc, seed=SEED, drho=0.002, du=0.005, dT=0.002, instance=rank)

    lat = lbm.Lattice(NX, NY, prec, device=local)
    lat.set_params(p)
    if args.tiling:
        c, r = (int(x) for x in args.tiling.split("x"))
        lat.set_tiling(c, r)
    lat.set_kernel(args.kernel)
    lat.set_step_loop(args.loop)
    step_kernel = lat.step_kernel  # the form the timed launches take
    t = lat.tiling
    tiling_desc = (f"{t['cols']} columns; per strip {t['tall_count']} bands of {t['tall_rows']} rows, then bands of "
                   f"{t['short_rows']}" + ("" if args.tiling else " (default plan)"))
    lat.init_fields(*fields)
    stream = lat.stream
    nodes = NX * NY

    # warm-up
    lat.step(args.warmup)

    # ---- device-timed region: inputs resident in HBM (state 2 x 0.92 GB > L2) ----
    # one call advances the K timed steps, as a user's multi-step call does: the library's
    # default loop runs them as one overlapped persistent launch on this lattice (or one
    # launch per step where that is its choice); CUDA events on the library's stream bracket it
    loop = lat.step_loop
    events = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(local) if rank == 0 else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    launches0 = lat.launches
    events[0].record(stream)
    lat.step_async(args.steps)
    events[1].record(stream)
    torch.cuda.synchronize()
    lat.sync()
    gpu_launches = lat.launches - launches0
    total_ms = events[0].elapsed_time(events[1])
    clocks = sampler.stop() if sampler else None
    if world > 1:
        dist.barrier()
    total_ms = max_over_ranks(total_ms, world, dev)
    value = whole_job_mlups(nodes, args.steps, world, total_ms * 1e-3)

    # ---- end to end through the public API with host buffers ----
    pinned = [torch.empty((NY, NX), dtype=torch.float64).pin_memory() for _ in range(4)]
    for a, src in zip(pinned, fields):
        a.numpy()[...] = src
    outs = [torch.empty((NY, NX), dtype=torch.float64).pin_memory() for _ in range(4)]
    e2e_steps = args.steps
    e2e_s = None
    for _ in range(2):  # the better of two runs: one host-side stall should not decide the figure
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.init_fields(*[a.numpy() for a in pinned])
        lat.step(e2e_steps)
        got = lat.fields(out={k: o.numpy() for o, k in zip(outs, ("rho", "ux", "uy", "T"))})  # into pinned memory
        dt = time.perf_counter() - t0
        e2e_s = dt if e2e_s is None else min(e2e_s, dt)
    e2e_value = whole_job_mlups(nodes, e2e_steps, world, max_over_ranks(e2e_s, world, dev))
    if not np.isfinite(got["rho"]).all():
        raise RuntimeError("non-finite density after the e2e run")

    if rank == 0:
        peak, peak_kind = read_peaks()
        bpn = bytes_per_node(prec)
        step_ms = total_ms / args.steps  # the step kernel's time per step (launches or one persistent launch)
        achieved = bpn * nodes / (step_ms * 1e-3) / 1e9
        tpn, tsrc = profiled_traffic_per_node(step_kernel)
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if prec == "fp32" else WORKLOAD.replace("FP32", "FP64"),
                       "nx": NX, "ny": NY, "nodes_per_gpu": nodes, "precision": prec,
                       "tiling": tiling_desc,
                       "kernel": f"{step_kernel} (requested {args.kernel})",
                       "loop": loop,
                       "l2": "inputs larger than L2: 2 x 0.92 GB population buffers vs 129 MB L2",
                       "parallelism": f"{world} independent channel replicas"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": tpn * nodes if tpn else None,
                         "traffic_per": "step (the timed launch runs all timed steps; achieved is per step too)",
                         "traffic_source": tsrc,
                         "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "algorithmic_bytes_per_node": bpn,
                         "kernel": KERNEL_LABELS[step_kernel] + (
                             ", all timed steps in one lbm_persistent_kernel launch that overlaps consecutive steps"
                             if loop == "overlapped" else "")},
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": 4 * nodes * 8 / e2e_steps, "d2h_bytes_per_step": 4 * nodes * 8 / e2e_steps,
                    "note": f"init_fields from pinned host arrays + {e2e_steps} steps + read_fields into pinned host arrays"
                            " (the better of two runs)"},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
        }
        if prec == "fp32":  # FP32 arithmetic is far from its rate: reported to show it is not the bound
            alu = fp32_alu_roofline(step_kernel, nodes, step_ms * 1e-3)
            if alu:
                line["roofline"]["alu"] = alu
        ipn = profiled_inst_per_node(step_kernel) if prec == "fp32" else None
        if ipn and clocks and clocks.get("sm_mhz"):  # the step is issue-bound: its fraction of the issue peak
            try:
                sms = torch.cuda.get_device_properties(dev).multi_processor_count
                line["roofline"]["issue"] = issue_roofline(ipn, nodes, step_ms * 1e-3, sms, clocks["sm_mhz"])
            except Exception as exc:  # reporting only: never lose the line over it
                line["roofline"]["issue"] = {"unavailable": repr(exc)}
        if world == 1 and not args.no_extras:
            lat.close()
            line["fp64"] = run_fp64(max(10, args.steps // 10))
            line["c2"] = run_c2()
            line["batch"] = run_batch(args.batch_steps)
            # the server keeps each member's default band plan: a fixed band height tuned for the
            # 64-channel sweep leaves the served mix (a few lattices, some 4000 x 400) slower
            line["serve"] = run_serve(args.serve_requests, args.serve_steps, tiling=None)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--tiling", default=None, help="COLSxROWS, e.g. 128x32")
    ap.add_argument("--kernel", default="auto", choices=["auto", "scalar", "paired", "tma", "interior"],
                    help="step kernel form")
    ap.add_argument("--loop", default="auto", choices=["auto", "launches", "persistent"],
                    help="profiling only: the step loop of the timed call (default: the library's choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the fp64, batch and serve measurements")
    ap.add_argument("--batch-steps", type=int, default=300)
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve-steps", type=int, default=20000)
    ap.add_argument("--nx", type=int, default=None, help="profiling only: smaller channel length")
    ap.add_argument("--ny", type=int, default=None, help="profiling only: smaller channel height")
    args = ap.parse_args()
    global NX, NY
    if args.nx:
        NX = args.nx
    if args.ny:
        NY = args.ny
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
