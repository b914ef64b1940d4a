"""Serving loop for parameter-sweep channel solves: continuous batching on one GPU.

Requests (a lattice size, parameters, initial fields and a number of steps) are
admitted into a running batch (``lbm.Batch``) as soon as device memory allows:
admission happens between chunks of steps, first come first served, against a
device-memory budget counted with ``lbm_required_bytes``.  Admitted lattices stay
resident on the device; every chunk advances all of them with one fused launch
per step, so work that arrives while others are running overlaps with them on the
GPU.  When a request has done its steps its fields are read back, its memory is
freed and its time-to-result recorded.  A request's result is the same as the
lattice run alone with the batch's tiling.

The clock and the batch backend are injectable: tests drive the loop with a fake
clock and (for the scheduling logic alone) a fake backend.
"""
from __future__ import annotations

import dataclasses
import heapq
import math
import time
from typing import Callable

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    nx: int
    ny: int
    params: dict
    fields: tuple          # (rho, ux, uy, T) initial fields, (ny, nx) each
    steps: int
    arrival: float = 0.0   # clock time at which the request becomes visible
    # filled in by the server
    admitted: float | None = None
    done: float | None = None
    result: dict | None = None
    status: str = "queued"  # queued, running, done, rejected, failed

    @property
    def latency(self) -> float | None:
        return None if self.done is None else self.done - self.arrival


class Server:
    """Continuous-batching loop over one ``lbm.Batch``.

    hbm_budget: bytes of device memory the resident lattices may use (None: no limit).
    chunk: most steps advanced between admission points.
    """

    def __init__(self, precision: str = "fp32", thermal: bool = True, hbm_budget: int | None = None,
                 chunk: int = 500, clock: Callable[[], float] | None = None, backend=None,
                 bytes_of: Callable[[int, int], int] | None = None, tiling: tuple | None = None):
        self.precision = precision
        self.chunk = int(chunk)
        self.clock = clock or time.monotonic
        if backend is None:
            from . import lbm

            backend = lbm.Batch(precision, thermal=thermal)
            lib = lbm.load()
            code = lbm.FP64 if precision in ("fp64", "f64") else lbm.FP32
            bytes_of = bytes_of or (lambda nx, ny: int(lib.lbm_required_bytes(nx, ny, code)))
        self.batch = backend
        if tiling:
            self.batch.set_tiling(*tiling)
        self.bytes_of = bytes_of or (lambda nx, ny: 0)
        self.hbm_budget = hbm_budget
        self.in_use = 0
        self._arrivals: list = []        # heap of (arrival, rid, request) not yet visible
        self._queue: list[Request] = []  # visible, waiting for memory (FIFO)
        self._running: dict[int, tuple] = {}  # slot -> (request, member, remaining steps)
        self.finished: list[Request] = []
        self.node_updates = 0
        self.busy_time = 0.0
        self.peak_resident = 0

    # ------------------------------------------------------------------ intake
    def submit(self, req: Request):
        heapq.heappush(self._arrivals, (req.arrival, req.rid, req))

    def _release_arrivals(self, now: float):
        while self._arrivals and self._arrivals[0][0] <= now:
            self._queue.append(heapq.heappop(self._arrivals)[2])

    def _admit(self, now: float):
        while self._queue:
            req = self._queue[0]
            need = self.bytes_of(req.nx, req.ny)
            if self.hbm_budget is not None and need > self.hbm_budget:
                self._queue.pop(0)
                req.status = "rejected"  # can never fit
                self.finished.append(req)
                continue
            if self.hbm_budget is not None and self.in_use + need > self.hbm_budget:
                break  # first come first served: wait for memory
            self._queue.pop(0)
            member = self.batch.add(req.nx, req.ny, req.params)
            member.init_fields(*req.fields)
            self.in_use += need
            req.admitted = now
            req.status = "running"
            self._running[member.slot] = (req, member, req.steps)
            self.peak_resident = max(self.peak_resident, len(self._running))

    # ------------------------------------------------------------------ loop
    @property
    def idle(self) -> bool:
        return not (self._arrivals or self._queue or self._running)

    def run_once(self) -> bool:
        """One admission point and at most one chunk of steps; False when idle."""
        now = self.clock()
        self._release_arrivals(now)
        self._admit(now)
        if not self._running:
            if self._arrivals:
                self._wait_until(self._arrivals[0][0])
                return True
            return bool(self._queue)
        n = min(self.chunk, min(rem for _, _, rem in self._running.values()))
        t0 = time.perf_counter()
        try:
            self.batch.step(n)
        except Exception as exc:  # one or more members left the EOS domain
            self._fail_unstable(exc)
        self.busy_time += time.perf_counter() - t0
        now = self.clock()
        for slot, (req, member, rem) in list(self._running.items()):
            self.node_updates += req.nx * req.ny * n
            rem -= n
            if rem > 0:
                self._running[slot] = (req, member, rem)
                continue
            req.result = member.fields()
            req.result["diagnostics"] = member.diagnostics()
            req.done = self.clock()
            req.status = "done"
            self.finished.append(req)
            self._retire(slot, req)
        return True

    def _fail_unstable(self, exc: Exception):
        """Retire the members whose own state reports the failure; the others carry on.

        Members are independent lattices, so one that diverged does not touch the
        rest of the batch.  If no member owns the error, the whole running set fails.
        """
        bad = []
        for slot, (req, member, rem) in self._running.items():
            try:
                member.sync()
            except Exception as e:  # this member's own status is set
                bad.append((slot, req, str(e)))
        if not bad:
            bad = [(slot, req, str(exc)) for slot, (req, _, _) in self._running.items()]
        for slot, req, msg in bad:
            req.status = "failed"
            req.result = {"error": msg}
            req.done = self.clock()
            self.finished.append(req)
            self._retire(slot, req)

    def _retire(self, slot: int, req: Request):
        self._running.pop(slot, None)
        self.batch.remove(slot)
        self.in_use -= self.bytes_of(req.nx, req.ny)

    def _wait_until(self, t: float):
        advance = getattr(self.clock, "advance_to", None)
        if advance is not None:
            advance(t)
        else:
            delay = t - self.clock()
            if delay > 0:
                time.sleep(delay)

    def run(self):
        while not self.idle:
            self.run_once()
        return self.finished

    # ------------------------------------------------------------------ report
    def stats(self) -> dict:
        lat = sorted(r.latency for r in self.finished if r.status == "done")
        def pct(q):
            if not lat:
                return None
            k = min(len(lat) - 1, max(0, math.ceil(q * len(lat)) - 1))
            return lat[k]
        return {"completed": len(lat), "rejected": sum(r.status == "rejected" for r in self.finished),
                "failed": sum(r.status == "failed" for r in self.finished), "p50_s": pct(0.50), "p99_s": pct(0.99),
                "node_updates": self.node_updates, "gpu_busy_s": self.busy_time}


class FakeClock:
    """Deterministic clock for tests: advances by a fixed amount per reading."""

    def __init__(self, tick: float = 0.0):
        self.t = 0.0
        self.tick = tick

    def __call__(self) -> float:
        self.t += self.tick
        return self.t

    def advance_to(self, t: float):
        self.t = max(self.t, t)


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times of n requests of a Poisson process with the given rate (per second)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
