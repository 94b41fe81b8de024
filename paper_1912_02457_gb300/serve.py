"""Continuous-batching forecast server on top of the libswe batch API.

On-demand forecasts (the search-and-rescue / oil-spill use the paper's
introduction motivates) arrive at random times with uneven domain sizes and
horizons. The server:

* admits waiting requests in arrival order whenever their device memory fits
  the budget (each admitted domain keeps its state and forcing resident);
* advances every admitted domain together in rounds of ``round_steps``
  batched steps (one launch per RK stage, graph-replayed), each
  domain on its own clock up to its own horizon;
* after each round retires the domains that reached their horizon (their
  final state is downloaded to the host) and admits new arrivals, so work
  from requests that arrive while others run overlaps on the device.

The GPU side is ``swe.Batch``; everything here is host bookkeeping. A fake
backend with the same interface lets the admission logic be tested without
a GPU.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, List, Optional

import numpy as np


def domain_bytes(nx: int, ny: int, precision: str = "f32_kahan", f_plane=True,
                 theta_plane=True) -> int:
    """Device bytes a domain holds (planes padded to 128-byte rows)."""
    pitch = -(-nx // 32) * 32
    cpitch = -(-(nx + 1) // 32) * 32
    planes = 6 + 3 + (3 if precision == "f32_kahan" else 0) + int(f_plane) + int(theta_plane)
    return 4 * (planes * pitch * ny + cpitch * (ny + 1)) + 64 * 1024


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the trace
    make_workload: Callable        # () -> synth.Workload (client side)
    horizon: float                 # simulated seconds
    nx: int = 0
    ny: int = 0
    precision: str = "f32_kahan"
    cancelled: bool = False
    # filled by the server
    admitted: Optional[float] = None
    finished: Optional[float] = None
    result: Optional[tuple] = None
    steps: int = 0
    error: Optional[str] = None


class GpuBackend:
    """libswe-backed execution (one batch on one stream)."""

    def __init__(self, stream: int = 0):
        from paper_1912_02457_gb300 import swe
        self.swe = swe
        self.batch = swe.Batch(stream)
        self.stream = stream

    def open(self, wl, precision, horizon):
        d = self.swe.Domain(wl, precision, stream=self.stream)
        d.set_end_time(wl.t0 + horizon)
        self.batch.add(d)
        return d

    def step(self, n):
        self.batch.step(n)

    def poll(self, handles):
        done, t = self.batch.poll()
        idx = {id(d): k for k, d in enumerate(self.batch.domains)}
        return [bool(done[idx[id(h)]]) for h in handles]

    def close(self, h, download=True):
        self.batch.remove(h)
        out = h.state() if download else None
        info = h.info(check=False)
        h.close()
        return out, info.step

    def shutdown(self):
        self.batch.close()


class ForecastServer:
    def __init__(self, backend, budget_bytes: float = 150e9, round_steps: int = 64,
                 clock: Callable[[], float] = time.perf_counter):
        self.backend = backend
        self.budget = float(budget_bytes)
        self.round_steps = int(round_steps)
        self.clock = clock
        self.used = 0
        self.peak_used = 0
        self.active = []           # (request, handle, bytes)
        self.rounds = 0

    def _admit(self, waiting: List[Request], now: float):
        while waiting and waiting[0].arrival <= now:
            r = waiting[0]
            if r.cancelled:
                waiting.pop(0)
                r.error = "cancelled before admission"
                r.finished = now
                continue
            need = domain_bytes(r.nx, r.ny, r.precision)
            if need > self.budget:
                waiting.pop(0)
                r.error = "larger than the device budget"
                r.finished = now
                continue
            if self.used + need > self.budget:
                return                    # wait for memory (arrival order kept)
            waiting.pop(0)
            try:
                wl = r.make_workload()
                h = self.backend.open(wl, r.precision, r.horizon)
            except Exception as exc:      # malformed request / allocation failure
                r.error = f"rejected: {exc}"
                r.finished = now
                continue
            r.admitted = now
            self.used += need
            self.peak_used = max(self.peak_used, self.used)
            self.active.append((r, h, need))

    def run(self, requests: List[Request], time_limit: float = 3600.0):
        waiting = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock()
        while waiting or self.active:
            now = self.clock() - t0
            if now > time_limit:
                break
            self._admit(waiting, now)
            # requests cancelled while running leave at the next round boundary
            for r, h, need in list(self.active):
                if r.cancelled:
                    self.backend.close(h, download=False)
                    self.used -= need
                    self.active.remove((r, h, need))
                    r.error = "cancelled"
                    r.finished = self.clock() - t0
            if not self.active:
                if waiting:
                    nxt = waiting[0].arrival
                    delay = nxt - (self.clock() - t0)
                    if delay > 0:
                        time.sleep(min(delay, 0.05))
                continue
            self.backend.step(self.round_steps)
            self.rounds += 1
            done = self.backend.poll([h for _, h, _ in self.active])
            for (r, h, need), d in list(zip(self.active, done)):
                if d:
                    r.result, r.steps = self.backend.close(h)
                    r.finished = self.clock() - t0
                    self.used -= need
                    self.active.remove((r, h, need))
        return requests

    @staticmethod
    def stats(requests: List[Request], wall: float):
        ok = [r for r in requests if r.finished is not None and r.error is None]
        lat = np.array([r.finished - r.arrival for r in ok]) if ok else np.zeros(0)
        cells = sum(r.nx * r.ny * r.steps for r in ok)
        span = max((r.finished for r in ok), default=0.0)
        return {
            "served": len(ok), "rejected": sum(1 for r in requests if r.error),
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "cell_updates": int(cells),
            "served_cell_updates_per_s": cells / span if span > 0 else 0.0,
            "wall_s": wall,
        }
