"""Continuous-batching forecast server on top of the libswe batch API.

On-demand forecasts (the search-and-rescue / oil-spill use the paper's
introduction motivates) arrive at random times with uneven domain sizes and
horizons. The server:

* admits waiting requests in arrival order whenever their device memory fits
  the budget (each admitted domain keeps its state and forcing resident);
* advances every admitted domain together in rounds of ``round_steps``
  batched steps (one launch per RK stage, graph-replayed), each
  domain on its own clock up to its own horizon;
* overlaps the host side with the device: while a round runs, arrivals are
  admitted (their domains created and uploaded on a side stream) and the
  domains that finished in the previous round are read back; at the round's
  end finished domains leave the batch and admitted ones join it, so work
  from requests that arrive while others run shares the next launches.

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
    """libswe-backed execution: one batch on one stream, plus a side stream
    on which admitted domains are created and uploaded and finished domains
    read back while the batch's round runs. Device memory comes from
    PyTorch's caching allocator, so freeing a retired domain does not wait
    for the running round."""

    def __init__(self, stream: int = 0, side_stream: Optional[int] = None):
        from paper_1912_02457_gb300 import swe
        self.swe = swe
        swe.use_torch_allocator()
        self.batch = swe.Batch(stream)
        self.stream = stream
        if side_stream is None:
            import torch
            self._side = torch.cuda.Stream()
            side_stream = self._side.cuda_stream
        self.side = side_stream

    def create(self, wl, precision, horizon):
        d = self.swe.Domain(wl, precision, stream=self.side)
        d.set_end_time(wl.t0 + horizon)
        return d

    def join(self, h):
        self.batch.add(h)

    def step(self, n):
        self.batch.step(n)                 # enqueued; returns at once

    def poll(self, handles):
        done, t = self.batch.poll()        # waits for the round
        idx = {id(d): k for k, d in enumerate(self.batch.domains)}
        return [bool(done[idx[id(h)]]) for h in handles]

    def leave(self, h):
        self.batch.remove(h)

    def result(self, h, download=True):
        out = h.state() if download else None
        info = h.info(check=False)
        h.close()
        return out, info.step

    def shutdown(self):
        self.batch.close()
        self.swe.use_default_allocator()


class ForecastServer:
    """Continuous batching in rounds. Each round goes to the device first;
    while it runs, the host admits the requests that have arrived (their
    domains are created and uploaded on the backend's side stream) and reads
    back the domains that finished in the previous round. At the end of the
    round, finished domains leave the batch and admitted ones join it, so a
    request waits at most one round for a slot once memory allows."""

    def __init__(self, backend, budget_bytes: float = 150e9, round_steps: int = 64,
                 clock: Callable[[], float] = time.perf_counter):
        self.backend = backend
        self.budget = float(budget_bytes)
        self.round_steps = int(round_steps)
        self.clock = clock
        self.used = 0
        self.peak_used = 0
        self.active = []           # (request, handle, bytes) in the batch
        self.staged = []           # admitted and created, joining at the next boundary
        self.retired = []          # left the batch, result not yet read
        self.rounds = 0
        self.overlapped = 0        # admissions made while a round was running

    def _admit(self, waiting: List[Request], now: float, running: bool):
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
                h = self.backend.create(wl, r.precision, r.horizon)
            except Exception as exc:      # malformed request / allocation failure
                r.error = f"rejected: {exc}"
                r.finished = now
                continue
            r.admitted = now
            self.used += need
            self.peak_used = max(self.peak_used, self.used)
            self.staged.append((r, h, need))
            self.overlapped += int(running)

    def _collect(self, t0: float):
        for r, h, need in self.retired:
            r.result, r.steps = self.backend.result(h)
            r.finished = self.clock() - t0
            self.used -= need
        self.retired = []

    def run(self, requests: List[Request], time_limit: float = 3600.0):
        waiting = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock()
        while waiting or self.active or self.staged or self.retired:
            now = self.clock() - t0
            if now > time_limit:
                break
            running = bool(self.active)
            if running:                   # the round goes to the device first
                self.backend.step(self.round_steps)
                self.rounds += 1
            # while it runs: read back the previous round's finished domains
            # and admit arrivals
            self._collect(t0)
            self._admit(waiting, self.clock() - t0, running)
            if running:
                done = self.backend.poll([h for _, h, _ in self.active])
                for (r, h, need), d in list(zip(self.active, done)):
                    if d or r.cancelled:
                        self.backend.leave(h)
                        self.active.remove((r, h, need))
                        if d and not r.cancelled:
                            self.retired.append((r, h, need))
                        else:             # cancelled while running: no result
                            self.backend.result(h, download=False)
                            self.used -= need
                            r.error = "cancelled"
                            r.finished = self.clock() - t0
            for item in self.staged:
                self.backend.join(item[1])
                self.active.append(item)
            self.staged = []
            if not self.active and not self.retired and waiting:
                delay = waiting[0].arrival - (self.clock() - t0)
                if delay > 0:
                    time.sleep(min(delay, 0.05))
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
