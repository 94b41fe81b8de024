"""Admission, retirement and fault handling of the continuous-batching
server, against a fake backend (CPU only; the faults are made on the host:
an allocation that fails, a malformed request, a cancellation, a request
larger than the budget)."""
import itertools

import pytest

from paper_1912_02457_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """Each domain needs `steps_needed` steps; one step costs `dt_wall`."""

    def __init__(self, clock, dt_wall=1e-3):
        self.clock = clock
        self.dt_wall = dt_wall
        self.live = {}
        self.ids = itertools.count()
        self.max_live = 0

    def create(self, wl, precision, horizon):
        if wl == "boom":
            raise RuntimeError("allocation failed")
        h = next(self.ids)
        self.live[h] = [0, int(horizon), False]
        self.max_live = max(self.max_live, len(self.live))
        return h

    def join(self, h):
        self.live[h][2] = True

    def step(self, n):
        self.clock.t += n * self.dt_wall
        for v in self.live.values():
            if v[2]:
                v[0] = min(v[0] + n, v[1])

    def poll(self, handles):
        return [self.live[h][0] >= self.live[h][1] for h in handles]

    def leave(self, h):
        self.live[h][2] = False

    def result(self, h, download=True):
        steps = self.live.pop(h)[0]
        return ("state", h) if download else None, steps

    def shutdown(self):
        pass


def _req(rid, arrival, n, steps, wl="ok"):
    return serve.Request(rid=rid, arrival=arrival, make_workload=lambda: wl, horizon=steps,
                         nx=n, ny=n)


def test_tiny_budget_is_respected_and_all_are_served():
    clock = FakeClock()
    be = FakeBackend(clock)
    one = serve.domain_bytes(256, 256)
    srv = serve.ForecastServer(be, budget_bytes=2.5 * one, round_steps=10, clock=clock)
    reqs = [_req(k, 0.001 * k, 256, 50 + 10 * k) for k in range(7)]
    srv.run(reqs)
    assert all(r.error is None and r.result is not None for r in reqs)
    assert srv.peak_used <= 2.5 * one and be.max_live == 2
    # admitted in arrival order
    adm = [r.admitted for r in reqs]
    assert adm == sorted(adm)
    st = serve.ForecastServer.stats(reqs, wall=clock.t)
    assert st["served"] == 7 and st["p99_latency_s"] >= st["p50_latency_s"] > 0
    # later arrivals were admitted while earlier ones were on the device
    assert srv.overlapped > 0


def test_faults_do_not_stop_the_server():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = serve.ForecastServer(be, budget_bytes=4 * serve.domain_bytes(512, 512), round_steps=5,
                               clock=clock)
    big = _req(1, 0.0, 8192, 10)                  # larger than the whole budget
    bad = _req(2, 0.0, 64, 10, wl="boom")         # backend refuses it
    cancel_early = _req(3, 0.0, 64, 10)
    cancel_early.cancelled = True
    good = [_req(10 + k, 0.0, 128, 20) for k in range(3)]
    late_cancel = _req(4, 0.0, 128, 10_000)
    reqs = [big, bad, cancel_early, late_cancel] + good

    orig_step = be.step

    def step_and_cancel(n):
        orig_step(n)
        if clock.t > 0.02:
            late_cancel.cancelled = True

    be.step = step_and_cancel
    srv.run(reqs)
    assert big.error and "budget" in big.error
    assert bad.error and "rejected" in bad.error
    assert cancel_early.error == "cancelled before admission"
    assert late_cancel.error == "cancelled" and late_cancel.result is None
    assert all(r.error is None and r.steps == 20 for r in good)
    assert srv.used == 0 and not be.live


def test_domain_bytes_counts_planes():
    b32 = serve.domain_bytes(1024, 1024, "f32")
    bk = serve.domain_bytes(1024, 1024, "f32_kahan")
    assert bk - b32 == 3 * 4 * 1024 * 1024
    assert 50e6 < bk < 70e6
