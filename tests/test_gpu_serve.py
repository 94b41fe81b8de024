"""The continuous-batching forecast server on the GPU (serve.ForecastServer
with serve.GpuBackend): requests of uneven sizes and horizons arrive while
others are on the device, join the running batch at round boundaries, and
every served forecast is the same as the domain stepped alone, bit for bit,
and matches the FP64 oracle within the front-aware float32 bounds."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers
from tests.test_gpu_parity import T_FRONTS, assert_f32_parity_fronts, swe  # noqa: F401

pytestmark = pytest.mark.gpu

# (nx, ny, simulated horizon s, wall-clock arrival s, static coast)
TRACE = [(64, 64, 900.0, 0.0, True), (96, 64, 2400.0, 0.0, False), (128, 96, 3000.0, 0.002, False),
         (64, 96, 900.0, 0.004, False), (160, 128, 2000.0, 0.006, False),
         (200, 150, 1500.0, 0.010, False), (48, 40, 600.0, 0.012, True)]


def _workload(k):
    """The coastal recipe; a static coast keeps its land mask but has every
    wet corner at least 5 m deep. The members checked against the oracle
    with drying shelves would meet thin-film events within their horizon
    (time steps down to 0.025 s), after which float32 and float64 runs part
    ways (the 24 h horizon test shows it); the static coasts and member 3
    step without them."""
    nx, ny, horizon, _, static = TRACE[k]
    wl = synth.coastal(nx, ny, seed_config=96, member=k, dtype=np.float32, hours=1)
    if static:
        land_corner = wl.H == synth.LAND
        wl.H = np.where(land_corner, wl.H, np.maximum(wl.H, 5.0)).astype(np.float32)
        wl.eta = np.zeros_like(wl.eta)
    return wl


@pytest.fixture(scope="module")
def served(swe):
    import torch
    from paper_1912_02457_gb300 import serve
    wls = [_workload(k) for k in range(len(TRACE))]
    reqs = [serve.Request(rid=k, arrival=a, make_workload=(lambda w=wls[k]: w), horizon=h,
                          nx=nx, ny=ny)
            for k, (nx, ny, h, a, _) in enumerate(TRACE)]
    stream = torch.cuda.Stream()
    backend = serve.GpuBackend(stream=stream.cuda_stream)
    srv = serve.ForecastServer(backend, budget_bytes=2e9, round_steps=32)
    srv.run(reqs, time_limit=300.0)
    backend.shutdown()
    return wls, reqs, srv


def test_every_request_is_served(served):
    wls, reqs, srv = served
    assert all(r.error is None and r.result is not None for r in reqs), [r.error for r in reqs]
    assert srv.used == 0 and srv.rounds > 0
    # continuous batching: later requests were admitted while earlier ones
    # ran, and joined a batch that was already stepping
    assert srv.overlapped > 0
    first_done = min(r.finished for r in reqs)
    assert sum(r.admitted > reqs[0].admitted for r in reqs if r.admitted < first_done) >= 1
    st = srv.stats(reqs, wall=max(r.finished for r in reqs))
    print("SERVE", st)
    assert st["served"] == len(reqs) and st["p99_latency_s"] >= st["p50_latency_s"] > 0


def test_served_equals_alone_bitwise(swe, served):
    """The same domain stepped alone to its horizon gives the same bits as
    its share of the batched rounds (same per-cell arithmetic, own clock)."""
    wls, reqs, srv = served
    for wl, r in zip(wls, reqs):
        with swe.Domain(wl, "f32_kahan") as d:
            d.set_end_time(wl.t0 + r.horizon)
            d.step(10 ** 6)
            info = d.info()
            alone = d.state()
        assert info.done == 1 and info.step == r.steps
        for a, b in zip(alone, r.result):
            assert np.array_equal(a, b), r.rid


def test_served_matches_oracle(oracle_mod, served):
    """The members with a horizon of about 1000 steps against the oracle."""
    wls, reqs, srv = served
    checked = 0
    for wl, r in zip(wls, reqs):
        if r.horizon > 900.0:           # members 0, 3 and 6
            continue
        ref = oracle_mod.Oracle(wl).run(10 ** 6, t_end=wl.t0 + r.horizon)
        front = helpers.front_set(wl, ref[0])
        assert_f32_parity_fronts(r.result, wl, ref, front)
        checked += 1
    assert checked == 3
