"""Domain decomposition on one GPU (swe_split_sync / swe_split_step): the
windows of a partition, exchanging their two-cell halos after every RK
stage and sharing one clock evaluation per step, step the whole domain bit
for bit (state, t, dt); what is not a decomposition is rejected."""
import numpy as np
import pytest

from helpers import gridded_wind
from paper_1912_02457_gb300 import synth

pytestmark = pytest.mark.gpu

STEPS = 60


@pytest.fixture(scope="module")
def swe():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1912_02457_gb300 import build, swe as S
    build.build()
    S.load()
    return S


def _workload():
    """Coastal 256 x 192: nested S, N, W edges with tide frames, east wall,
    land and drying shelves, varying f, drag, gridded wind varying in x, y
    and time."""
    wl = synth.coastal(256, 192, dtype=np.float32)
    wl.wind = gridded_wind(7, 5)
    return wl


_WHOLE = {}


def _whole(swe, prec, t_end=0.0):
    key = (prec, t_end)
    if key not in _WHOLE:
        with swe.Domain(_workload(), prec) as d:
            if t_end:
                d.set_end_time(t_end)
            d.step(STEPS)
            i = d.info()
            _WHOLE[key] = (d.state(), (i.t, i.dt, i.step, i.done))
    return _WHOLE[key]


@pytest.mark.parametrize("prec", ["f32_kahan", "f32"])
@pytest.mark.parametrize("px,py", [(2, 1), (1, 2), (2, 2), (3, 2), (4, 4)])
def test_split_equals_whole_bit_for_bit(swe, prec, px, py):
    from paper_1912_02457_gb300.split import SplitDomain
    (ref, clock) = _whole(swe, prec)
    with SplitDomain(_workload(), px, py, prec) as s:
        s.step(STEPS)
        i = s.info()
        out = s.state()
        # every sub-domain's clock is the same
        for d in s.doms:
            j = d.info()
            assert (j.t, j.dt, j.step) == (i.t, i.dt, i.step)
    assert (i.t, i.dt, i.step, i.done) == clock
    for a, b in zip(out, ref):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_split_reaches_the_horizon_like_the_whole_domain(swe):
    from paper_1912_02457_gb300.split import SplitDomain
    t_end = 40.0                     # the horizon falls inside the 60 steps
    ref, clock = _whole(swe, "f32_kahan", t_end)
    assert clock[3] == 1
    with SplitDomain(_workload(), 2, 2, "f32_kahan") as s:
        for d in s.doms:
            d.set_end_time(t_end)
        s.step(STEPS)
        i = s.info()
        out = s.state()
    assert (i.t, i.dt, i.step, i.done) == clock and i.t == t_end
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_split_matches_the_oracle_decomposition(swe, oracle_mod, prec):
    """The GPU's windows against the FP64 oracle stepped as the same 3 x 2
    windows (oracle/decomp.py), 300 steps on a coast whose wet corners are
    at least 5 m deep (no drying fronts to amplify rounding), gridded wind
    and tide frames sampled at whole-domain positions: the FP32 parity
    bounds of a whole domain (max |d eta| <= 1e-4 m, relative L2 of the
    momenta <= 1e-4)."""
    from oracle import decomp
    from paper_1912_02457_gb300.split import SplitDomain
    wl = synth.coastal(120, 84, seed_config=31, dtype=np.float32)
    wl.wind = gridded_wind(7, 5, hours=3, seed=3)
    land_corner = wl.H == synth.LAND
    wl.H = np.where(land_corner, wl.H, np.maximum(wl.H, 5.0)).astype(np.float32)
    wl.eta = np.zeros_like(wl.eta)
    (re, ru, rv), (t, _) = decomp.run_split(wl.astype(np.float64), 3, 2, 300)
    with SplitDomain(wl, 3, 2, prec) as s:
        s.step(300)
        e, u, v = s.state()
        info = s.info()

    def rel_l2(a, b):
        return float(np.linalg.norm(a.astype(np.float64) - b) / max(np.linalg.norm(b), 1e-300))
    deta = float(np.abs(e.astype(np.float64) - re).max())
    print("SPLIT_VS_ORACLE", prec, deta, rel_l2(u, ru), rel_l2(v, rv), info.t, t)
    assert deta <= 1e-4 and rel_l2(u, ru) <= 1e-4 and rel_l2(v, rv) <= 1e-4
    assert abs(info.t - t) <= 1e-6 * t


def test_what_is_not_a_decomposition_is_rejected(swe):
    import ctypes as C
    from paper_1912_02457_gb300.split import SplitDomain
    wl = _workload()
    L = swe.load()
    with SplitDomain(wl, 2, 2, "f32") as s:
        hs = [d.h.value for d in s.doms]

        def step(handles):
            arr = (C.c_void_p * len(handles))(*handles)
            return L.swe_split_step(arr, len(handles), 1)
        assert step(hs[:3]) == swe.ERR_INVALID_ARG                 # a part missing
        assert step(hs[:3] + [hs[0]]) == swe.ERR_INVALID_ARG       # a part twice
        assert step([]) == swe.ERR_INVALID_ARG
        # a window steps only with its sub-domains, and is not batchable
        assert L.swe_step(s.doms[0].h, 1) == swe.ERR_UNSUPPORTED
        with swe.Batch() as b:
            assert L.swe_batch_add(b.h, s.doms[0].h) == swe.ERR_UNSUPPORTED
        # a whole domain is not a window
        with swe.Domain(wl, "f32") as whole:
            assert step([whole.h.value]) == swe.ERR_INVALID_ARG
    # windows with a one-cell halo tile the domain but miss the stencil
    thin = synth.partition(wl.nx, wl.ny, 2, 1, halo=1)
    ds = [swe.Domain(synth.window(wl, p), "f32", window=(p, wl.nx, wl.ny)) for p in thin]
    try:
        arr = (C.c_void_p * 2)(*[d.h.value for d in ds])
        assert L.swe_split_sync(arr, 2) == swe.ERR_INVALID_ARG
        assert L.swe_split_step(arr, 2, 1) == swe.ERR_INVALID_ARG
    finally:
        for d in ds:
            d.close()
    part = synth.partition(wl.nx, wl.ny, 2, 1)[0]
    with pytest.raises(swe.SweError) as e:
        swe.Domain(synth.window(wl.astype(np.float64), part), "f64", window=(part, wl.nx, wl.ny))
    assert e.value.status == swe.ERR_UNSUPPORTED
    bad = dict(part, own=(0, 300, 0, 192))                        # own cells outside the window
    with pytest.raises(swe.SweError) as e:
        swe.Domain(synth.window(wl, part), "f32", window=(bad, wl.nx, wl.ny))
    assert e.value.status == swe.ERR_INVALID_ARG
