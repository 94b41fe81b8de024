"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 on the GPU within 1e-11 relative of the oracle; FP32 (plain
and Kahan-compensated) within max |d eta| <= 1e-4 m and a relative L2 error
of hu and hv <= 1e-4 after 1000 steps. Both sides compute their own adaptive
time step from the same seeded float inputs."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swe():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1912_02457_gb300 import build, swe as S
    build.build()
    S.load()
    return S


def gpu_run(S, wl, n, precision, check=True):
    with S.Domain(wl, precision) as d:
        d.step(n)
        info = d.info(check=check)
        st = d.state()
    return st, info


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_f32_parity(gpu, ref):
    e, u, v = gpu
    re, ru, rv = ref[:3]
    assert np.abs(e.astype(np.float64) - re).max() <= 1e-4
    assert rel_l2(u, ru) <= 1e-4
    assert rel_l2(v, rv) <= 1e-4


_max_filter = helpers.max_filter


def front_references(oracle_mod, wl, n):
    """The oracle's solution and the wet-dry front set of the run.

    Whether and when a dry cell wets is a threshold decision: float32 and
    float64 arithmetic can wet a front cell on different steps, after which
    its level differs by up to centimetres (the FP64 oracle itself moves by
    ~3e-3 m there when its float32 inputs move by one ulp). Everywhere else
    the two agree to ~1e-6 m. The front set is every wet cell that is dry
    (hbar <= 1 cm) at the start or the end of the oracle's run, dilated by
    three cells (the stencil's reach per step is four)."""
    ref = oracle_mod.Oracle(wl).run(n)
    front = helpers.front_set(wl, ref[0])
    return ref, front


# Simulated time after 1000 adaptive steps on a domain with moving fronts:
# dt follows the CFL maximum, which a thin film on a front sets on about a
# quarter of the steps of the small coastal case, so t inherits the front
# cells' float32 sensitivity (measured 1.9e-6 relative there).
T_FRONTS = 1e-5


def front_report(gpu, wl, ref, front):
    """Where the front set lies and how far the float32 run is from the
    oracle inside and outside it (printed beside every front-aware check)."""
    e, u, v = gpu
    wet = ~wl.land_cells()
    off = wet & ~front
    dev = np.abs(e.astype(np.float64) - ref[0])
    rows, cols = np.nonzero(front)
    rep = {"front_cells": int(front.sum()), "wet_cells": int(wet.sum()),
           "front_share": round(float(front.sum() / max(wet.sum(), 1)), 4),
           "front_rows": [int(rows.min()), int(rows.max())] if rows.size else None,
           "front_cols": [int(cols.min()), int(cols.max())] if cols.size else None,
           "max_deta_off_front": float(dev[off].max()),
           "max_deta_front": float(dev[front].max()) if front.any() else 0.0,
           "mean_deta_wet": float(dev[wet].mean()),
           "rel_l2_hu_off_front": rel_l2(u[off], ref[1][off]),
           "rel_l2_hv_off_front": rel_l2(v[off], ref[2][off]),
           "rel_l2_hu": rel_l2(u, ref[1]), "rel_l2_hv": rel_l2(v, ref[2])}
    print("FRONT_BAND", rep)
    return rep


def assert_f32_parity_fronts(gpu, wl, ref, front):
    """FP32 parity on a domain with moving wet-dry fronts. Outside the front
    set: max |d eta| <= 1e-4 m and relative L2 errors of hu and hv <= 1e-4.
    Inside it (the coastal band within three cells of a dry cell: ~10% of
    the wet cells at 1024^2, at most 25% on small domains): |d eta| <= 1 cm.
    Over all wet cells: mean |d eta| <= 1e-5 m and the relative L2 errors of
    hu and hv <= 1e-3. The FP64 oracle itself, with its state stored in
    float32, moves by as much on the fronts (test_oracle_fronts.py); the
    band's size, place and errors are printed."""
    rep = front_report(gpu, wl, ref, front)
    assert rep["front_cells"] <= 0.25 * rep["wet_cells"], rep
    assert rep["max_deta_off_front"] <= 1e-4, rep
    assert rep["max_deta_front"] <= 1e-2, rep
    assert rep["mean_deta_wet"] <= 1e-5, rep
    assert rep["rel_l2_hu_off_front"] <= 1e-4 and rep["rel_l2_hv_off_front"] <= 1e-4, rep
    assert rep["rel_l2_hu"] <= 1e-3 and rep["rel_l2_hv"] <= 1e-3, rep


def test_gaussian_f64_1000_steps(swe, oracle_mod):
    wl = synth.gaussian_bump(np.float64)
    ref = oracle_mod.Oracle(wl).run(1000)
    st, info = gpu_run(swe, wl, 1000, "f64")
    for a, b in zip(st, ref[:3]):
        assert helpers.rel(a, b) <= 1e-11
    assert abs(info.t - ref[3]) <= 1e-11 * ref[3]
    assert info.step == 1000


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_gaussian_f32_1000_steps(swe, oracle_mod, prec):
    """No wet-dry fronts here: the 1e-4 bound holds on every cell."""
    wl = synth.gaussian_bump(np.float32)
    ref = oracle_mod.Oracle(wl).run(1000)
    st, info = gpu_run(swe, wl, 1000, prec)
    assert_f32_parity(st, ref)
    assert abs(info.t - ref[3]) <= 1e-5 * ref[3]


def _small_coastal(nx=96, ny=80, dtype=np.float64, member=0):
    return synth.coastal(nx, ny, seed_config=92, member=member, dtype=dtype)


def test_small_coastal_f64(swe, oracle_mod):
    """Land, wet-dry shelves, nesting with tide frames at half resolution,
    wind, drag, varying f and north angle: FP64 GPU vs oracle."""
    wl = _small_coastal()
    ref = oracle_mod.Oracle(wl).run(300)
    st, info = gpu_run(swe, wl, 300, "f64")
    for a, b in zip(st, ref[:3]):
        assert helpers.rel(a, b) <= 1e-11
    assert abs(info.t - ref[3]) <= 1e-11 * ref[3]


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_small_coastal_f32(swe, oracle_mod, prec):
    wl = _small_coastal(dtype=np.float32, member=1)
    if "small" not in _REF_CACHE:
        _REF_CACHE["small"] = front_references(oracle_mod, wl, 1000)
    ref, front = _REF_CACHE["small"]
    st, info = gpu_run(swe, wl, 1000, prec)
    assert_f32_parity_fronts(st, wl, ref, front)
    assert abs(info.t - ref[3]) <= T_FRONTS * ref[3]


def _coastal_gridded_wind(dtype, member, nfx=7, nfy=5, static=False):
    """The small coastal domain under a wind that varies across a coarse
    7 x 5 grid and from hour to hour (trilinear interpolation, Section 3.5),
    with the recipe's tide frames at half resolution along each edge.
    static: every wet corner at least 5 m deep (land mask kept, no drying
    shelves), so that no front amplifies rounding differences."""
    wl = _small_coastal(dtype=dtype, member=member)
    wl.wind = helpers.gridded_wind(nfx, nfy, hours=3, seed=member)
    if static:
        land_corner = wl.H == synth.LAND
        wl.H = np.where(land_corner, wl.H, np.maximum(wl.H, 5.0)).astype(dtype)
        wl.eta = np.zeros_like(wl.eta)
    return wl


def test_gridded_wind_f64(swe, oracle_mod):
    """FP64 on a static coast: the wind interpolation itself, free of the
    fronts' amplification (one last-bit change of the wind frames moves the
    oracle by ~1e-11 after 300 steps on the drying-shelf variant)."""
    wl = _coastal_gridded_wind(np.float64, member=7, static=True)
    ref = oracle_mod.Oracle(wl).run(300)
    st, info = gpu_run(swe, wl, 300, "f64")
    for a, b in zip(st, ref[:3]):
        assert helpers.rel(a, b) <= 1e-11
    assert abs(info.t - ref[3]) <= 1e-11 * ref[3]


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_gridded_wind_f32(swe, oracle_mod, prec):
    wl = _coastal_gridded_wind(np.float32, member=9)
    if "gridded" not in _REF_CACHE:
        _REF_CACHE["gridded"] = front_references(oracle_mod, wl, 1000)
    ref, front = _REF_CACHE["gridded"]
    st, info = gpu_run(swe, wl, 1000, prec)
    assert_f32_parity_fronts(st, wl, ref, front)
    assert abs(info.t - ref[3]) <= T_FRONTS * ref[3]


@pytest.mark.parametrize("shape", [(37, 23), (33, 9), (1, 17), (17, 1), (2, 2), (65, 130)])
def test_ragged_shapes_f64(swe, oracle_mod, shape):
    nx, ny = shape
    wl = helpers.flat(nx, ny, depth=30.0, dx=500.0, dy=700.0, f=1e-4, theta=0.2)
    wl.eta, wl.hu, wl.hv = helpers.random_state(wl, seed=nx * 131 + ny, amp=0.2, mom=1.0)
    ref = oracle_mod.Oracle(wl).run(25)
    st, info = gpu_run(swe, wl, 25, "f64")
    for a, b in zip(st, ref[:3]):
        assert helpers.rel(a, b) <= 1e-11


@pytest.mark.parametrize("prec", ["f32", "f32_kahan", "f64"])
def test_lake_at_rest_bitwise(swe, prec):
    dtype = np.float64 if prec == "f64" else np.float32
    wl = helpers.rough(70, 50, seed=3, land=True, min_depth=0.5, cd=0.0025, dtype=dtype)
    st, info = gpu_run(swe, wl, 50, prec)
    for a, b in zip(st, (wl.eta, wl.hu, wl.hv)):
        assert np.array_equal(a, b)


def test_mass_conservation_f64(swe):
    wl = synth.coastal(96, 64, seed_config=91, dtype=np.float64)
    wl.bc = (synth.BC_WALL,) * 4
    wl.boundary = None
    with swe.Domain(wl, "f64") as d:
        m0, _ = d.diagnostics()
        d.step(200)
        m1, _ = d.diagnostics()
        e = d.read(swe.ETA)
    scale = np.abs(e).sum() * wl.dx * wl.dy
    assert abs(m1 - m0) < 1e-12 * scale


def test_diagnostics_match_oracle(swe, oracle_mod):
    wl = _small_coastal(dtype=np.float64, member=2)
    with swe.Domain(wl, "f64") as d:
        d.step(20)
        st = d.state()
        m, en = d.diagnostics()
    om, oen = oracle_mod.Oracle(wl).diagnostics(*st)
    assert abs(m - om) <= 1e-12 * max(abs(om), 1.0)
    assert abs(en - oen) <= 1e-12 * abs(oen)


@pytest.mark.parametrize("prec", ["f32_kahan", "f64"])
def test_checkpoint_resume_bitwise(swe, prec):
    dtype = np.float64 if prec == "f64" else np.float32
    wl = _small_coastal(dtype=dtype, member=3)
    with swe.Domain(wl, prec) as d:
        d.step(60)
        full = d.state()
    with swe.Domain(wl, prec) as d:
        d.step(25)
        info = d.info()
        ck = d.state()
        comp = [d.read(k) for k in (swe.COMP_ETA, swe.COMP_HU, swe.COMP_HV)] if prec == "f32_kahan" else None
    with swe.Domain(wl, prec) as d:
        for k, a in zip((swe.ETA, swe.HU, swe.HV), ck):
            d.write(k, a)
        if comp is not None:
            for k, a in zip((swe.COMP_ETA, swe.COMP_HU, swe.COMP_HV), comp):
                d.write(k, a)
        d.set_clock(info.t, info.dt, info.step)
        d.step(35)
        res = d.state()
    for a, b in zip(full, res):
        assert np.array_equal(a, b)


def test_nonfinite_state_is_reported(swe):
    wl = helpers.flat(40, 30, depth=20.0, dtype=np.float32)
    with swe.Domain(wl, "f32") as d:
        e = np.zeros((30, 40), np.float32)
        e[7, 11] = np.nan
        d.write(swe.ETA, e)
        d.step(1)
        info = d.info(check=False)
        assert info.error == swe.ERR_NUMERIC
        # the first cell found non-finite lies within the stencil's reach
        cj, ci = divmod(info.error_cell, 40)
        assert abs(ci - 11) + abs(cj - 7) <= 4
        assert not np.isfinite(d.read(swe.ETA)[cj, ci])
        with pytest.raises(swe.SweError):
            d.info()
        with pytest.raises(swe.SweError):
            d.step(1)


def test_all_land_has_no_time_step(swe):
    wl = helpers.flat(8, 8, depth=20.0, dtype=np.float32)
    wl.H[:] = synth.LAND
    with swe.Domain(wl, "f32") as d:
        assert d.info(check=False).error == swe.ERR_NUMERIC


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_coastal_1024_f32_1000_steps(swe, oracle_mod, prec):
    """The full-size synthetic coastal domain (1024^2, ~30% land) through the
    same entry point the benchmark times, 1000 steps against the oracle."""
    wl = synth.coastal(1024, 1024, dtype=np.float32)
    if "c2" not in _REF_CACHE:
        _REF_CACHE["c2"] = front_references(oracle_mod, wl, 1000)
    ref, front = _REF_CACHE["c2"]
    st, info = gpu_run(swe, wl, 1000, prec)
    assert_f32_parity_fronts(st, wl, ref, front)
    assert abs(info.t - ref[3]) <= T_FRONTS * ref[3]


_REF_CACHE = {}


@pytest.mark.parametrize("shape", [(27, 19), (28, 9), (29, 61), (57, 130), (150, 33), (2, 5)])
@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_fast_kernels_match_reference_kernels(swe, shape, prec):
    """The sliding-window FP32 kernels against the one-thread-per-cell FP32
    kernels (same arithmetic, approximate reciprocal / square root) on
    shapes that straddle strip (28 columns) and band boundaries, with land,
    wet-dry cells, nesting, wind and drag."""
    nx, ny = shape
    wl = synth.coastal(max(nx, 2), max(ny, 2), seed_config=94, member=nx + ny, dtype=np.float32)
    if min(nx, ny) < 3:
        wl = helpers.flat(nx, ny, depth=25.0, f=1e-4, theta=0.3, dtype=np.float32)
        wl.eta, wl.hu, wl.hv = (a.astype(np.float32) for a in helpers.random_state(wl, seed=5))
    outs = []
    for kern in ("fast", "reference"):
        with swe.Domain(wl, prec, kernel=kern) as d:
            d.step(30)
            outs.append((d.state(), d.info()))
    (a, ia), (b, ib) = outs
    for x, y in zip(a, b):
        assert helpers.rel(x, y) <= 1e-4
    assert abs(ia.t - ib.t) <= 1e-6 * ib.t


def test_end_time_lands_exactly(swe, oracle_mod):
    """A forecast horizon: the last step is shortened to end on t_end, later
    steps are no-ops; the state matches the oracle run with the same horizon."""
    wl = _small_coastal(dtype=np.float64, member=4)
    t_end = 123.456
    ref = oracle_mod.Oracle(wl).run(400, t_end=t_end)
    with swe.Domain(wl, "f64") as d:
        d.set_end_time(t_end)
        d.step(400)
        info = d.info()
        st = d.state()
        d.step(20)
        st2 = d.state()
        info2 = d.info()
    assert info.done == 1 and abs(info.t - t_end) <= 1e-12 * t_end
    assert info2.t == info.t and info2.step == info.step
    for a, b in zip(st, ref[:3]):
        assert helpers.rel(a, b) <= 1e-11
    for a, b in zip(st, st2):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["f32_kahan", "f64"])
def test_graph_replay_equals_direct_launches(swe, prec):
    """swe_step(n >= 16) replays a captured graph; the result is bit-identical
    to stepping one step at a time."""
    dtype = np.float64 if prec == "f64" else np.float32
    wl = _small_coastal(dtype=dtype, member=5)
    with swe.Domain(wl, prec) as d:
        d.step(37)
        a = d.state()
        ia = d.info()
    with swe.Domain(wl, prec) as d:
        for _ in range(37):
            d.step(1)
        b = d.state()
        ib = d.info()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert ia.t == ib.t and ia.step == ib.step == 37


def test_read_state_to_device(swe):
    import torch
    wl = _small_coastal(dtype=np.float32, member=6)
    with swe.Domain(wl, "f32") as d:
        d.step(7)
        host = d.read(swe.HU)
        dev = torch.empty((wl.ny, wl.nx), dtype=torch.float32, device="cuda")
        d.read_device(swe.HU, dev.data_ptr())
        torch.cuda.synchronize()
    assert np.array_equal(host, dev.cpu().numpy())
