"""The face-speed time step on the GPU (swe_params.cfl_faces): eq:cfl with
the faces' one-sided speeds of the state's reconstruction, Kurganov &
Petrova's condition for non-negative depths over moving wet-dry fronts. A
speed pass before each step finds the largest face speed and sets dt. The
FP32 kernels against the oracle run the same way, the depths on a drying
shelf against the cell-average step, and a resumed run bit for bit."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers
from tests.test_gpu_parity import T_FRONTS, _small_coastal, assert_f32_parity_fronts, swe  # noqa: F401

pytestmark = pytest.mark.gpu


def _faces(wl):
    wl.params.cfl_faces = 1
    return wl


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_face_step_matches_oracle(swe, oracle_mod, prec):
    wl = _faces(_small_coastal(dtype=np.float32, member=1))
    ref = oracle_mod.Oracle(wl).run(1000, return_dts=True)
    front = helpers.front_set(wl, ref[0])
    with swe.Domain(wl, prec) as d:
        assert d.launch_names() == ["speed", "stage1", "stage2"]
        d.step(1000)
        info = d.info()
        st = d.state()
    assert info.step == 1000
    assert_f32_parity_fronts(st, wl, ref, front)
    assert abs(info.t - ref[3]) <= T_FRONTS * ref[3]


def _shelf(dtype=np.float32):
    wl = synth.coastal(32, 32, seed_config=95, member=0, dtype=dtype)
    wl.bc = (synth.BC_WALL,) * 4
    wl.boundary = None
    return wl


def _min_depth_run(swe, wl, t_end, chunk):
    land = wl.land_cells()
    Hm = np.where(wl.H == np.float32(synth.LAND), np.nan, wl.H.astype(np.float64))
    Hbar = 0.25 * (Hm[:-1, :-1] + Hm[1:, :-1] + Hm[:-1, 1:] + Hm[1:, 1:])
    worst = np.inf
    with swe.Domain(wl, "f32_kahan") as d:
        d.set_end_time(t_end)
        while d.info().done == 0:
            d.step(chunk)
            e = d.read(swe.ETA).astype(np.float64)
            worst = min(worst, float(np.where(land, np.inf, e + Hbar).min()))
        steps = d.info().step
    return worst, steps


def test_face_step_keeps_depths_nonnegative(swe):
    """The drying-shelf case of the oracle pins in float32: with the
    cell-average step a depth goes below -1e-4 m within 300 s, with the
    face-speed step none goes below float32 rounding of the shelf levels."""
    cell, n_cell = _min_depth_run(swe, _shelf(), 300.0, 25)
    face, n_face = _min_depth_run(swe, _faces(_shelf()), 300.0, 500)
    assert cell < -1e-4
    assert face >= -1e-5
    assert n_face > 10 * n_cell


def test_face_step_resume_bitwise(swe):
    wl = _faces(_small_coastal(dtype=np.float32, member=3))
    with swe.Domain(wl, "f32_kahan") as d:
        d.step(60)
        full = d.state()
    with swe.Domain(wl, "f32_kahan") as d:
        d.step(25)
        info = d.info()
        ck = d.state()
        comp = [d.read(k) for k in (swe.COMP_ETA, swe.COMP_HU, swe.COMP_HV)]
    with swe.Domain(wl, "f32_kahan") as d:
        for k, a in zip((swe.ETA, swe.HU, swe.HV, swe.COMP_ETA, swe.COMP_HU, swe.COMP_HV),
                        list(ck) + comp):
            d.write(k, a)
        d.set_clock(info.t, info.dt, info.step)
        d.step(35)
        res = d.state()
    for a, b in zip(full, res):
        assert np.array_equal(a, b)


def test_face_step_domains_do_not_join_batches(swe):
    wl = _faces(_small_coastal(dtype=np.float32, member=4))
    with swe.Domain(wl, "f32_kahan") as d, swe.Batch() as b:
        with pytest.raises(swe.SweError) as ei:
            b.add(d)
        assert ei.value.status == swe.ERR_UNSUPPORTED
