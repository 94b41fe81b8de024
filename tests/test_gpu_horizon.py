"""The full forecast horizon of the synthetic coastal recipe: 24 simulated
hours (about 1.2e5 adaptive steps: nested M2 tide, wind, drag, moving
wet-dry fronts) on the GPU in FP32 against the FP64 oracle, at 128 x 128
cells of 800 m, a size at which the oracle finishes the horizon in about
two minutes. Both sides compute their own adaptive time step and both stop
exactly on t = 24 h.

Parity is gated at 1000 steps elsewhere. Over the full horizon the moving
wet-dry fronts of this recipe produce what Section 3.4 warns of (non-physical
waves and small time steps): thin drying films on raised shelves carry
momentum, their desingularised velocities spike, and the CFL step drops to
a few hundredths of a second at times, in the oracle as on the GPU. The
mechanism is pinned in test_oracle_positivity.py: the cell-average time
step exceeds the faces' one-sided speeds there by a factor of ten or more,
so Kurganov & Petrova's condition for non-negative depths fails. After the
first such event runs that differ by rounding take different step
sequences, so the end states differ at the level of the waves themselves
(the FP64 GPU path, within 1e-11 of the oracle per step, ends as far from
it as FP32).
The moving-front test therefore reports the deviation and checks only
that a run is sound: finite, no sticky error, the exact end time, a step
count close to the oracle's, and deviations no larger than twice those
between the oracle and the same oracle with its stored state rounded to
FP32 (the spread rounding alone produces on this recipe). The same recipe on a static coast (land mask, no drying shelves)
holds the 1000-step parity bounds over the whole 24 h."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers
from tests.test_gpu_parity import rel_l2, swe  # noqa: F401

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

T_END = 24 * 3600.0
N = 128
MAX_STEPS = 300000          # far more than the horizon takes; the clock stops at T_END

_REF = {}


def _reference(oracle_mod, wl):
    if "ref" not in _REF:
        ref = oracle_mod.Oracle(wl).run(MAX_STEPS, t_end=T_END, return_dts=True)
        steps = int((ref[5] > 0).sum())
        _REF["ref"] = (ref, steps, helpers.front_set(wl, ref[0]))
    return _REF["ref"]


def _deviation(wl, e, u, v, ref, front):
    wet = ~wl.land_cells()
    dev = np.abs(np.asarray(e, np.float64) - ref[0])
    return {"max_deta_off_front_m": float(dev[wet & ~front].max()),
            "mean_deta_wet_m": float(dev[wet].mean()),
            "rel_l2_hu": rel_l2(u, ref[1]), "rel_l2_hv": rel_l2(v, ref[2])}


def _yardstick(oracle_mod, wl):
    """How far the FP64 oracle itself ends from its own 24 h run when only
    its stored state is rounded to FP32 after every stage (its arithmetic
    stays FP64): the spread that rounding alone produces through the
    moving-front events (measured: max 2.6 m off the front band, mean
    0.076 m, relative L2 0.95 / 1.19)."""
    if "yard" not in _REF:
        ref, _, front = _reference(oracle_mod, wl)
        r32 = oracle_mod.Oracle(wl, round_state_f32=True).run(MAX_STEPS, t_end=T_END)
        _REF["yard"] = _deviation(wl, r32[0], r32[1], r32[2], ref, front)
    return _REF["yard"]


@pytest.mark.parametrize("prec", ["f32_kahan", "f32"])
def test_coastal_24h_horizon(swe, oracle_mod, prec):
    wl = synth.coastal(N, N, dtype=np.float32)
    ref, ref_steps, front = _reference(oracle_mod, wl)
    with swe.Domain(wl, prec) as d:
        d.set_end_time(T_END)
        d.step(MAX_STEPS)
        info = d.info()
        e, u, v = d.state()
    assert info.done == 1 and info.error == 0
    assert abs(info.t - T_END) <= 1e-9 * T_END and abs(ref[3] - T_END) <= 1e-9 * T_END
    report = {"precision": prec, "steps": int(info.step), "oracle_steps": ref_steps,
              "oracle_dt_min_s": float(ref[5][:ref_steps].min())}
    report.update(_deviation(wl, e, u, v, ref, front))
    yard = _yardstick(oracle_mod, wl)
    print("HORIZON", report, "ORACLE_FP32_STORAGE", yard)
    assert np.isfinite(e).all() and np.isfinite(u).all() and np.isfinite(v).all()
    # soundness, not parity (see the module docstring): the step count
    # follows the oracle's, and the run ends no farther from the oracle
    # than twice what rounding the oracle's own stored state to FP32 does
    # to it over the same 24 h (earlier realisations of this FP32 path ended
    # at 0.13-2.1 m off the front band, mean 0.009-0.074 m, L2 0.14-1.0: any
    # change of rounding picks another one)
    assert abs(info.step - ref_steps) <= 0.2 * ref_steps
    for key in ("max_deta_off_front_m", "mean_deta_wet_m", "rel_l2_hu", "rel_l2_hv"):
        assert report[key] <= 2.0 * yard[key], key


def _static_coast():
    """The same recipe with every wet corner at least 5 m deep: the land mask
    stays, the drying shelves go (the static coast Section 3.4 recommends
    for real coasts). The oracle then needs no step below 0.9 s."""
    wl = synth.coastal(N, N, dtype=np.float32)
    land_corner = wl.H == np.float32(synth.LAND)
    wl.H = np.where(land_corner, wl.H, np.maximum(wl.H, 5.0)).astype(np.float32)
    land = wl.land_cells()
    Hm = np.where(land_corner, np.nan, wl.H.astype(np.float64))
    Hbar = 0.25 * (Hm[:-1, :-1] + Hm[1:, :-1] + Hm[:-1, 1:] + Hm[1:, 1:])
    wl.eta = np.where(land, 0.0, np.maximum(0.0, -Hbar)).astype(np.float32)
    return wl


@pytest.mark.parametrize("prec", ["f32_kahan", "f32"])
def test_static_coast_24h_horizon(swe, oracle_mod, prec):
    wl = _static_coast()
    if "static" not in _REF:
        ref = oracle_mod.Oracle(wl).run(MAX_STEPS, t_end=T_END, return_dts=True)
        _REF["static"] = (ref, int((ref[5] > 0).sum()))
    ref, ref_steps = _REF["static"]
    with swe.Domain(wl, prec) as d:
        d.set_end_time(T_END)
        d.step(MAX_STEPS)
        info = d.info()
        e, u, v = d.state()
    assert info.done == 1 and info.error == 0 and abs(info.t - T_END) <= 1e-9 * T_END
    wet = ~wl.land_cells()
    dev = np.abs(e.astype(np.float64) - ref[0])
    report = {"precision": prec, "steps": int(info.step), "oracle_steps": ref_steps,
              "oracle_dt_min_s": float(ref[5][:ref_steps].min()),
              "max_deta_m": float(dev[wet].max()), "mean_deta_m": float(dev[wet].mean()),
              "rel_l2_hu": rel_l2(u, ref[1]), "rel_l2_hv": rel_l2(v, ref[2])}
    print("STATIC_HORIZON", report)
    # without moving fronts the 1000-step parity bounds hold over the whole
    # horizon (measured: max 7.8e-5 m, mean 3.9e-7 m with Kahan and 4.7e-7 m
    # without, L2 1.4e-5 / 1.4e-5, the same 89,240 steps as the oracle). The
    # margin is thin and the run is sensitive to the time step: dt as an FP32
    # quotient instead of the FP64 one (a relative change below 6e-8 per
    # step) ended at max 1.2e-4 m, mean 6.6e-7 m
    # after 24 h.
    assert ref_steps == pytest.approx(info.step, rel=1e-3)
    assert report["max_deta_m"] <= 1e-4 and report["mean_deta_m"] <= 1e-5
    assert report["rel_l2_hu"] <= 1e-4 and report["rel_l2_hv"] <= 1e-4
