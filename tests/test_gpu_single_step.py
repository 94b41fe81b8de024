"""One and three steps on tiny grids (odd sizes, land across strip and tile
edges, every boundary kind) against the oracle: the kernel-level check.

FP64 (reference kernels): 1e-12 relative. FP32 (the fast kernels, plain and
Kahan): the deviation of the new state from the oracle's, in units of the
FP32 spacing of the largest |state| component, stays within a bound set from
the arithmetic: the state itself is stored to within half an ulp, and the
increment dt M(Q) is a sum of O(10^2) rounded terms of the same scale as the
state change, each off by at most a few ulp of its own size (measured on a
GB300: at most 4.3 ulp over every case below; the bound is 16 ulp)."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers
from tests.test_gpu_parity import swe  # noqa: F401

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8), (17, 13), (29, 3), (57, 31), (3, 40), (31, 31)]
UPP = 16                 # ulps of the largest state component


def _case(shape, kind, seed):
    nx, ny = shape
    if kind == "periodic":
        wl = helpers.periodic_rough(nx, ny, seed=seed, land=min(nx, ny) >= 8)
    else:
        wl = helpers.rough(nx, ny, seed=seed, land=min(nx, ny) >= 8, min_depth=5.0, cd=0.002)
        if kind == "nested":
            wl.bc = (synth.BC_NESTED, synth.BC_NESTED, synth.BC_NESTED, synth.BC_WALL)
            wl.boundary = synth.still_boundary(nx, ny, eta=0.05)
            wl.wind = synth.uniform_wind(8.0, -3.0)
    wl.eta, wl.hu, wl.hv = helpers.random_state(wl, seed=seed + 7, amp=0.2, mom=0.5)
    return wl


def _deviation_ulps(gpu, ref):
    scale = max(float(np.abs(np.asarray(r)).max()) for r in ref[:3])
    ulp = float(np.spacing(np.float32(scale)))
    return max(float(np.abs(np.asarray(g, np.float64) - r).max()) for g, r in zip(gpu, ref[:3])) / ulp


@pytest.mark.parametrize("kind", ["walls", "nested", "periodic"])
@pytest.mark.parametrize("shape", SHAPES)
def test_one_and_three_steps_f64(swe, oracle_mod, shape, kind):
    wl = _case(shape, kind, shape[0] * 7 + shape[1])
    for n in (1, 3):
        ref = oracle_mod.Oracle(wl).run(n)
        with swe.Domain(wl, "f64") as d:
            d.step(n)
            st = d.state()
        for a, b in zip(st, ref[:3]):
            assert helpers.rel(a, b) <= 1e-12


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
@pytest.mark.parametrize("kind", ["walls", "nested", "periodic"])
@pytest.mark.parametrize("shape", SHAPES)
def test_one_and_three_steps_f32(swe, oracle_mod, shape, kind, prec):
    wl = _case(shape, kind, shape[0] * 7 + shape[1]).astype(np.float32)
    for n in (1, 3):
        ref = oracle_mod.Oracle(wl).run(n)
        with swe.Domain(wl, prec) as d:
            d.step(n)
            st = d.state()
        dev = _deviation_ulps(st, ref)
        print(f"ULPS {shape} {kind} {prec} n={n}: {dev:.2f}")
        assert dev <= UPP, dev
