"""Periodic boundaries (Section 3.3) and the beta-plane Rossby workload
(Section 3.7) on the GPU, through the C ABI, against the FP64 oracle.

Tolerances as for the other parity tests: FP64 within 1e-11 relative of the
oracle; FP32 (plain and Kahan) max |d eta| <= 1e-4 m and relative L2 of hu,
hv <= 1e-4 (these domains have no wet-dry fronts)."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers
from tests.test_gpu_parity import assert_f32_parity, gpu_run, rel_l2, swe  # noqa: F401

pytestmark = pytest.mark.gpu


def _rough_state(nx, ny, seed, land, periodic):
    wl = helpers.periodic_rough(nx, ny, seed=seed, land=land, periodic=periodic)
    wl.eta, wl.hu, wl.hv = helpers.random_state(wl, seed=seed + 1, amp=0.2, mom=0.4)
    return wl


CASES = [((40, 28), (True, True), True), ((33, 17), (True, False), False),
         ((19, 35), (False, True), True), ((1, 9), (True, True), False),
         ((7, 1), (True, True), False), ((65, 3), (True, False), False)]


@pytest.mark.parametrize("shape,periodic,land", CASES)
def test_periodic_f64_matches_oracle(swe, oracle_mod, shape, periodic, land):
    wl = _rough_state(*shape, 3, land, periodic)
    ref = oracle_mod.Oracle(wl).run(200)
    (e, u, v), info = gpu_run(swe, wl, 200, "f64")
    for a, b in zip((e, u, v), ref[:3]):
        assert helpers.rel(a, b) <= 1e-11
    assert abs(info.t - ref[3]) <= 1e-9 * ref[3]


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
@pytest.mark.parametrize("shape,periodic,land", CASES[:3])
def test_periodic_f32_matches_oracle(swe, oracle_mod, shape, periodic, land, prec):
    wl = _rough_state(*shape, 5, land, periodic).astype(np.float32)
    ref = oracle_mod.Oracle(wl).run(1000)
    gpu, _ = gpu_run(swe, wl, 1000, prec)
    assert_f32_parity(gpu, ref)


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_periodic_lake_at_rest_is_bitwise(swe, prec):
    wl = helpers.periodic_rough(48, 40, seed=2, land=True).astype(np.float32)
    (e, u, v), _ = gpu_run(swe, wl, 300, prec)
    assert np.all(e == 0) and np.all(u == 0) and np.all(v == 0)


def test_periodic_mass_is_conserved_f64(swe):
    wl = _rough_state(64, 48, 7, True, (True, True))
    (e, _, _), _ = gpu_run(swe, wl, 500, "f64")
    assert abs(e.sum() - wl.eta.sum()) <= 1e-12 * np.abs(wl.eta).sum()


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_fast_and_reference_kernels_agree_periodic(swe, prec):
    wl = _rough_state(70, 45, 9, True, (True, True)).astype(np.float32)
    with swe.Domain(wl, prec, kernel="fast") as d:
        d.step(300)
        a = d.state()
    with swe.Domain(wl, prec, kernel="reference") as d:
        d.step(300)
        b = d.state()
    for x, y in zip(a, b):
        assert helpers.rel(x, y) <= 1e-4


def test_cyclic_shift_on_the_gpu_is_bitwise(swe):
    """The fast kernel's tiling differs between a domain and its cyclic
    shift, and every cell still runs the same arithmetic."""
    wl = _rough_state(72, 40, 11, True, (True, True)).astype(np.float32)
    dj, di = 5, 9
    sh = wl.copy()
    for k in ("eta", "hu", "hv", "f", "theta"):
        setattr(sh, k, np.roll(np.roll(getattr(wl, k), dj, axis=0), di, axis=1).copy())
    core = np.roll(np.roll(wl.H[:-1, :-1], dj, axis=0), di, axis=1)
    H = np.concatenate([core, core[:, :1]], axis=1)
    sh.H = np.concatenate([H, H[:1, :]], axis=0)
    a, _ = gpu_run(swe, wl, 200, "f32_kahan")
    b, _ = gpu_run(swe, sh, 200, "f32_kahan")
    for x, y in zip(a, b):
        np.testing.assert_array_equal(np.roll(np.roll(x, dj, axis=0), di, axis=1), y)


def test_unpaired_or_inconsistent_periodic_domains_are_rejected(swe):
    wl = helpers.periodic_rough(16, 12, seed=1).astype(np.float32)
    bad = wl.copy()
    bad.bc = (synth.BC_PERIODIC, synth.BC_WALL, synth.BC_PERIODIC, synth.BC_PERIODIC)
    with pytest.raises(swe.SweError):
        swe.Domain(bad, "f32")
    bad = wl.copy()
    bad.H = bad.H.copy()
    bad.H[3, -1] += 1.0                    # last corner column no longer repeats the first
    with pytest.raises(swe.SweError):
        swe.Domain(bad, "f32")


@pytest.mark.parametrize("theta", [0.0, np.pi / 2])
def test_rossby_350_matches_oracle(swe, oracle_mod, theta):
    """The beta-plane workload at its full size, 500 steps (~1 day), FP32 +
    Kahan in the configuration bench.py times."""
    wl = synth.rossby(n=350, theta=theta).astype(np.float32)
    ref = oracle_mod.Oracle(wl).run(500)
    gpu, info = gpu_run(swe, wl, 500, "f32_kahan")
    assert_f32_parity(gpu, ref)
    assert abs(info.t - ref[3]) <= 1e-6 * ref[3]
