"""Launches cover only the warp items (28-column strips by `rows` rows) that
hold a wet output cell: an all-land item writes nothing, so skipping it
must leave every result unchanged. Cases: a domain that is all land (one
no-op item still runs the clock), and wet pools scattered through land so
that most items are skipped, against the oracle and, batched with other
tile heights, bitwise against the domain alone."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers
from tests.test_gpu_parity import swe  # noqa: F401

pytestmark = pytest.mark.gpu

DT = 3.0


def _pools(nx=230, ny=170, seed=5):
    """Land everywhere except rectangular pools that straddle strip (28
    columns) and band edges, plus one pool of 2 x 2 cells."""
    wl = helpers.rough(nx, ny, seed=seed, land=False, min_depth=5.0, cd=0.002)
    land = np.ones((ny, nx), dtype=bool)
    for (j0, j1, i0, i1) in [(3, 20, 25, 60), (40, 41 + 30, 80, 140), (100, 160, 150, 229),
                             (150, 152, 10, 12), (60, 90, 0, 27)]:
        land[j0:j1, i0:i1] = False
    wl.H = synth.encode_land(np.where(wl.H == synth.LAND, 50.0, wl.H), land)
    wl.eta, wl.hu, wl.hv = helpers.random_state(wl, seed=seed + 3, amp=0.2, mom=0.4)
    return wl


def test_all_land_domain_steps_and_stays_put(swe):
    wl = helpers.flat(64, 40, dtype=np.float32, dt_fixed=DT)
    wl.H = np.full_like(wl.H, synth.LAND)
    rng = np.random.default_rng(1)
    wl.eta = rng.standard_normal(wl.eta.shape).astype(np.float32)  # land values are kept as given
    for prec in ("f32", "f32_kahan"):
        with swe.Domain(wl, prec) as d:
            d.step(5)
            st = d.state()
            info = d.info()
        assert info.error == 0 and info.step == 5 and info.t == pytest.approx(5 * DT)
        assert np.array_equal(st[0], wl.eta) and not st[1].any() and not st[2].any()


@pytest.mark.parametrize("prec", ["f32", "f32_kahan"])
def test_wet_pools_in_land_match_the_oracle(swe, oracle_mod, prec):
    wl = _pools().astype(np.float32)
    wl.params = synth.Params(dt_fixed=DT, cd=0.002)
    ref = oracle_mod.Oracle(wl).run(4)
    with swe.Domain(wl, prec) as d:
        d.step(4)
        st = d.state()
    scale = max(float(np.abs(r).max()) for r in ref[:3])
    dev = max(float(np.abs(np.asarray(g, np.float64) - r).max()) for g, r in zip(st, ref[:3]))
    assert dev <= 16 * float(np.spacing(np.float32(scale))), dev


def test_wet_pools_in_land_f64(swe, oracle_mod):
    wl = _pools()
    wl.params = synth.Params(dt_fixed=DT, cd=0.002)
    ref = oracle_mod.Oracle(wl).run(3)
    with swe.Domain(wl, "f64") as d:
        d.step(3)
        st = d.state()
    for a, b in zip(st, ref[:3]):
        assert helpers.rel(a, b) <= 1e-12


@pytest.mark.parametrize("rows", [8, 13, 64])
def test_wet_pools_batched_bitwise_equal_alone(swe, rows):
    wls = [_pools(seed=s).astype(np.float32) for s in (5, 6)]
    wls.append(synth.coastal(96, 80, seed_config=95, member=2, dtype=np.float32))
    wls.append(helpers.flat(50, 30, dtype=np.float32))
    wls[-1].H = np.full_like(wls[-1].H, synth.LAND)
    wls[-1].params = synth.Params(dt_fixed=DT)
    n = 12
    doms = [swe.Domain(wl, "f32_kahan") for wl in wls]
    with swe.Batch() as b:
        for d in doms:
            b.add(d)
        b.set_rows(rows)
        b.step(n)
        b.sync()
        got = [(d.state(), d.info()) for d in doms]
    for d in doms:
        d.close()
    for wl, (st, info) in zip(wls, got):
        with swe.Domain(wl, "f32_kahan") as d:
            d.step(n)
            ref, rinfo = d.state(), d.info()
        for a, r in zip(st, ref):
            assert np.array_equal(a, r), wl.name
        assert info.t == rinfo.t and info.step == rinfo.step == n
