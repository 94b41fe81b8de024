"""Parity on the other benchmark shapes, 1000 steps against the FP64 oracle
through the entry points the benchmark times: the coastline-scale
2600 x 900 and the 2048 x 2048 domains of the size sweep (stepped alone),
and a 2048 x 1024 ensemble member stepped inside a batch of uneven
domains. Front-aware float32 bounds as for the 1024 x 1024 workload.

Both sides step with the same fixed time step (0.15 of the CFL step of the
initial state; the oracle's adaptive step on the 2048 x 2048 recipe never
falls below 0.16 of it in 1000 steps). With adaptive steps the CFL maximum sits on thin films at
fronts on many steps, so after 1000 steps the two clocks differ by a
fraction of a second on these domains and the tide moves every level by
its rate times that shift; the fixed step compares the arithmetic at equal
times (the adaptive clock is checked on the 1024 x 1024 workload)."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests.test_gpu_parity import assert_f32_parity_fronts, front_references, gpu_run, swe  # noqa: F401

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def fixed_step(oracle_mod, wl, factor=0.15):
    """Set a fixed time step of `factor` times the CFL step of the initial state."""
    o = oracle_mod.Oracle(wl)
    wl.params.dt_fixed = factor * wl.params.courant * 0.25 / o.max_speed(wl.eta, wl.hu, wl.hv)
    return wl.params.dt_fixed


@pytest.mark.parametrize("shape", [(2600, 900), (2048, 2048)])
def test_sweep_shape_1000_steps(swe, oracle_mod, shape):
    nx, ny = shape
    wl = synth.coastal(nx, ny, dtype=np.float32)
    dt = fixed_step(oracle_mod, wl)
    ref, front = front_references(oracle_mod, wl, 1000)
    st, info = gpu_run(swe, wl, 1000, "f32_kahan")
    assert info.step == 1000 and info.dt == dt
    assert_f32_parity_fronts(st, wl, ref, front)
    assert abs(info.t - ref[3]) <= 1e-9 * ref[3]


def test_ensemble_member_in_a_batch_1000_steps(swe, oracle_mod):
    """The first 2048 x 1024 member of the seeded ensemble, advanced in one
    batch with three smaller members (one launch per stage for all four)."""
    wls = synth.ensemble(64)
    big = next(w for w in wls if (w.nx, w.ny) == (2048, 1024))
    small = [w for w in wls if w.nx * w.ny <= 512 * 384][:3]
    for w in [big] + small:
        fixed_step(oracle_mod, w)
    ref, front = front_references(oracle_mod, big, 1000)
    doms = [swe.Domain(w, "f32_kahan") for w in [big] + small]
    with swe.Batch() as b:
        for d in doms:
            b.add(d)
        b.step(1000)
        b.sync()
    st = doms[0].state()
    info = doms[0].info()
    for d in doms:
        d.close()
    assert info.step == 1000
    assert_f32_parity_fronts(st, big, ref, front)
    assert abs(info.t - ref[3]) <= 1e-9 * ref[3]
