"""Parity on the other benchmark shapes, 1000 steps against the FP64 oracle
through the entry points the benchmark times: the coastline-scale
2600 x 900 and the 2048 x 2048 domains of the size sweep (stepped alone),
and a 2048 x 1024 ensemble member stepped inside a batch of uneven
domains. Front-aware float32 bounds as for the 1024 x 1024 workload."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests.test_gpu_parity import (T_FRONTS, assert_f32_parity_fronts, front_references, gpu_run,  # noqa: F401
                                   swe)

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("shape", [(2600, 900), (2048, 2048)])
def test_sweep_shape_1000_steps(swe, oracle_mod, shape):
    nx, ny = shape
    wl = synth.coastal(nx, ny, dtype=np.float32)
    ref, front = front_references(oracle_mod, wl, 1000)
    st, info = gpu_run(swe, wl, 1000, "f32_kahan")
    assert info.step == 1000
    assert_f32_parity_fronts(st, wl, ref, front)
    assert abs(info.t - ref[3]) <= T_FRONTS * ref[3]


def test_ensemble_member_in_a_batch_1000_steps(swe, oracle_mod):
    """The first 2048 x 1024 member of the seeded ensemble, advanced in one
    batch with three smaller members (one launch per stage for all four)."""
    wls = synth.ensemble(64)
    big = next(w for w in wls if (w.nx, w.ny) == (2048, 1024))
    small = [w for w in wls if w.nx * w.ny <= 512 * 384][:3]
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
    assert abs(info.t - ref[3]) <= T_FRONTS * ref[3]
