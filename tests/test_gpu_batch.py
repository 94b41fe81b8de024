"""The batched path: many domains of uneven sizes advanced by one launch per
stage (graph-captured, autotuned tiles). Every domain's result
must be bitwise the one it gets alone: the per-cell arithmetic does not
depend on the tiling, and each domain keeps its own clock and reduction."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swe():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1912_02457_gb300 import build, swe as S
    build.build()
    S.load()
    return S


SHAPES = [(60, 40), (100, 90), (33, 150), (256, 200), (31, 7), (112, 64)]


def _members(dtype=np.float32):
    return [synth.coastal(nx, ny, seed_config=95, member=k, dtype=dtype, tide_phase=0.3 * k,
                          wind_speed=8.0 + k)
            for k, (nx, ny) in enumerate(SHAPES)]


def _alone(swe, wl, prec, n, t_end=0.0):
    with swe.Domain(wl, prec) as d:
        if t_end:
            d.set_end_time(t_end)
        d.step(n)
        return d.state(), d.info()


@pytest.mark.parametrize("rows", [0, 8, 64])
def test_batch_bitwise_equals_alone(swe, rows):
    wls = _members()
    precs = ["f32_kahan" if k % 2 == 0 else "f32" for k in range(len(wls))]
    n = 40
    doms = [swe.Domain(wl, p) for wl, p in zip(wls, precs)]
    with swe.Batch() as b:
        for d in doms:
            b.add(d)
        if rows:
            b.set_rows(rows)
        b.step(n)
        b.sync()
        if rows == 0:
            assert b.rows() in (8, 16, 32, 64)
        got = [(d.state(), d.info()) for d in doms]
    for d in doms:
        d.close()
    for wl, p, (st, info) in zip(wls, precs, got):
        ref, rinfo = _alone(swe, wl, p, n)
        for a, r in zip(st, ref):
            assert np.array_equal(a, r), wl.name
        assert info.t == rinfo.t and info.step == rinfo.step == n


def test_batch_serial_baseline_equals_batched(swe):
    wls = _members()[:4]
    outs = []
    for mode in ("batched", "serial"):
        doms = [swe.Domain(wl, "f32_kahan") for wl in wls]
        with swe.Batch() as b:
            for d in doms:
                b.add(d)
            b.set_rows(16)
            (b.step if mode == "batched" else b.step_serial)(21)
            b.sync()
            outs.append([d.state() for d in doms])
        for d in doms:
            d.close()
    for sa, sb in zip(*outs):
        for a, r in zip(sa, sb):
            assert np.array_equal(a, r)


def test_batch_horizons_and_membership(swe):
    """Domains with different end times: each lands exactly on its own, is
    skipped afterwards, and a domain added mid-run and one removed mid-run
    match their stand-alone runs."""
    wls = _members()[:4]
    t_ends = [60.0, 95.5, 0.0, 30.25]
    doms = [swe.Domain(wl, "f32_kahan") for wl in wls]
    for d, te in zip(doms[:3], t_ends[:3]):
        if te:
            d.set_end_time(te)
    with swe.Batch() as b:
        for d in doms[:3]:
            b.add(d)
        b.set_rows(32)
        b.step(30)
        b.remove(doms[1])                    # leaves after 30 steps
        doms[3].set_end_time(t_ends[3])
        b.add(doms[3])                        # joins after 30 steps
        b.step(170)
        done, t = b.poll()
        states = {k: doms[k].state() for k in (0, 2, 3)}
        infos = {k: doms[k].info() for k in (0, 2, 3)}
    removed_state, removed_info = doms[1].state(), doms[1].info()
    for d in doms:
        d.close()
    assert list(done) == [True, False, True]
    assert abs(infos[0].t - 60.0) <= 1e-12 * 60 and abs(infos[3].t - 30.25) <= 1e-12 * 30.25
    ref0 = _alone(swe, wls[0], "f32_kahan", 200, t_end=60.0)
    ref2 = _alone(swe, wls[2], "f32_kahan", 200)
    ref3 = _alone(swe, wls[3], "f32_kahan", 170, t_end=30.25)
    ref1 = _alone(swe, wls[1], "f32_kahan", 30, t_end=95.5)
    for (st, _), k in ((ref0, 0), (ref2, 2), (ref3, 3)):
        for a, r in zip(states[k], st):
            assert np.array_equal(a, r), k
    for a, r in zip(removed_state, ref1[0]):
        assert np.array_equal(a, r)
    assert removed_info.step == 30


def test_batch_rejects_f64(swe):
    wl = _members(np.float64)[0]
    with swe.Domain(wl, "f64") as d, swe.Batch() as b:
        with pytest.raises(swe.SweError):
            b.add(d)
