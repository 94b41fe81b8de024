"""Equivariance and invariance pins of the FP64 oracle (CPU only).

Mirroring x or y, or swapping the axes, reverses the sense of rotation
(f -> -f) and maps the north vector accordingly; a half turn keeps f. The
discrete scheme must commute with each map to round-off. Also: the north
vector enters only through f (Section 3.7's projection reduces to
f [0, hv, -hu] for every angle), so changing theta alone changes nothing."""
import numpy as np
import pytest

from tests import helpers


def _case(seed=11):
    wl = helpers.rough(40, 32, seed=seed, land=True, cd=0.002)
    wl.eta, wl.hu, wl.hv = helpers.random_state(wl, seed=seed, amp=0.2, mom=0.5)
    wl.eta = np.where(wl.land_cells(), 0.0, wl.eta + 0.05)
    return wl


def _run(oracle_mod, wl, n=8):
    return oracle_mod.Oracle(wl).run(n, dt_fixed=4.0)[:3]


@pytest.mark.parametrize("name", ["flip_x", "flip_y", "transpose", "rot180"])
def test_equivariance(oracle_mod, name):
    wl = _case()
    T = getattr(helpers, name)
    Ts = getattr(helpers, name + "_state")
    base = _run(oracle_mod, wl)
    twl = T(wl)
    twl.eta, twl.hu, twl.hv = (np.ascontiguousarray(a) for a in Ts(wl.eta, wl.hu, wl.hv))
    moved = _run(oracle_mod, twl)
    expect = Ts(*base)
    for a, b in zip(moved, expect):
        assert helpers.rel(a, b) < 1e-12, name


def test_north_vector_invariance(oracle_mod):
    wl = _case(12)
    a = _run(oracle_mod, wl)
    wl0 = wl.copy()
    wl0.theta = np.zeros_like(wl.theta)
    b = _run(oracle_mod, wl0)
    wl1 = wl.copy()
    wl1.theta = wl.theta + 1.234
    c = _run(oracle_mod, wl1)
    for x, y, z in zip(a, b, c):
        assert helpers.rel(x, y) < 1e-12
        assert helpers.rel(x, z) < 1e-12


def test_rotation_sense_matters(oracle_mod):
    """Sanity of the pins above: flipping x *without* flipping f does change
    the result (so the equivariance test is not vacuous)."""
    wl = _case(13)
    base = _run(oracle_mod, wl)
    twl = helpers.flip_x(wl)
    twl.f = -twl.f
    twl.eta, twl.hu, twl.hv = (np.ascontiguousarray(a) for a in helpers.flip_x_state(wl.eta, wl.hu, wl.hv))
    moved = _run(oracle_mod, twl)
    expect = helpers.flip_x_state(*base)
    assert helpers.rel(moved[1], expect[1]) > 1e-6
