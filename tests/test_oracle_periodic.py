"""Pins of the oracle's periodic boundaries (Section 3.3) and of the
beta-plane workload (eq:betaplane, Section 3.7): cyclic-shift equivariance
bit for bit, lake at rest, exact mass conservation, reflection equivariance,
and the westward drift of a geostrophic bump on a beta plane (Rossby-wave
dynamics), for two orientations of north."""
import numpy as np
import pytest

import helpers
from paper_1912_02457_gb300 import synth


def _roll_wl(wl, dj, di):
    c = wl.copy()
    for k in ("eta", "hu", "hv", "f", "theta"):
        setattr(c, k, np.roll(np.roll(getattr(wl, k), dj, axis=0), di, axis=1).copy())
    # roll the corner plane on its periodic lattice (the last line repeats the first)
    H = wl.H.copy()
    if wl.bc[2] == synth.BC_PERIODIC:
        core = np.roll(H[:, :-1], di, axis=1)
        H = np.concatenate([core, core[:, :1]], axis=1)
    if wl.bc[0] == synth.BC_PERIODIC:
        core = np.roll(H[:-1, :], dj, axis=0)
        H = np.concatenate([core, core[:1, :]], axis=0)
    c.H = H
    return c


@pytest.mark.parametrize("periodic,shift", [((True, True), (3, 5)), ((True, False), (0, 7)),
                                            ((False, True), (4, 0))])
@pytest.mark.parametrize("land", [False, True])
def test_cyclic_shift_equivariance_is_bitwise(oracle_mod, periodic, shift, land):
    wl = helpers.periodic_rough(24, 18, seed=3, land=land, periodic=periodic)
    e, u, v = helpers.random_state(wl, seed=4, amp=0.2, mom=0.4)
    wl.eta, wl.hu, wl.hv = e, u, v
    dj, di = shift
    a = oracle_mod.Oracle(wl).run(25)
    b = oracle_mod.Oracle(_roll_wl(wl, dj, di)).run(25)
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(np.roll(np.roll(x, dj, axis=0), di, axis=1), y)


def test_lake_at_rest_is_exact_with_periodic_edges(oracle_mod):
    wl = helpers.periodic_rough(20, 16, seed=1, land=True)
    out = oracle_mod.Oracle(wl).run(50)
    for x in out[:3]:
        assert np.all(x == 0.0)


def test_mass_is_conserved_with_periodic_edges(oracle_mod):
    wl = helpers.periodic_rough(22, 20, seed=2, land=True)
    e, u, v = helpers.random_state(wl, seed=5, amp=0.3, mom=0.5)
    wl.eta, wl.hu, wl.hv = e, u, v
    m0 = e.sum()
    out = oracle_mod.Oracle(wl).run(100)
    assert abs(out[0].sum() - m0) <= 1e-12 * np.abs(e).sum()


@pytest.mark.parametrize("transform", ["flip_x", "flip_y", "transpose", "rot180"])
def test_reflections_with_periodic_edges(oracle_mod, transform):
    wl = helpers.periodic_rough(18, 14, seed=6, land=True)
    e, u, v = helpers.random_state(wl, seed=7)
    wl.eta, wl.hu, wl.hv = e, u, v
    T = getattr(helpers, transform)
    TS = getattr(helpers, transform + "_state")
    w2 = T(wl)
    w2.eta, w2.hu, w2.hv = TS(e, u, v)
    a = oracle_mod.Oracle(wl).run(20)
    b = oracle_mod.Oracle(w2).run(20)
    for x, y in zip(TS(*a[:3]), b[:3]):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-12 * max(np.abs(y).max(), 1e-30))


def test_unpaired_periodic_edge_is_rejected(oracle_mod):
    wl = helpers.periodic_rough(8, 8, seed=1)
    wl.bc = (synth.BC_PERIODIC, synth.BC_WALL, synth.BC_PERIODIC, synth.BC_PERIODIC)
    with pytest.raises(Exception):
        oracle_mod.Oracle(wl).run(1)


def _centroid(eta, c0):
    """eta-weighted centre of the bump's core (eta above half its maximum),
    in cells, unwrapped around the initial centre c0."""
    n = eta.shape[0]
    j, i = np.mgrid[0:n, 0:n]
    w = np.where(eta > 0.5 * eta.max(), eta, 0.0)
    dx = (i + 0.5 - c0 + n / 2) % n - n / 2
    dy = (j + 0.5 - c0 + n / 2) % n - n / 2
    return float((w * dx).sum() / w.sum()), float((w * dy).sum() / w.sum())


def _drift(oracle_mod, theta, beta, days, n=64):
    wl = synth.rossby(n=n, theta=theta, days=days, beta=beta)
    out = oracle_mod.Oracle(wl).run(100000, t_end=days * 86400.0)
    d = np.array(_centroid(out[0], n / 2.0))
    east = np.array([np.cos(theta), -np.sin(theta)])
    north = np.array([np.sin(theta), np.cos(theta)])
    return -(d @ east), d @ north          # westward and northward, in cells


def test_bump_drifts_west_on_a_beta_plane_for_any_north(oracle_mod):
    days, dx, g, H, f, beta, R = 2.0, 20e3, 9.81, 50.0, 8e-5, 2e-11, 10 * 20e3
    # linear estimate of the westward drift of a Gaussian of radius R: the
    # long-Rossby-wave speed beta Rd^2 reduced by the finite scale,
    # beta Rd^2 / (1 + Rd^2 / R^2), Rd = sqrt(g H) / f (~0.5 m/s here)
    Rd2 = g * H / f ** 2
    est = beta * Rd2 / (1.0 + Rd2 / R ** 2) * days * 86400.0 / dx
    west0, north0 = _drift(oracle_mod, 0.0, beta, days)
    west90, north90 = _drift(oracle_mod, np.pi / 2, beta, days)
    assert 0.5 * est < west0 < 1.5 * est
    assert abs(north0) < 0.25 * west0        # nearly linear: no marked meridional drift
    # the same drift relative to north whatever the grid's orientation
    assert abs(west90 - west0) < 0.05 and abs(north90 - north0) < 0.05
    # without beta the bump stays in place
    w, nn = _drift(oracle_mod, 0.0, 0.0, days)
    assert abs(w) < 0.05 and abs(nn) < 0.05
