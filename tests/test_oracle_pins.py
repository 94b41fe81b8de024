"""Pins of the FP64 oracle's building blocks against closed forms the paper
fixes (CPU only)."""
import os

import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_desingularisation_closed_form(oracle_mod):
    """eq:desing_ours: h* = h for |h| >= kappa, kappa/2 at h = 0 (sign(0)=+1),
    +-kappa at +-kappa, odd, continuous with a continuous slope at kappa,
    and never smaller in magnitude than |h|."""
    k = 1e-2
    d = oracle_mod.desing
    for h in (k, 2 * k, 1.0, 3000.0, -k, -5.0):
        assert d(h, k) == h
    assert d(0.0, k) == k / 2
    hs = np.linspace(-3 * k, 3 * k, 6001)
    v = np.array([d(h, k) for h in hs])
    assert np.all(np.abs(v) >= np.abs(hs))
    assert np.all(np.diff(v[hs > 0]) > 0)
    # below kappa: the quadratic kappa/2 + h^2/(2 kappa); odd symmetry
    h = 0.37 * k
    assert abs(d(h, k) - (k / 2 + h * h / (2 * k))) < 1e-18
    assert d(-h, k) == -d(h, k)
    # continuity of value and slope at kappa
    eps = 1e-9
    assert abs(d(k - eps, k) - d(k + eps, k)) < 3 * eps
    slope_l = (d(k - eps, k) - d(k - 2 * eps, k)) / eps
    assert abs(slope_l - 1.0) < 1e-5


def test_minmod(oracle_mod):
    mm = oracle_mod.minmod
    assert mm(1.0, 2.0, 3.0) == 1.0
    assert mm(-1.0, -2.0, -0.5) == -0.5
    assert mm(1.0, -2.0, 3.0) == 0.0
    assert mm(0.0, 2.0, 3.0) == 0.0


def test_wind_stress_golden(oracle_mod):
    rows = np.loadtxt(os.path.join(GOLDEN, "wind_stress.txt"))
    for wx, wy, tx, ty in rows:
        gx, gy = oracle_mod.wind_stress(wx, wy)
        assert abs(gx - tx) <= 1e-12 * max(abs(tx), 1e-30) + 1e-20
        assert abs(gy - ty) <= 1e-12 * max(abs(ty), 1e-30) + 1e-20


def test_wind_drives_uniform_water(oracle_mod):
    """Uniform 10 m/s wind on still, flat, non-rotating water: in the
    interior every flux difference vanishes and RK2 integrates the constant
    stress exactly, hu = n dt tau with tau from the golden table."""
    wl = helpers.flat(96, 96, depth=50.0, dx=2000.0, dy=2000.0, dt_fixed=20.0)
    wl.wind = synth.uniform_wind(10.0, 0.0)
    o = oracle_mod.Oracle(wl)
    n = 8
    e, u, v, t, dt = o.run(n)
    tau = 1.43414634146341e-04
    c = 48
    assert abs(u[c, c] - n * 20.0 * tau) < 1e-12 * n * 20.0 * tau
    assert v[c, c] == 0.0
    assert abs(e[c, c]) < 1e-15


def test_cfl_closed_form(oracle_mod):
    """eq:cfl on still water of depth H: dt = C/4 * dx / sqrt(g H)."""
    wl = helpers.flat(16, 12, depth=100.0, dx=800.0, dy=600.0)
    o = oracle_mod.Oracle(wl)
    s = o.max_speed(wl.eta, wl.hu, wl.hv)
    assert abs(s - np.sqrt(9.81 * 100.0) / 600.0) < 1e-15
    # a moving cell: (|u| + c)/dx wins when it is larger
    e, u, v = wl.eta.copy(), wl.hu.copy(), wl.hv.copy()
    u[3, 4] = 100.0 * 40.0
    s = o.max_speed(e, u, v)
    assert abs(s - (40.0 + np.sqrt(981.0)) / 800.0) < 1e-14
    e2, *_ , dt = o.run(1, courant=0.8)
    assert abs(dt - 0.8 * 0.25 * 600.0 / np.sqrt(981.0)) < 1e-12


def test_frames_time_interpolation(oracle_mod):
    """Nested edges with frames eta = a + b t on the whole boundary and a flat
    lake inside: stage one sees the frame at t, and the relaxation at the
    outermost interior cell (alpha = 1) writes the frame at t + dt exactly."""
    nx = ny = 24
    wl = helpers.flat(nx, ny, depth=20.0, dx=500.0, dy=500.0, dt_fixed=5.0,
                      bc=(synth.BC_NESTED,) * 4)
    times = np.array([0.0, 100.0, 300.0])
    vals = np.array([0.0, 0.1, -0.2])
    bnd = synth.still_boundary(nx, ny, 0.0, times=times)
    lay = synth.boundary_layout(nx, ny)
    for e, (o_, s) in lay.items():
        blk = bnd.frames[:, o_:o_ + s].reshape(3, 2, 3, -1)
        blk[:, :, 0, :] = vals[:, None, None]
    wl.boundary = bnd
    o = oracle_mod.Oracle(wl)
    e, u, v, t, dt = o.run(1, t=140.0)
    # frame value at 145 s, between the (float32) frames at 100 s and 300 s
    v32 = vals.astype(np.float32).astype(np.float64)
    sw = 45.0 / 200.0
    expect = (1.0 - sw) * v32[1] + sw * v32[2]
    assert abs(e[ny // 2, 0] - expect) < 1e-15
    assert abs(e[0, nx // 2] - expect) < 1e-15


def test_frs_weights(oracle_mod):
    """eq:frs: a still lake relaxed toward a still external level eta_ext
    keeps the interior exactly and moves each cell of the zone by
    alpha(d) = 1 - tanh(d/d0) of the difference."""
    nx, ny = 40, 30
    wl = helpers.flat(nx, ny, depth=20.0, dx=500.0, dy=500.0, dt_fixed=1e-9,
                      bc=(synth.BC_WALL, synth.BC_WALL, synth.BC_NESTED, synth.BC_WALL),
                      frs_width=10, frs_d0=2.5)
    wl.boundary = synth.still_boundary(nx, ny, 0.5)
    o = oracle_mod.Oracle(wl)
    e, u, v, t, dt = o.run(1)
    row = e[ny // 2]
    for d in range(12):
        a = 1.0 - np.tanh(d / 2.5) if d < 10 else 0.0
        assert abs(row[d] - a * 0.5) < 1e-9, d
