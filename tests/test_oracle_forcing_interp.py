"""Pins of the oracle's spatial interpolation of forcing frames (CPU only).

Section 3.5 interpolates the wind trilinearly (bilinear in space, linear in
time, eq:windstress_interpol) and Section 3.6 interpolates the nesting data
the same way along each edge. The frames are stored on their own, coarser
grids; a cell samples them texture-like at its centre. Linear interpolation
reproduces linear (and bilinear) data exactly, and beyond the outermost
samples the end value is held, so with such frames every interpolated value
has a closed form: the linear field evaluated at the cell centre, with the
coordinate clamped to the span of the samples. These tests feed frames that
vary along every axis (stored in float32 with dyadic values, so they are
exact) and compare the oracle's ghost cells and wind stress with that
closed form. A half-cell offset, swapped axes, a wrong clamp or a dropped
time weight each fails them."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers

T_A, T_B = 0.0, 4096.0


def _edge_value(e, r, v, x, t):
    """The external solution on edge e (0 S, 1 N, 2 W, 3 E), ghost ring r,
    variable v at along-edge position x (in cells from the edge's start) and
    time t: a different linear field for every edge, ring and variable."""
    a = 0.5 + 0.25 * r + 0.125 * v - 0.0625 * e
    b = (e + 1) * (-1) ** v * 2.0 ** -5
    c = (1 + v) * 2.0 ** -14
    return a + b * x + c * t


def _sample_pos(nb, n):
    """Sample s of nb samples spread over n cells sits at (s + 1/2) n / nb."""
    return (np.arange(nb) + 0.5) * n / nb


def _nested_linear(nx, ny, nbx, nby):
    wl = helpers.flat(nx, ny, depth=40.0, dx=600.0, dy=900.0, bc=(synth.BC_NESTED,) * 4)
    times = np.array([T_A, T_B])
    fr = np.zeros((2, 12 * (nbx + nby)), dtype=np.float32)
    lay = synth.boundary_layout(nbx, nby)
    for e, name in enumerate(synth.EDGES):
        o, s = lay[name]
        nb, n = (nbx, nx) if e < 2 else (nby, ny)
        blk = fr[:, o:o + s].reshape(2, 2, 3, nb)
        xs = _sample_pos(nb, n)
        for q, tq in enumerate(times):
            for r in range(2):
                for v in range(3):
                    blk[q, r, v, :] = _edge_value(e, r, v, xs, tq)
    assert np.array_equal(fr.astype(np.float64), fr)
    wl.boundary = synth.Forcing(times=times, frames=fr, nfx=nbx, nfy=nby)
    return wl


@pytest.mark.parametrize("nx,ny,nbx,nby", [
    (24, 18, 16, 8),     # n/nb = 1.5 and 2.25
    (20, 16, 10, 8),     # half resolution, as in the coastal recipe
    (12, 10, 12, 10),    # full resolution: every weight zero
    (9, 14, 1, 7),       # a single sample: held along the whole edge
])
def test_nested_ghosts_follow_linear_frames(oracle_mod, nx, ny, nbx, nby):
    wl = _nested_linear(nx, ny, nbx, nby)
    t = 1234.5
    st = helpers.random_state(wl, seed=2)
    G = oracle_mod.Oracle(wl).ghosts(*st, t=t)
    # interior untouched
    for v in range(3):
        assert np.array_equal(G[v, 2:-2, 2:-2], st[v])
    worst = 0.0
    for e in range(4):
        n, nb = (nx, nbx) if e < 2 else (ny, nby)
        xs = _sample_pos(nb, n)
        x = np.clip(np.arange(n) + 0.5, xs[0], xs[-1])
        for r in range(2):
            if e == 0:
                got = G[:, 1 - r, 2:-2]
            elif e == 1:
                got = G[:, ny + 2 + r, 2:-2]
            elif e == 2:
                got = G[:, 2:-2, 1 - r]
            else:
                got = G[:, 2:-2, nx + 2 + r]
            for v in range(3):
                want = _edge_value(e, r, v, x, t)
                err = np.abs(got[v] - want) / np.maximum(np.abs(want), 1.0)
                worst = max(worst, float(err.max()))
    assert worst <= 1e-14, worst


def test_clamp_holds_the_end_samples(oracle_mod):
    """Cells beyond the first / last sample centre take exactly the end
    sample (no extrapolation); between the sample centres the values follow
    the frames' slope."""
    nx, ny, nbx, nby = 24, 18, 6, 3       # 4 and 6 cells per sample
    wl = _nested_linear(nx, ny, nbx, nby)
    st = helpers.random_state(wl, seed=3)
    G = oracle_mod.Oracle(wl).ghosts(*st, t=T_A)
    south = G[0, 1, 2:-2]                  # ring 0 of the S edge, eta
    first, last = _edge_value(0, 0, 0, 2.0, T_A), _edge_value(0, 0, 0, 22.0, T_A)
    # cell centres 0.5, 1.5 lie before the first sample centre (2.0)
    assert south[0] == first and south[1] == first
    assert south[-1] == last and south[-2] == last
    # in between: the edge's slope (1/32 per cell) on every step
    assert np.abs(np.diff(south[2:-2]) - 2.0 ** -5).max() <= 1e-15


def _wind_field(X, Y, t):
    """Wind in grid axes (m/s) at (X, Y) in cells and time t: linear in each
    coordinate with a bilinear cross term."""
    wx = 4.0 + 0.25 * X - 0.125 * Y + 2.0 ** -9 * X * Y + 2.0 ** -12 * t
    wy = -3.0 + 0.0625 * X + 0.1875 * Y - 2.0 ** -13 * t
    return wx, wy


@pytest.mark.parametrize("nx,ny,nfx,nfy", [(24, 16, 6, 4), (30, 12, 5, 12), (16, 20, 1, 5)])
def test_wind_is_bilinear_in_space(oracle_mod, nx, ny, nfx, nfy):
    """Still, flat, non-rotating water: every flux and bed term vanishes, so
    the momentum tendency of each cell is the Large & Pond stress (pinned
    separately against hand-worked values) of the wind interpolated at the
    cell centre, here the closed-form field at the clamped centre."""
    wl = helpers.flat(nx, ny, depth=50.0, dx=1000.0, dy=1000.0)
    xs, ys = _sample_pos(nfx, nx), _sample_pos(nfy, ny)
    times = np.array([T_A, T_B])
    fr = np.zeros((2, nfy, nfx, 2), dtype=np.float32)
    for q, tq in enumerate(times):
        wx, wy = _wind_field(xs[None, :], ys[:, None], tq)
        fr[q, :, :, 0], fr[q, :, :, 1] = wx, wy
    assert np.array_equal(fr.astype(np.float64),
                          np.stack(np.broadcast_arrays(*_stack_field(xs, ys, times)), -1))
    wl.wind = synth.Forcing(times=times, frames=fr, nfx=nfx, nfy=nfy)
    t = 1000.5
    M, S = oracle_mod.Oracle(wl).rhs(wl.eta, wl.hu, wl.hv, t=t)
    X = np.clip(np.arange(nx) + 0.5, xs[0], xs[-1])[None, :] * np.ones((ny, 1))
    Y = np.clip(np.arange(ny) + 0.5, ys[0], ys[-1])[:, None] * np.ones((1, nx))
    wx, wy = _wind_field(X, Y, t)
    speed = np.hypot(wx, wy)
    assert np.abs(speed - 11.0).min() > 1e-3      # away from the drag-law switch
    assert np.all(M[0] == 0.0) and np.all(S == 0.0)
    for j in range(ny):
        for i in range(nx):
            tx, ty = oracle_mod.wind_stress(wx[j, i], wy[j, i])
            assert abs(M[1, j, i] - tx) <= 1e-13 * abs(tx) + 1e-300
            assert abs(M[2, j, i] - ty) <= 1e-13 * abs(ty) + 1e-300


def _stack_field(xs, ys, times):
    wx, wy = _wind_field(xs[None, None, :], ys[None, :, None], times[:, None, None])
    return wx, wy
