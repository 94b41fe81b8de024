"""Steady states and conservation the paper names, pinned on the FP64 oracle
(CPU only): lake at rest (eq:lakeatrest) with and without land, geostrophic
balance (eq:geostrophicBalance), exact mass conservation under walls, and
the wall-boundary construction of Section 3.3 against a land ring."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers


@pytest.mark.parametrize("land", [False, True])
def test_lake_at_rest_bitwise(oracle_mod, land):
    """eta = 0, hu = hv = 0 over rough bathymetry, a land mask, varying f and
    north angle and quadratic drag: every step leaves the state bit-exact."""
    wl = helpers.rough(48, 40, seed=3, land=land, min_depth=0.5, cd=0.0025, courant=0.8)
    assert (wl.land_cells().sum() > 0) == land
    o = oracle_mod.Oracle(wl)
    e, u, v, t, dt = o.run(20)
    assert np.array_equal(e, wl.eta)
    assert np.array_equal(u, wl.hu)
    assert np.array_equal(v, wl.hv)


@pytest.mark.parametrize("land", [False, True])
def test_lake_at_rest_raised_level(oracle_mod, land):
    """eta = 0.25 m everywhere (still a lake at rest): changes stay at
    round-off of the pressure terms."""
    wl = helpers.rough(48, 40, seed=4, land=land, min_depth=0.5)
    wl.eta = np.where(wl.land_cells(), 0.0, 0.25)
    o = oracle_mod.Oracle(wl)
    e, u, v, t, dt = o.run(20)
    wet = ~wl.land_cells()
    # eta is reconstructed exactly flat, so the mass flux is exactly zero
    assert np.abs(e[wet] - 0.25).max() == 0.0
    assert np.abs(u).max() < 1e-9 and np.abs(v).max() < 1e-9


def test_lake_at_rest_nested_still_frames(oracle_mod):
    """Nested edges whose frames hold the same still water: bit-exact rest."""
    wl = helpers.rough(40, 36, seed=5, land=True, min_depth=0.5)
    wl.bc = (synth.BC_NESTED, synth.BC_NESTED, synth.BC_NESTED, synth.BC_WALL)
    wl.boundary = synth.still_boundary(wl.nx, wl.ny, 0.0)
    o = oracle_mod.Oracle(wl)
    e, u, v, t, dt = o.run(10)
    assert np.array_equal(e, wl.eta) and np.array_equal(u, wl.hu) and np.array_equal(v, wl.hv)


def _geostrophic_profile(nx, dx, H, f, q, g=9.81):
    """eta_i with hv = q, u = 0 so that the local K differences of
    eq:Kbackwards vanish: eta_{i+1} - eta_i = dx/(2g)(f_i v_i + f_{i+1} v_{i+1}),
    v = q / (eta + H). Solved cell by cell (a quadratic per step)."""
    k = dx / (2 * g)
    eta = np.zeros(nx)
    for i in range(nx - 1):
        R = eta[i] + k * f[i] * q / (eta[i] + H[i])
        a = k * f[i + 1] * q
        b = H[i + 1]
        # x - a/(x+b) = R  ->  x^2 + (b-R) x - (R b + a) = 0
        B = b - R
        eta[i + 1] = 0.5 * (-B + np.sqrt(B * B + 4 * (R * b + a)))
    return eta


def test_geostrophic_balance(oracle_mod):
    """A jet in geostrophic balance (eq:geostrophicBalance): u = 0, constant
    hv, eta built from the local reformulation, f varying with x, walls in x,
    nested y edges whose (float32) frames hold the same state.

    Rows out of reach of the ghost rows see the exact balance: M vanishes to
    double round-off, and stays so for the steps the stencil needs to carry
    the float32 rounding of the frames inward (two cells per stage)."""
    nx, ny = 64, 40
    dx = 2000.0
    xc = np.arange(nx + 1)
    Hx = 200.0 + 60.0 * np.sin(xc / 9.0)           # corner depth, x only
    Hbar = 0.5 * (Hx[:-1] + Hx[1:])
    fx = 1.1e-4 + 4e-7 * np.arange(nx)
    q = 20.0
    eta_x = _geostrophic_profile(nx, dx, Hbar, fx, q)
    wl = helpers.flat(nx, ny, dx=dx, dy=dx,
                      bc=(synth.BC_NESTED, synth.BC_NESTED, synth.BC_WALL, synth.BC_WALL),
                      dt_fixed=30.0)
    wl.H = np.tile(Hx, (ny + 1, 1))
    wl.f = np.tile(fx, (ny, 1))
    wl.theta = np.zeros((ny, nx))
    wl.eta = np.tile(eta_x, (ny, 1))
    wl.hv = np.full((ny, nx), q)
    bnd = synth.still_boundary(nx, ny, 0.0)
    lay = synth.boundary_layout(nx, ny)
    for e in ("S", "N"):
        o_, s = lay[e]
        blk = bnd.frames[:, o_:o_ + s].reshape(2, 2, 3, nx)
        blk[:, :, 0, :] = eta_x.astype(np.float32)
        blk[:, :, 2, :] = q
    wl.boundary = bnd
    o = oracle_mod.Oracle(wl)
    M, S = o.rhs(wl.eta, wl.hu, wl.hv)
    inner = slice(3, ny - 3)
    assert np.abs(fx * q).max() > 2e-3          # size of each balanced term
    assert np.abs(M[0][inner]).max() < 1e-15
    assert np.abs(M[1][inner]).max() < 1e-13
    assert np.abs(M[2][inner]).max() < 1e-13
    e, u, v, t, dt = o.run(3)
    core = slice(3 * 4 + 2, ny - 3 * 4 - 2)
    assert helpers.rel(e[core], wl.eta[core]) < 1e-12
    assert np.abs(u[core]).max() < 1e-10
    assert helpers.rel(v[core], wl.hv[core]) < 1e-13
    # the whole domain stays balanced to the float32 rounding of the frames
    e, u, v, t, dt = o.run(20)
    assert helpers.rel(e, wl.eta) < 1e-4
    assert helpers.rel(v, wl.hv) < 1e-4


def test_geostrophic_balance_exact_float64(oracle_mod):
    """Same jet with walls on all four sides and eta kept in float64: the
    reconstruction balances f hv to round-off of double precision."""
    nx, ny = 64, 8
    dx = 2000.0
    Hbar = np.full(nx, 150.0)
    fx = 1.1e-4 + 4e-7 * np.arange(nx)
    q = 20.0
    eta_x = _geostrophic_profile(nx, dx, Hbar, fx, q)
    wl = helpers.flat(nx, ny, depth=150.0, dx=dx, dy=dx, dt_fixed=30.0)
    wl.f = np.tile(fx, (ny, 1))
    wl.eta = np.tile(eta_x, (ny, 1))
    wl.hv = np.full((ny, nx), q)
    o = oracle_mod.Oracle(wl)
    M, S = o.rhs(wl.eta, wl.hu, wl.hv)
    # interior rows are steady; the walls in y reflect hv (normal momentum
    # there), so only the x-balance is checked on the middle rows
    mid = slice(3, ny - 3)
    assert np.abs(M[0][mid]).max() < 1e-15
    assert np.abs(M[1][mid]).max() < 1e-13   # vs f hv ~ 2.4e-3
    assert np.abs(fx * q).max() > 2e-3


def test_mass_conservation_walls(oracle_mod):
    """Walls, land, wet-dry fronts, drag and wind: sum(eta) changes only by
    round-off (every interior mass flux telescopes; wall and coast faces
    carry exactly none)."""
    wl = synth.coastal(64, 48, seed_config=91, dtype=np.float64)
    wl.bc = (synth.BC_WALL,) * 4
    wl.boundary = None
    wl.params.courant = 0.8
    o = oracle_mod.Oracle(wl)
    m0, _ = o.diagnostics(wl.eta, wl.hu, wl.hv)
    e, u, v, t, dt = o.run(40)
    m1, _ = o.diagnostics(e, u, v)
    scale = np.abs(e).sum() * wl.dx * wl.dy
    assert abs(m1 - m0) < 1e-12 * max(scale, 1.0)
    assert np.abs(u).max() > 0  # wind and wet-dry really moved water


def test_wall_equals_land_ring(oracle_mod):
    """Section 3.3's wall (ghost mirror with odd f) and Section 3.4's land
    wall give the same solution: a walled domain equals the same domain
    inside a two-cell ring of land."""
    wl = helpers.rough(36, 30, seed=6, land=True, cd=0.001)
    wl.eta, wl.hu, wl.hv = helpers.random_state(wl, seed=2, amp=0.2, mom=0.4)
    wl.eta = np.where(wl.land_cells(), 0.0, wl.eta + 0.1)
    ring = helpers.land_ring(wl, 2)
    a = oracle_mod.Oracle(wl).run(12, dt_fixed=5.0)
    b = oracle_mod.Oracle(ring).run(12, dt_fixed=5.0)
    for x, y in zip(a[:3], b[:3]):
        assert helpers.rel(x, y[2:-2, 2:-2]) < 1e-13


def test_wall_equals_land_ring_one_cell_wide(oracle_mod):
    """A domain one cell wide (x or y) with walls: the second ghost row is
    the double reflection of the single cell, which must again equal the same
    column standing inside a ring of land."""
    for nx, ny in ((1, 17), (17, 1)):
        wl = helpers.flat(nx, ny, depth=30.0, dx=500.0, dy=700.0, f=1e-4, theta=0.2)
        wl.eta, wl.hu, wl.hv = helpers.random_state(wl, seed=nx * 131 + ny, amp=0.2, mom=1.0)
        ring = helpers.land_ring(wl, 2)
        a = oracle_mod.Oracle(wl).run(25, dt_fixed=2.0)
        b = oracle_mod.Oracle(ring).run(25, dt_fixed=2.0)
        for x, y in zip(a[:3], b[:3]):
            assert helpers.rel(x, y[2:-2, 2:-2]) < 1e-13
