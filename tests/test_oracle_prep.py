"""Pins of the pre-processing oracle (oracle/prep.py) against what the
mathematics fixes: closed forms on linear and bilinear surfaces, brute force
on tiny grids, and library routines (scipy.ndimage) for the morphology."""
import numpy as np
import pytest

from oracle import prep


def _lin_cells(nx, ny, a, b, c, d=0.0):
    """Cell averages of a + b x + c y + d x y over the unit cells (the
    average of x y over a cell is the product of the centre coordinates)."""
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    return a + b * x[None, :] + c * y[:, None] + d * (y[:, None] * x[None, :])


def _lin_corners(nx, ny, a, b, c, d=0.0):
    X = np.arange(nx + 1, dtype=np.float64)
    Y = np.arange(ny + 1, dtype=np.float64)
    return a + b * X[None, :] + c * Y[:, None] + d * (Y[:, None] * X[None, :])


def test_gminmod_cases():
    assert prep.gminmod(1.0, 2.0, 3.0) == 1.0
    assert prep.gminmod(3.0, 0.5, 2.0) == 0.5
    assert prep.gminmod(-1.0, -2.0, -3.0) == -1.0
    assert prep.gminmod(1.0, -1.0, 2.0) == 0.0
    assert prep.gminmod(0.0, 1.0, 1.0) == 0.0


@pytest.mark.parametrize("nx,ny", [(7, 5), (1, 6), (9, 1), (2, 2)])
def test_linear_surface_is_reconstructed_exactly(nx, ny):
    Hm = _lin_cells(nx, ny, 40.0, 3.0, -2.0)
    exact = _lin_corners(nx, ny, 40.0, 3.0, -2.0)
    if nx == 1:        # a single column has no x slope: only the y part is recoverable
        exact = _lin_corners(nx, ny, 40.0 + 3.0 * 0.5, 0.0, -2.0)
    if ny == 1:
        exact = _lin_corners(nx, ny, 40.0 - 2.0 * 0.5, 3.0, 0.0)
    np.testing.assert_allclose(prep.initial_corners(Hm), exact, rtol=0, atol=1e-12)
    Hc, misfit, change = prep.reconstruct_bathymetry(Hm, n_iter=8)
    np.testing.assert_allclose(Hc, exact, rtol=0, atol=1e-11)
    assert max(misfit) < 1e-11 and max(change) < 1e-11


def test_bilinear_surface_initial_guess_errs_only_at_domain_corners():
    nx, ny, d = 8, 6, 0.8
    Hm = _lin_cells(nx, ny, 100.0, 1.5, 2.5, d)
    exact = _lin_corners(nx, ny, 100.0, 1.5, 2.5, d)
    err = prep.initial_corners(Hm) - exact
    corners = np.zeros_like(err, dtype=bool)
    corners[[0, 0, -1, -1], [0, -1, 0, -1]] = True
    # a cell's plane misses the x y term by -+ d/4 at its corners; four (or
    # two) estimates cancel it, a domain corner has only one
    np.testing.assert_allclose(err[~corners], 0.0, atol=1e-12)
    np.testing.assert_allclose(np.abs(err[corners]), d / 4, atol=1e-12)
    # the exact bilinear corners are a fixed point of the iteration
    Hc = exact.copy()
    dH = Hm - prep.midpoints(Hc)
    np.testing.assert_allclose(dH, 0.0, atol=1e-12)
    np.testing.assert_allclose(prep.smooth_corners(Hc, 0.3), exact, atol=1e-11)
    # and the iteration moves the domain corners towards it
    Hc10, _, _ = prep.reconstruct_bathymetry(Hm, n_iter=10)
    assert np.abs(Hc10 - exact).max() < 0.5 * d / 4


def test_one_cell_domain_and_constant():
    Hc = prep.initial_corners(np.array([[17.0]]))
    np.testing.assert_array_equal(Hc, np.full((2, 2), 17.0))
    Hc, misfit, _ = prep.reconstruct_bathymetry(np.full((4, 5), 250.0), n_iter=3)
    np.testing.assert_allclose(Hc, 250.0, atol=1e-12)


def test_iteration_fits_a_rough_field():
    rng = np.random.default_rng(3)
    ny, nx = 48, 64
    k = np.fft.fftfreq(ny)[:, None] ** 2 + np.fft.fftfreq(nx)[None, :] ** 2
    spec = (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))) / np.maximum(k, 1e-3) ** 1.2
    Hm = 500.0 + 200.0 * np.real(np.fft.ifft2(spec)) / np.abs(np.real(np.fft.ifft2(spec))).max()
    H0 = prep.initial_corners(Hm)
    r0 = Hm - prep.midpoints(H0)
    Hc, misfit, change = prep.reconstruct_bathymetry(Hm, n_iter=10)
    r = Hm - prep.midpoints(Hc)
    # the cell means move towards the targets (the smoothing stage keeps the
    # fit from being exact on a field this rough), and the corner updates
    # die out within the ten iterations the paper finds sufficient
    assert np.sqrt((r ** 2).mean()) < 0.7 * np.sqrt((r0 ** 2).mean())
    assert misfit[-1] < np.abs(r0).max()
    assert change[-1] < 0.05 * change[0]
    assert all(b <= a * 1.0001 for a, b in zip(change[1:], change[2:]))


def test_land_corner_encoding_brute_force():
    rng = np.random.default_rng(5)
    land = rng.random((6, 7)) < 0.5
    Hc = prep.land_corners(np.full((7, 8), 10.0), land)
    for J in range(7):
        for I in range(8):
            adj = [land[j, i] for j in (J - 1, J) for i in (I - 1, I) if 0 <= j < 6 and 0 <= i < 7]
            assert (Hc[J, I] == prep.LAND) == all(adj)
    # and the land flag read back from the corners is "any corner LAND"
    back = prep.land_from_corners(Hc)
    for j in range(6):
        for i in range(7):
            assert back[j, i] == any(Hc[J, I] == prep.LAND for J in (j, j + 1) for I in (i, i + 1))


def test_erosion_matches_scipy_morphology():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(11)
    land = rng.random((20, 30)) < 0.55
    eta = rng.standard_normal((20, 30))
    Hm = rng.uniform(5, 300, (20, 30))
    stays, eta2, H2, opened = prep.erode_land(land, eta, Hm, land_depth=5.0)
    cross = ndi.generate_binary_structure(2, 1)
    ref = ndi.binary_erosion(land, structure=cross, border_value=1)
    np.testing.assert_array_equal(stays, ref)
    np.testing.assert_array_equal(opened, land & ~ref)
    dil = ndi.grey_dilation(np.where(land, -np.inf, eta), footprint=cross, mode="constant", cval=-np.inf)
    np.testing.assert_array_equal(eta2[opened], dil[opened])
    np.testing.assert_array_equal(eta2[~opened], eta[~opened])
    assert np.all(H2[opened] == 5.0) and np.array_equal(H2[~opened], Hm[~opened])


def test_erosion_opens_a_one_cell_strait_and_thins_a_block():
    land = np.zeros((7, 9), dtype=bool)
    land[:, 4] = True                       # a wall of land one cell thick...
    land[3, 4] = False                      # ...with a one-cell strait
    land[0:3, 0:3] = True                   # a 3x3 block in a corner
    stays, *_ = prep.erode_land(land, np.zeros((7, 9)), np.ones((7, 9)))
    assert not stays[:, 4].any()            # the thin wall is gone
    # the block touches the domain edge, which counts as land: only its
    # cells with a water 4-neighbour open
    exp = np.zeros((7, 9), dtype=bool)
    exp[0:2, 0:2] = True
    np.testing.assert_array_equal(stays, exp)


def _coastal_like(nx, ny, seed):
    rng = np.random.default_rng(seed)
    land = np.zeros((ny, nx), dtype=bool)
    land[rng.integers(1, ny - 2):, rng.integers(nx // 2, nx - 2):] = True   # a 2x2-openable block
    Hc = prep.land_corners(rng.uniform(5.0, 200.0, (ny + 1, nx + 1)), land)
    L = prep.land_from_corners(Hc)
    q = [np.where(L, 0.0, rng.standard_normal((ny, nx))) for _ in range(3)]
    return q, Hc, L


def test_coarsening_undoes_refinement():
    q, Hc, L = _coastal_like(11, 9, 2)
    fe, fu, fv, Fc = prep.refine2(*q, Hc)
    assert fe.shape == (18, 22) and Fc.shape == (19, 23)
    ce, cu, cv, Cc = prep.coarsen2(fe, fu, fv, Fc)
    np.testing.assert_array_equal(Cc, Hc)                  # sampling: exact
    for a, b in zip((ce, cu, cv), q):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
    # children of a land cell are land, children of a water cell are water
    FL = prep.land_from_corners(Fc)
    np.testing.assert_array_equal(FL, np.kron(L, np.ones((2, 2), dtype=bool)))


def test_refinement_of_a_linear_state_and_bilinear_bathymetry_is_exact():
    nx, ny = 10, 8
    eta = _lin_cells(nx, ny, 0.3, 0.02, -0.01)
    Hc = _lin_corners(nx, ny, 50.0, 1.0, 2.0, 0.25)
    fe, fu, fv, Fc = prep.refine2(eta, eta, eta, Hc)
    # fine cells of width 1/2: centres at (k + 1/2)/2
    xf = (np.arange(2 * nx) + 0.5) / 2
    yf = (np.arange(2 * ny) + 0.5) / 2
    ref = 0.3 + 0.02 * xf[None, :] - 0.01 * yf[:, None]
    inner = (slice(2, -2), slice(2, -2))      # the edge cells are first order by reading
    np.testing.assert_allclose(fe[inner], ref[inner], rtol=0, atol=1e-14)
    Xf = np.arange(2 * nx + 1) / 2
    Yf = np.arange(2 * ny + 1) / 2
    np.testing.assert_allclose(Fc, 50.0 + Xf[None, :] + 2.0 * Yf[:, None] + 0.25 * Yf[:, None] * Xf[None, :],
                               rtol=0, atol=1e-12)
