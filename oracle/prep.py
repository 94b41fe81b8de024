"""FP64 CPU oracle of the grid pre-processing of arXiv 1912.02457 (TEST
INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU baseline may use it; it shares no code with the CUDA
library).

* Corner bathymetry from cell averages (Section 3.8 "Bathymetry",
  eqn:recon_1 - eqn:recon_3 and the correct-and-smooth iteration that
  follows them).
* Land erosion with gray dilation of eta into the opened cells (same
  section, the paragraph on narrow straits).
* Refinement and coarsening by a factor of two (Section 3.9 "Refinement
  and coarsening of grid").

Plain numpy on whole arrays, written step by step in the paper's order.
Where the paper is silent the reading taken is stated at the function.
Arrays are indexed [j, i] (y, x); cell planes are ny x nx, corner planes
(ny+1) x (nx+1), and corner [J, I] sits at the intersection x = I, y = J
(cell (j, i) spans x in [i, i+1], y in [j, j+1]).
"""
from __future__ import annotations

import numpy as np

LAND = float(np.finfo(np.float32).max)     # corner marker of a land cell


def gminmod(a, b, c):
    """Generalised minmod: the smallest of (a, b, c) when all are positive,
    the largest when all are negative, else 0 (Section 3.1)."""
    a, b, c = (np.asarray(v, dtype=np.float64) for v in (a, b, c))
    pos = (a > 0) & (b > 0) & (c > 0)
    neg = (a < 0) & (b < 0) & (c < 0)
    lo = np.minimum(a, np.minimum(b, c))
    hi = np.maximum(a, np.maximum(b, c))
    return np.where(pos, lo, np.where(neg, hi, 0.0))


# ---------------------------------------------------------------------------
# corner bathymetry from cell averages

def _neighbours_extrapolated(H, axis):
    """H shifted by -1 and +1 along `axis`; beyond the domain the neighbour
    is the linear extrapolation 2 H_0 - H_1 (reading: the paper gives no
    boundary rule; extrapolation keeps a linear surface exact up to the
    edge). With a single cell along the axis the neighbours are the cell."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[axis]
    if n == 1:
        return H.copy(), H.copy()
    first = np.take(H, [0], axis=axis)
    second = np.take(H, [1], axis=axis)
    last = np.take(H, [n - 1], axis=axis)
    before = np.take(H, [n - 2], axis=axis)
    lower = np.concatenate([2.0 * first - second, np.take(H, range(0, n - 1), axis=axis)], axis=axis)
    upper = np.concatenate([np.take(H, range(1, n), axis=axis), 2.0 * last - before], axis=axis)
    return lower, upper


def cell_slopes(H, theta=1.3):
    """eqn:recon_1: the gradient [H^x, H^y] of each cell, per cell width.
    Reading: the limited slope of the scheme's reconstruction, the
    generalised minmod of theta x backward, central and theta x forward
    differences."""
    H = np.asarray(H, dtype=np.float64)
    out = []
    for axis in (1, 0):                               # x, then y
        lo, up = _neighbours_extrapolated(H, axis)
        bw = H - lo
        fw = up - H
        out.append(gminmod(theta * bw, 0.5 * (bw + fw), theta * fw))
    return out[0], out[1]


def corners_from_cells(H, Hx, Hy):
    """eqn:recon_2 and eqn:recon_3: every cell evaluates its plane at its
    four corners; each intersection takes the mean of the estimates of the
    cells that meet there (four inside the domain; reading: two on an edge,
    one at a domain corner)."""
    H, Hx, Hy = (np.asarray(a, dtype=np.float64) for a in (H, Hx, Hy))
    ny, nx = H.shape
    total = np.zeros((ny + 1, nx + 1))
    count = np.zeros((ny + 1, nx + 1))
    for sy in (-1, 1):                # corner below (-1) or above (+1) the cell centre
        for sx in (-1, 1):            # corner left (-1) or right (+1) of the cell centre
            est = H + 0.5 * sx * Hx + 0.5 * sy * Hy
            J0 = 0 if sy < 0 else 1
            I0 = 0 if sx < 0 else 1
            total[J0:J0 + ny, I0:I0 + nx] += est
            count[J0:J0 + ny, I0:I0 + nx] += 1.0
    return total / count


def midpoints(Hc):
    """H*(i, j): the bilinear surface of the corners at the cell centres,
    i.e. the mean of the cell's four corners."""
    Hc = np.asarray(Hc, dtype=np.float64)
    return 0.25 * (Hc[:-1, :-1] + Hc[:-1, 1:] + Hc[1:, :-1] + Hc[1:, 1:])


def smooth_corners(Hc, weight):
    """One smoothing pass of the corner surface. Reading (the paper only says
    that H* is smoothed): Hc := (1 - w) Hc + w x (mean of the four
    edge-neighbour corners), a missing neighbour beyond the edge being the
    linear extrapolation 2 Hc - (opposite neighbour); this leaves every
    bilinear surface unchanged."""
    Hc = np.asarray(Hc, dtype=np.float64)
    W, E = _neighbours_extrapolated(Hc, 1)
    S, N = _neighbours_extrapolated(Hc, 0)
    return (1.0 - weight) * Hc + weight * 0.25 * (W + E + S + N)


def initial_corners(Hm, theta=1.3):
    """The initial guess H* (eqn:recon_1 - eqn:recon_3 on the cell averages)."""
    Hx, Hy = cell_slopes(Hm, theta)
    return corners_from_cells(Hm, Hx, Hy)


def reconstruct_bathymetry(Hm, n_iter=10, theta=1.3, smooth=0.125):
    """Corner bathymetry whose cell means approach the averages Hm.

    Each iteration: dH = Hm - H*(i, j); apply eqn:recon_1 - eqn:recon_3 to
    dH and add the corner estimate to H* (the paper's formula adds it; its
    text says "subtract", but dH is target minus estimate, so adding is the
    step towards the target); then smooth H*. Returns the corners and, per
    iteration, the largest midpoint misfit max|Hm - H*(i, j)| and the
    largest change of a corner."""
    Hm = np.asarray(Hm, dtype=np.float64)
    Hc = initial_corners(Hm, theta)
    misfit, change = [], []
    for _ in range(n_iter):
        dH = Hm - midpoints(Hc)
        dHx, dHy = cell_slopes(dH, theta)
        new = smooth_corners(Hc + corners_from_cells(dH, dHx, dHy), smooth)
        change.append(float(np.abs(new - Hc).max()))
        Hc = new
        misfit.append(float(np.abs(Hm - midpoints(Hc)).max()))
    return Hc, misfit, change


def land_corners(Hc, land):
    """Land encoding of the corner plane: an intersection whose adjacent
    cells are all land gets the LAND marker."""
    Hc = np.asarray(Hc, dtype=np.float64).copy()
    land = np.asarray(land, dtype=bool)
    ny, nx = land.shape
    allland = np.ones((ny + 1, nx + 1), dtype=bool)
    for dj in (0, 1):
        for di in (0, 1):
            m = np.zeros((ny + 1, nx + 1), dtype=bool)
            m[dj:dj + ny, di:di + nx] = True
            blk = np.ones((ny + 1, nx + 1), dtype=bool)
            blk[dj:dj + ny, di:di + nx] = land
            allland &= np.where(m, blk, True)
    Hc[allland] = LAND
    return Hc


# ---------------------------------------------------------------------------
# land erosion

def erode_land(land, eta, Hm, land_depth=5.0):
    """One step of the strait widening: binary erosion of the land mask,
    gray dilation of eta into the cells it opens, and the land depth there.

    Readings: the structuring element is the 4-neighbour cross (a land cell
    stays land only if its four neighbours are land); outside the domain
    counts as land, so the domain edge does not erode; an opened cell takes
    the largest eta of its 4-neighbours that were water before the step
    ("maximum of neighbours"), depth `land_depth` (the NorKyst-800 land
    value, 5 m) and zero momentum."""
    land = np.asarray(land, dtype=bool)
    eta = np.asarray(eta, dtype=np.float64)
    Hm = np.asarray(Hm, dtype=np.float64)
    ny, nx = land.shape
    padded = np.ones((ny + 2, nx + 2), dtype=bool)
    padded[1:-1, 1:-1] = land
    stays = (padded[1:-1, 1:-1] & padded[:-2, 1:-1] & padded[2:, 1:-1]
             & padded[1:-1, :-2] & padded[1:-1, 2:])
    opened = land & ~stays
    e = np.full((ny + 2, nx + 2), -np.inf)
    e[1:-1, 1:-1] = np.where(land, -np.inf, eta)
    dil = np.maximum(np.maximum(e[:-2, 1:-1], e[2:, 1:-1]), np.maximum(e[1:-1, :-2], e[1:-1, 2:]))
    eta_out = np.where(opened, dil, eta)
    H_out = np.where(opened, land_depth, Hm)
    return stays, eta_out, H_out, opened


# ---------------------------------------------------------------------------
# refinement and coarsening by two

def _state_slopes(q, land, theta, axis):
    """Limited slope of q along `axis` in cell widths (the scheme's
    generalised minmod). Reading: a neighbour that is land or lies beyond
    the domain contributes a zero difference, which makes the slope zero
    (first order at coasts and edges, as in the scheme)."""
    q = np.asarray(q, dtype=np.float64)
    n = q.shape[axis]
    idx = np.arange(n)
    lo_i = np.clip(idx - 1, 0, n - 1)
    up_i = np.clip(idx + 1, 0, n - 1)
    q_lo = np.take(q, lo_i, axis=axis)
    q_up = np.take(q, up_i, axis=axis)
    l_lo = np.take(land, lo_i, axis=axis)
    l_up = np.take(land, up_i, axis=axis)
    shape = [1, 1]
    shape[axis] = n
    edge_lo = (idx == 0).reshape(shape)
    edge_up = (idx == n - 1).reshape(shape)
    bw = np.where(l_lo | edge_lo, 0.0, q - q_lo)
    fw = np.where(l_up | edge_up, 0.0, q_up - q)
    return gminmod(theta * bw, 0.5 * (bw + fw), theta * fw)


def land_from_corners(Hc):
    Hc = np.asarray(Hc)
    L = Hc == np.asarray(LAND, dtype=Hc.dtype)
    return L[:-1, :-1] | L[:-1, 1:] | L[1:, :-1] | L[1:, 1:]


def refine2(eta, hu, hv, Hc, theta=1.3):
    """Section 3.9: each water cell's slope-limited reconstruction evaluated
    at the centres of its four children (x +- 1/4, y +- 1/4 of the cell);
    the bathymetry surface evaluated at the refined intersections (an even
    intersection is the coarse corner, an edge midpoint the mean of its two
    corners, a cell centre the mean of four; LAND if any of them is LAND).
    Land cells give land children with zero state."""
    Hc = np.asarray(Hc, dtype=np.float64)
    land = land_from_corners(Hc)
    ny, nx = land.shape
    out = []
    for q in (eta, hu, hv):
        q = np.where(land, 0.0, np.asarray(q, dtype=np.float64))
        sx = _state_slopes(q, land, theta, 1)
        sy = _state_slopes(q, land, theta, 0)
        f = np.zeros((2 * ny, 2 * nx))
        for b in (0, 1):
            for a in (0, 1):
                child = q + (a - 0.5) * 0.5 * sx + (b - 0.5) * 0.5 * sy
                f[b::2, a::2] = np.where(land, 0.0, child)
        out.append(f)
    Fc = np.zeros((2 * ny + 1, 2 * nx + 1))
    isl = Hc == LAND
    Fc[::2, ::2] = Hc
    ex = 0.5 * (Hc[:, :-1] + Hc[:, 1:])
    ex[isl[:, :-1] | isl[:, 1:]] = LAND
    Fc[::2, 1::2] = ex
    ey = 0.5 * (Hc[:-1, :] + Hc[1:, :])
    ey[isl[:-1, :] | isl[1:, :]] = LAND
    Fc[1::2, ::2] = ey
    cc = midpoints(Hc)
    cc[land] = LAND
    Fc[1::2, 1::2] = cc
    return out[0], out[1], out[2], Fc


def coarsen2(eta, hu, hv, Hc):
    """Section 3.9: a coarse cell is the average of its four children
    (reading: of its water children; a block of land children gives zero),
    and the coarse intersections are sampled from the even fine ones."""
    Hc = np.asarray(Hc, dtype=np.float64)
    fland = land_from_corners(Hc)
    ny2, nx2 = fland.shape
    assert ny2 % 2 == 0 and nx2 % 2 == 0
    Cc = Hc[::2, ::2].copy()
    cland = land_from_corners(Cc)           # the coarse cell's own land flag
    wet = (~fland).astype(np.float64)
    n_wet = sum(wet[b::2, a::2] for b in (0, 1) for a in (0, 1))
    out = []
    for q in (eta, hu, hv):
        q = np.where(fland, 0.0, np.asarray(q, dtype=np.float64))
        s = sum(q[b::2, a::2] for b in (0, 1) for a in (0, 1))
        out.append(np.where(cland | (n_wet == 0), 0.0, s / np.maximum(n_wet, 1.0)))
    return out[0], out[1], out[2], Cc
