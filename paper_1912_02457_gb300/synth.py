"""Seeded synthetic workloads for the rotating shallow-water scheme.

This module only *builds inputs*: corner bathymetry with its land no-data
value, Coriolis and north-angle planes, initial states and forcing frames.
It holds none of the finite-volume scheme's arithmetic. Both the CUDA path
and the FP64 CPU oracle consume the ``Workload`` objects made here, so the
two sides see bit-identical inputs.

The paper's own workloads (NorKyst-800 sections, the "peaks" convergence
benchmark of Section 4.1) are stood in for by the generators below; the
recipe of each is in its docstring.

Layouts (all row-major, x fastest):

* cell planes ``eta, hu, hv, f, theta``: shape ``(ny, nx)``;
* corner bathymetry ``H``: shape ``(ny+1, nx+1)``, equilibrium depth in m
  (positive below the reference level); ``LAND`` marks a corner whose
  adjacent in-domain cells are all land (Section 3.4: the mask is a unique
  no-data value in the bathymetry);
* wind frames: ``(n_frames, nfy, nfx, 2)`` float32 wind at 10 m in grid axes,
  times in seconds (float64);
* boundary frames: ``(n_frames, 12*(nbx+nby))`` float32, per frame the edges
  S, N (length ``nbx``) then W, E (length ``nby``), each edge stored as
  ``[ghost row r][variable v][k]`` with r = 0 the ghost row touching the
  domain, r = 1 the outer one, v in (eta, hu, hv).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

LAND = float(np.finfo(np.float32).max)

BC_WALL = 0
BC_NESTED = 1
BC_PERIODIC = 2      # opposite edges pair up; the corner plane's last line repeats its first
EDGES = ("S", "N", "W", "E")

OMEGA = 7.2921e-5   # Earth's rotation rate (Section 3.7)
M2_PERIOD = 44712.0  # 12.42 h


@dataclasses.dataclass
class Params:
    g: float = 9.81
    theta_mm: float = 1.3        # generalised-minmod parameter
    kappa: float = 1e-2          # desingularisation depth (m)
    cd: float = 0.0              # quadratic bottom-drag coefficient
    courant: float = 0.8
    frs_d0: float = 2.5          # flow-relaxation fall-off (cells)
    frs_width: int = 10          # flow-relaxation zone width (cells)
    dt_update_every: int = 1     # recompute dt every k steps
    dt_fixed: float = 0.0        # > 0: fixed time step
    rho_air: float = 1.225
    rho_water: float = 1025.0
    cfl_faces: int = 0           # 1: time step from the faces' one-sided speeds


@dataclasses.dataclass
class Forcing:
    times: np.ndarray            # float64 (n_frames,)
    frames: np.ndarray           # float32, layout per module docstring
    nfx: int                     # wind: grid width;  boundary: nbx
    nfy: int                     # wind: grid height; boundary: nby


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    eta: np.ndarray
    hu: np.ndarray
    hv: np.ndarray
    H: np.ndarray
    f: Optional[np.ndarray]
    theta: Optional[np.ndarray]
    bc: tuple
    params: Params
    f_const: float = 0.0
    theta_const: float = 0.0
    wind: Optional[Forcing] = None
    boundary: Optional[Forcing] = None
    t0: float = 0.0
    horizon: float = 0.0         # simulated seconds the workload asks for
    steps: int = 0               # steps the workload asks for (0: horizon)

    @property
    def dtype(self):
        return self.eta.dtype

    def copy(self) -> "Workload":
        c = dataclasses.replace(self)
        for k in ("eta", "hu", "hv", "H", "f", "theta"):
            v = getattr(self, k)
            if v is not None:
                setattr(c, k, v.copy())
        c.params = dataclasses.replace(self.params)
        return c

    def astype(self, dtype) -> "Workload":
        c = self.copy()
        for k in ("eta", "hu", "hv", "H", "f", "theta"):
            v = getattr(c, k)
            if v is not None:
                setattr(c, k, np.ascontiguousarray(v, dtype=dtype))
        return c

    def land_cells(self) -> np.ndarray:
        """Cells flagged as land by the corner encoding (any corner is LAND)."""
        L = self.H == np.asarray(LAND, dtype=self.H.dtype)
        return L[:-1, :-1] | L[1:, :-1] | L[:-1, 1:] | L[1:, 1:]


def rng_for(config: int, member: int = 0) -> np.random.Generator:
    """The seed recipe: 1912_02457 + 1000*config + member, PCG64."""
    return np.random.Generator(np.random.PCG64(1912_02457 + 1000 * config + member))


# --------------------------------------------------------------------------
# land encoding helpers (input format, not scheme arithmetic)
# --------------------------------------------------------------------------

def open_mask_2x2(land: np.ndarray) -> np.ndarray:
    """2x2 morphological opening: keep only land cells covered by an all-land
    2x2 block, so that the corner encoding below round-trips exactly."""
    ny, nx = land.shape
    blk = land[:-1, :-1] & land[1:, :-1] & land[:-1, 1:] & land[1:, 1:]
    out = np.zeros_like(land)
    out[:-1, :-1] |= blk
    out[1:, :-1] |= blk
    out[:-1, 1:] |= blk
    out[1:, 1:] |= blk
    return out


def corner_land(land: np.ndarray) -> np.ndarray:
    """A corner is LAND iff every in-domain cell touching it is land."""
    ny, nx = land.shape
    pad = np.ones((ny + 2, nx + 2), dtype=bool)   # outside counts as land
    pad[1:-1, 1:-1] = land
    return pad[:-1, :-1] & pad[1:, :-1] & pad[:-1, 1:] & pad[1:, 1:]


def encode_land(H: np.ndarray, land: np.ndarray) -> np.ndarray:
    """Write LAND into the corners of H that the (opened) mask makes land."""
    land = open_mask_2x2(land)
    cl = corner_land(land)
    H = H.copy()
    H[cl] = LAND
    return H


# --------------------------------------------------------------------------
# random fields
# --------------------------------------------------------------------------

def spectral_field(rng: np.random.Generator, ny: int, nx: int,
                   slope: float = -3.0, max_fft: int = 2049) -> np.ndarray:
    """Gaussian random field with isotropic power ~ |k|^slope, unit std.

    Fields larger than ``max_fft`` points per side are synthesised at that
    size and bilinearly upsampled (a slope of -3 puts almost all variance at
    the largest scales, so nothing visible is lost)."""
    gy, gx = min(ny, max_fft), min(nx, max_fft)
    w = rng.standard_normal((gy, gx))
    W = np.fft.rfft2(w)
    ky = np.fft.fftfreq(gy)[:, None]
    kx = np.fft.rfftfreq(gx)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    k[0, 0] = np.inf
    W *= k ** (slope / 2.0)
    z = np.fft.irfft2(W, s=(gy, gx))
    z = (z - z.mean()) / z.std()
    if (gy, gx) != (ny, nx):
        yi = np.linspace(0, gy - 1, ny)
        xi = np.linspace(0, gx - 1, nx)
        z = np.stack([np.interp(xi, np.arange(gx), row) for row in z])
        z = np.stack([np.interp(yi, np.arange(gy), col) for col in z.T]).T
    return z


# --------------------------------------------------------------------------
# forcing builders
# --------------------------------------------------------------------------

def uniform_wind(wx: float, wy: float, t_end: float = 1e7) -> Forcing:
    fr = np.array([[[[wx, wy]]], [[[wx, wy]]]], dtype=np.float32)
    return Forcing(times=np.array([0.0, t_end]), frames=fr, nfx=1, nfy=1)


def boundary_layout(nbx: int, nby: int):
    """Offsets of each edge's block inside one boundary frame."""
    sizes = (6 * nbx, 6 * nbx, 6 * nby, 6 * nby)
    offs = np.cumsum((0,) + sizes[:-1])
    return dict(zip(EDGES, zip(offs, sizes)))


def still_boundary(nx: int, ny: int, eta: float = 0.0,
                   times=(0.0, 1e7)) -> Forcing:
    n = len(times)
    fr = np.zeros((n, 12 * (nx + ny)), dtype=np.float32)
    lay = boundary_layout(nx, ny)
    for e, (o, s) in lay.items():
        nb = nx if e in "SN" else ny
        blk = fr[:, o:o + s].reshape(n, 2, 3, nb)
        blk[:, :, 0, :] = eta
    return Forcing(times=np.asarray(times, dtype=np.float64), frames=fr,
                   nfx=nx, nfy=ny)


def tide_boundary(nx: int, ny: int, dx: float, dy: float, H_edge: dict,
                  amp: float = 0.5, hours: int = 25, nb_div: int = 2,
                  phase0: float = 0.0, g: float = 9.81,
                  eta_floor: Optional[dict] = None) -> Forcing:
    """Hourly M2 frames: eta = amp*sin(2 pi t / T + phi), phi = 2 pi s / L.

    s is the along-boundary coordinate of the ghost-cell centre (x + y, m),
    L = T sqrt(g Hbar_edge) the tidal wavelength over the edge's mean depth;
    hu = hv = 0 in the frames. Frames are stored at 1/nb_div of the domain's
    resolution along each edge (a coarser parent model). ``eta_floor`` maps
    an edge to the lowest level each of its samples may take (an external
    model keeps dry land dry: its level never lies below the bed it
    covers)."""
    nbx, nby = max(nx // nb_div, 1), max(ny // nb_div, 1)
    times = 3600.0 * np.arange(hours + 1, dtype=np.float64)
    fr = np.zeros((len(times), 12 * (nbx + nby)), dtype=np.float32)
    lay = boundary_layout(nbx, nby)
    for e, (o, s) in lay.items():
        nb = nbx if e in "SN" else nby
        L = M2_PERIOD * math.sqrt(g * max(H_edge.get(e, 100.0), 1.0))
        blk = fr[:, o:o + s].reshape(len(times), 2, 3, nb)
        for r in range(2):
            # ghost-cell centres along the edge, in metres
            k = (np.arange(nb) + 0.5) / nb
            if e == "S":
                xs, ys = k * nx * dx, -(r + 0.5) * dy
            elif e == "N":
                xs, ys = k * nx * dx, (ny + r + 0.5) * dy
            elif e == "W":
                xs, ys = -(r + 0.5) * dx, k * ny * dy
            else:
                xs, ys = (nx + r + 0.5) * dx, k * ny * dy
            phi = 2 * np.pi * (xs + ys) / L + phase0
            eta = amp * np.sin(2 * np.pi * times[:, None] / M2_PERIOD + phi[None, :])
            if eta_floor is not None and e in eta_floor:
                eta = np.maximum(eta, eta_floor[e][None, :])
            blk[:, r, 0, :] = eta.astype(np.float32)
    return Forcing(times=times, frames=fr, nfx=nbx, nfy=nby)


def edge_sample_floor(Hbar: np.ndarray, land: np.ndarray, zone: int, nb_div: int = 2) -> dict:
    """The lowest external level each boundary sample of the S, N and W
    edges may take so that no cell it reaches lies below the bed. A cell
    filled from an edge (the ghost rings copy the statics of the first two
    rows) or relaxed toward it (the zone of ``zone`` rows) takes the edge's
    level interpolated linearly between the two nearest samples at the
    cell's position along the edge. Each sample is raised to at least -Hbar
    of every wet zone cell whose interpolation uses it, so every
    interpolated level covers the bed (a convex combination of levels that
    do). Plain data preparation, no step of the scheme."""
    out = {}
    for e in ("S", "N", "W"):
        if e == "S":
            hb, lm = Hbar[:zone, :].T, land[:zone, :].T
        elif e == "N":
            hb, lm = Hbar[::-1][:zone, :].T, land[::-1][:zone, :].T
        else:
            hb, lm = Hbar[:, :zone], land[:, :zone]
        need = np.where(lm, -np.inf, -hb).max(axis=1)   # per cell along the edge
        n = need.shape[0]
        nb = max(n // nb_div, 1)
        p = np.clip((np.arange(n) + 0.5) * nb / n - 0.5, 0.0, nb - 1)
        k0 = np.floor(p).astype(int)
        k1 = np.minimum(k0 + 1, nb - 1)
        floor = np.full(nb, -np.inf)
        np.maximum.at(floor, k0, need)
        np.maximum.at(floor, k1, need)
        out[e] = floor
    return out


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def partition(nx: int, ny: int, px: int, py: int, halo: int = 2) -> list:
    """Split an nx x ny domain into px x py sub-domains for a halo-exchange
    decomposition (each RK stage of the scheme reads two cells along x and
    y, so a sub-domain that holds ``halo`` = 2 cells of each neighbour
    beyond its own cells, refreshed after every stage, updates its own cells
    exactly as the whole domain would). Integer bookkeeping only.

    Returns one dict per sub-domain, row-major (x fastest):
    ``own`` (x0, x1, y0, y1), the owned cells in whole-domain coordinates;
    ``win`` (x0, x1, y0, y1), the window: the owned cells plus ``halo``
    cells on every side with a neighbour; ``cut`` (S, N, W, E), whether a
    neighbour lies beyond that edge of the window; ``rank`` its index.
    Owned extents differ by at most one cell and hold at least ``halo``
    cells each (so a halo comes from the adjacent sub-domain only)."""
    if px < 1 or py < 1 or nx < px * halo or ny < py * halo:
        raise ValueError(f"cannot split {nx}x{ny} into {px}x{py} parts of >= {halo} cells")

    def cuts(n, parts):
        return [n * k // parts for k in range(parts + 1)]

    xs, ys = cuts(nx, px), cuts(ny, py)
    out = []
    for b in range(py):
        for a in range(px):
            x0, x1, y0, y1 = xs[a], xs[a + 1], ys[b], ys[b + 1]
            cut = (b > 0, b < py - 1, a > 0, a < px - 1)
            win = (x0 - halo * cut[2], x1 + halo * cut[3], y0 - halo * cut[0], y1 + halo * cut[1])
            out.append({"own": (x0, x1, y0, y1), "win": win, "cut": cut, "rank": b * px + a})
    return out


def window(wl: Workload, part: dict) -> Workload:
    """The sub-workload of one ``partition`` entry: planes and corner
    bathymetry cut to the window, the edges that face a neighbour turned
    into walls (the cells next to them are halo cells, overwritten by the
    exchange, so what the wall does to them is never used), the whole
    domain's forcing (sampled at the whole domain's positions by the side
    that steps the window)."""
    x0, x1, y0, y1 = part["win"]
    if any(part["cut"]) and any(b == BC_PERIODIC for b in wl.bc):
        raise ValueError("periodic edges are not split")
    c = wl.copy()
    for k in ("eta", "hu", "hv", "f", "theta"):
        v = getattr(wl, k)
        if v is not None:
            setattr(c, k, np.ascontiguousarray(v[y0:y1, x0:x1]))
    c.H = np.ascontiguousarray(wl.H[y0:y1 + 1, x0:x1 + 1])
    c.nx, c.ny = x1 - x0, y1 - y0
    c.bc = tuple(BC_WALL if part["cut"][e] else wl.bc[e] for e in range(4))
    c.name = f"{wl.name}[{x0}:{x1},{y0}:{y1}]"
    return c


def gaussian_bump(dtype=np.float32, n: int = 128, steps: int = 1000) -> Workload:
    """Plain method: n x n cells, dx = dy = 800 m, flat 100 m depth, walls,
    f-plane f = 1.2e-4 1/s, north angle 0, no friction or wind, a 1 m
    Gaussian bump (sigma 10 cells) at the centre, u = v = 0, Courant 0.45."""
    c = n / 2.0
    j, i = np.mgrid[0:n, 0:n]
    r2 = (i + 0.5 - c) ** 2 + (j + 0.5 - c) ** 2
    eta = np.exp(-r2 / (2.0 * 10.0 ** 2)).astype(dtype)
    z = np.zeros((n, n), dtype=dtype)
    H = np.full((n + 1, n + 1), 100.0, dtype=dtype)
    return Workload(name=f"gaussian{n}", nx=n, ny=n, dx=800.0, dy=800.0,
                    eta=eta, hu=z.copy(), hv=z.copy(), H=H, f=None, theta=None,
                    f_const=1.2e-4, theta_const=0.0, bc=(BC_WALL,) * 4,
                    params=Params(courant=0.45), steps=steps)


def coastal(nx: int = 1024, ny: int = 1024, seed_config: int = 2,
            member: int = 0, land_frac: float = 0.30, dtype=np.float32,
            tide_phase: float = 0.0, wind_speed: float = 10.0,
            wind_dir_deg: float = 0.0, hours: int = 24) -> Workload:
    """Synthetic coastal domain (stand-in for a NorKyst-800 section).

    * corner heights: a seeded Gaussian random field with spectral slope -3
      plus an eastward ramp, so land gathers on the east side;
    * land: cells above the (1 - land_frac) quantile, opened 2x2, encoded as
      LAND corners;
    * depth at wet corners: H = -2 + 3002 q^2 with q the normalised height
      below the coast level, giving 0-3000 m with shallow (-2..5 m) shelves
      where wet-dry fronts move;
    * Coriolis from latitude 58-70 N (linear in y), f = 2 omega sin(lat);
      north angle linear in x over 0-0.3 rad;
    * quadratic drag Cd = 0.0025; uniform 10 m/s wind along +x;
    * nested S, N, W edges with hourly M2 tide frames (0.5 m), east wall;
      the frames' level is kept at or above the bed of every cell it fills
      or relaxes (raised shelves reaching the edge stay dry);
    * initial state at rest: eta = max(0, -Hbar) on water, 0 on land.
    """
    rng = rng_for(seed_config, member)
    dx = dy = 800.0
    z = spectral_field(rng, ny + 1, nx + 1)
    xs = np.linspace(-1.0, 1.0, nx + 1)[None, :]
    z = z + 2.2 * xs
    zc = 0.25 * (z[:-1, :-1] + z[1:, :-1] + z[:-1, 1:] + z[1:, 1:])
    thr = np.quantile(zc, 1.0 - land_frac)
    land = zc > thr
    zmin = z.min()
    q = np.clip((thr - z) / (thr - zmin), 0.0, 1.0)
    H = (-2.0 + 3002.0 * q * q)
    H = encode_land(H, land).astype(dtype)
    wl_land = Workload(name="tmp", nx=nx, ny=ny, dx=dx, dy=dy, eta=None, hu=None,
                       hv=None, H=H, f=None, theta=None, bc=(0,) * 4,
                       params=Params()).land_cells()
    Hm = np.where(H == np.asarray(LAND, dtype), 0.0, H.astype(np.float64))
    Hbar = 0.25 * (Hm[:-1, :-1] + Hm[1:, :-1] + Hm[:-1, 1:] + Hm[1:, 1:])
    eta = np.where(wl_land, 0.0, np.maximum(0.0, -Hbar)).astype(dtype)
    zero = np.zeros((ny, nx), dtype=dtype)
    lat = 58.0 + 12.0 * (np.arange(ny) + 0.5) / ny
    f = (2.0 * OMEGA * np.sin(np.deg2rad(lat)))[:, None] * np.ones((1, nx))
    theta = (0.3 * (np.arange(nx) + 0.5) / nx)[None, :] * np.ones((ny, 1))
    # mean wet depth along each nested edge, for the tidal wavelength
    H_edge = {}
    for e, row in (("S", Hbar[0]), ("N", Hbar[-1]), ("W", Hbar[:, 0])):
        wet = row[row > 0]
        H_edge[e] = float(wet.mean()) if wet.size else 100.0
    floor = edge_sample_floor(Hbar, wl_land, Params().frs_width)
    bnd = tide_boundary(nx, ny, dx, dy, H_edge, amp=0.5, hours=hours + 1,
                        phase0=tide_phase, eta_floor=floor)
    wr = math.radians(wind_dir_deg)
    wind = uniform_wind(wind_speed * math.cos(wr), wind_speed * math.sin(wr))
    return Workload(name=f"coastal{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dy,
                    eta=eta, hu=zero.copy(), hv=zero.copy(), H=H,
                    f=f.astype(dtype), theta=theta.astype(dtype),
                    bc=(BC_NESTED, BC_NESTED, BC_NESTED, BC_WALL),
                    params=Params(cd=0.0025, courant=0.8), wind=wind,
                    boundary=bnd, horizon=3600.0 * hours)


def peaks(s, t):
    """MATLAB's peaks surface (Section 4.1)."""
    return (3 * (1 - s) ** 2 * np.exp(-s ** 2 - (t + 1) ** 2)
            - 10 * (s / 5 - s ** 3 - t ** 5) * np.exp(-s ** 2 - t ** 2)
            - 1.0 / 3.0 * np.exp(-(s + 1) ** 2 - t ** 2))


def peaks_convergence(n: int, dtype=np.float64, bump_radius_km: float = 300.0
                      ) -> Workload:
    """Grid-convergence benchmark of Section 4.1 on an n x n grid.

    500 km box, H = 100 + 10 peaks(6x/500 - 3, 6y/500 - 3) at corners (x, y
    in km), cosine bump eta = (1 + cos(pi r / c))/2 for r <= c at cell
    centres, north pole at (3000 km, 3000 km): theta = atan2(3000-x, 3000-y),
    latitude = 90 deg - dist / R_E, f = 2 omega sin(lat); walls; fixed
    dt = 1600/n s (800 s simulated)."""
    L = 500.0
    dxk = L / n
    xc = (np.arange(n + 1) * dxk)[None, :]
    yc = (np.arange(n + 1) * dxk)[:, None]
    H = 100.0 + 10.0 * peaks(6 * xc / L - 3, 6 * yc / L - 3)
    x = ((np.arange(n) + 0.5) * dxk)[None, :]
    y = ((np.arange(n) + 0.5) * dxk)[:, None]
    r = np.sqrt((x - 250.0) ** 2 + (y - 250.0) ** 2)
    c = bump_radius_km
    eta = np.where(r <= c, 0.5 * (1 + np.cos(np.pi * r / c)), 0.0)
    px, py = 3000.0 - x, 3000.0 - y
    theta = np.arctan2(px, py) * np.ones((n, n))
    lat = np.pi / 2 - np.sqrt(px ** 2 + py ** 2) / 6371.0
    f = 2 * OMEGA * np.sin(lat) * np.ones((n, n))
    z = np.zeros((n, n))
    dt = 1600.0 / n
    return Workload(name=f"peaks{n}", nx=n, ny=n, dx=dxk * 1e3, dy=dxk * 1e3,
                    eta=eta.astype(dtype), hu=z.astype(dtype), hv=z.astype(dtype),
                    H=H.astype(dtype), f=f.astype(dtype), theta=theta.astype(dtype),
                    bc=(BC_WALL,) * 4, params=Params(dt_fixed=dt), steps=int(round(800.0 / dt)))


SWEEP_SIZES = ((512, 512), (2048, 2048), (2600, 900), (4096, 4096), (8192, 8192))


def beta_plane_f(nx: int, ny: int, dx: float, dy: float, f_ref: float, beta: float,
                 theta: float, x_ref: float = None, y_ref: float = None) -> np.ndarray:
    """Coriolis parameter of a beta plane (eq:betaplane): f_ref plus beta
    times the distance from (x_ref, y_ref) (default: the domain centre) along
    the north vector n = [sin theta, cos theta]; cell centres at ((i+1/2) dx,
    (j+1/2) dy). An input plane of the workload."""
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    x_ref = nx * dx / 2.0 if x_ref is None else x_ref
    y_ref = ny * dy / 2.0 if y_ref is None else y_ref
    return f_ref + beta * (np.sin(theta) * (x[None, :] - x_ref) + np.cos(theta) * (y[:, None] - y_ref))


def rossby(n: int = 350, dx: float = 20e3, depth: float = 50.0, f_ref: float = 8e-5,
           beta: float = 2e-11, theta: float = 0.0, amp: float = 0.1, radius_cells: float = 10.0,
           dtype=np.float64, days: float = 35.0) -> Workload:
    """Planetary Rossby waves (Section 3.7, the beta-plane experiment): n x n
    cells of dx = 20 km, flat depth 50 m, periodic on every edge, a beta
    plane around the domain centre (f_ref = 8e-5 1/s, the value of ~33 N;
    beta = 2e-11 1/(m s)) along the north angle theta, and a Gaussian bump of
    eta (amplitude `amp`, sigma `radius_cells`) at the centre in geostrophic
    balance with f_ref: hu = -(g h / f) d(eta)/dy, hv = (g h / f) d(eta)/dx."""
    g = 9.81
    c = n / 2.0
    j, i = np.mgrid[0:n, 0:n]
    X = (i + 0.5 - c) * dx
    Y = (j + 0.5 - c) * dx
    R = radius_cells * dx
    eta = amp * np.exp(-(X * X + Y * Y) / (2.0 * R * R))
    detadx = -X / (R * R) * eta
    detady = -Y / (R * R) * eta
    h = depth + eta
    hu = -(g * h / f_ref) * detady
    hv = (g * h / f_ref) * detadx
    H = np.full((n + 1, n + 1), depth)
    f = beta_plane_f(n, n, dx, dx, f_ref, beta, theta)
    wl = Workload(name=f"rossby{n}", nx=n, ny=n, dx=dx, dy=dx,
                  eta=eta.astype(dtype), hu=hu.astype(dtype), hv=hv.astype(dtype),
                  H=H.astype(dtype), f=f.astype(dtype),
                  theta=np.full((n, n), theta).astype(dtype),
                  bc=(BC_PERIODIC,) * 4, params=Params(courant=0.8),
                  horizon=days * 86400.0)
    return wl


def ensemble(n_domains: int = 64, seed_config: int = 4, hours: int = 24):
    """Batched ensemble: domains with sizes drawn uniformly from
    {256^2, 512x384, 1024^2, 2048x1024}, each with its own bathymetry seed,
    tide phase U(0, 2 pi) and wind 10 (1 + U(-0.3, 0.3)) m/s at
    U(-20, 20) degrees. Returns a list of Workloads (FP32)."""
    rng = rng_for(seed_config)
    shapes = ((256, 256), (512, 384), (1024, 1024), (2048, 1024))
    out = []
    for m in range(n_domains):
        nx, ny = shapes[int(rng.integers(0, 4))]
        phase = float(rng.uniform(0, 2 * np.pi))
        ws = 10.0 * (1.0 + float(rng.uniform(-0.3, 0.3)))
        wd = float(rng.uniform(-20.0, 20.0))
        wl = coastal(nx, ny, seed_config=seed_config, member=m + 1,
                     tide_phase=phase, wind_speed=ws, wind_dir_deg=wd, hours=hours)
        wl.name = f"member{m}_{nx}x{ny}"
        out.append(wl)
    return out


def serving_trace(n_requests: int = 256, rate: float = 20.0, seed_config: int = 5,
                  min_side: int = 128, max_side: int = 2048,
                  min_hours: float = 1.0, max_hours: float = 24.0):
    """Poisson arrivals (mean ``rate``/s) of forecast requests with square
    domains log-uniform in side between min_side and max_side (rounded to a
    multiple of 32) and horizons U(min_hours, max_hours) simulated hours.
    Returns a list of dicts (arrival time, side, horizon seconds, member)."""
    rng = rng_for(seed_config)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        side = math.exp(rng.uniform(math.log(min_side), math.log(max_side)))
        side = int(max(32, round(side / 32.0) * 32))
        hrs = float(rng.uniform(min_hours, max_hours))
        out.append(dict(arrival=t, side=side, horizon=3600.0 * hrs, member=r))
    return out
