"""Test-only workload builders and transforms (no scheme arithmetic)."""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_1912_02457_gb300 import synth


def flat(nx, ny, depth=100.0, dx=800.0, dy=800.0, f=0.0, theta=0.0, dtype=np.float64,
         bc=(synth.BC_WALL,) * 4, **params):
    z = np.zeros((ny, nx), dtype=dtype)
    H = np.full((ny + 1, nx + 1), depth, dtype=dtype)
    return synth.Workload(name=f"flat{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dy,
                          eta=z.copy(), hu=z.copy(), hv=z.copy(), H=H,
                          f=np.full((ny, nx), f, dtype=dtype),
                          theta=np.full((ny, nx), theta, dtype=dtype),
                          bc=tuple(bc), params=synth.Params(**params))


def rough(nx, ny, seed=0, land=True, min_depth=None, dtype=np.float64, **kw):
    """Small coastal-like domain: random bathymetry, land, varying f and theta,
    walls on all sides (no forcing), for invariance tests."""
    wl = synth.coastal(nx, ny, seed_config=90, member=seed,
                       land_frac=0.3 if land else 0.0, dtype=np.float64)
    wl.bc = (synth.BC_WALL,) * 4
    wl.wind = None
    wl.boundary = None
    wl.params = synth.Params(**kw)
    rng = np.random.default_rng(seed)
    wl.f = (1.2e-4 + 2e-5 * rng.standard_normal((ny, nx)))
    wl.theta = rng.uniform(-0.5, 0.5, (ny, nx))
    if min_depth is not None:
        Lm = wl.H == synth.LAND
        wl.H = np.where(Lm, wl.H, np.maximum(wl.H, min_depth))
        wl.eta = np.zeros((ny, nx))
    if not land:
        wl.H = np.where(wl.H == synth.LAND, 50.0, wl.H)
    return wl.astype(dtype)


def random_state(wl, seed=1, amp=0.3, mom=0.5):
    rng = np.random.default_rng(seed)
    ny, nx = wl.ny, wl.nx
    land = wl.land_cells()
    e = np.where(land, 0.0, amp * rng.standard_normal((ny, nx)))
    u = np.where(land, 0.0, mom * rng.standard_normal((ny, nx)))
    v = np.where(land, 0.0, mom * rng.standard_normal((ny, nx)))
    return e, u, v


# ---- symmetry transforms (state triples and workloads) -----------------------

def flip_x_state(e, u, v):
    return e[:, ::-1], -u[:, ::-1], v[:, ::-1]


def flip_y_state(e, u, v):
    return e[::-1, :], u[::-1, :], -v[::-1, :]


def transpose_state(e, u, v):
    return e.T, v.T, u.T


def rot180_state(e, u, v):
    return e[::-1, ::-1], -u[::-1, ::-1], -v[::-1, ::-1]


def _wl_with(wl, **kw):
    c = wl.copy()
    for k, val in kw.items():
        setattr(c, k, val)
    return c


def flip_x(wl):
    S, N, W, E = wl.bc
    return _wl_with(wl, H=wl.H[:, ::-1].copy(), f=-wl.f[:, ::-1].copy(),
                    theta=-wl.theta[:, ::-1].copy(), bc=(S, N, E, W))


def flip_y(wl):
    S, N, W, E = wl.bc
    return _wl_with(wl, H=wl.H[::-1, :].copy(), f=-wl.f[::-1, :].copy(),
                    theta=(np.pi - wl.theta[::-1, :]).copy(), bc=(N, S, W, E))


def transpose(wl):
    S, N, W, E = wl.bc
    return _wl_with(wl, nx=wl.ny, ny=wl.nx, dx=wl.dy, dy=wl.dx, H=wl.H.T.copy(),
                    f=-wl.f.T.copy(), theta=(np.pi / 2 - wl.theta.T).copy(),
                    bc=(W, E, S, N))


def rot180(wl):
    S, N, W, E = wl.bc
    return _wl_with(wl, H=wl.H[::-1, ::-1].copy(), f=wl.f[::-1, ::-1].copy(),
                    theta=(wl.theta[::-1, ::-1] + np.pi).copy(), bc=(N, S, E, W))


def land_ring(wl, r=2):
    """Embed a walled domain in an r-cell ring of land (corners of the ring
    become LAND), keeping the domain's own walls outside the ring."""
    nx, ny = wl.nx + 2 * r, wl.ny + 2 * r
    H = np.full((ny + 1, nx + 1), synth.LAND, dtype=wl.H.dtype)
    H[r:r + wl.ny + 1, r:r + wl.nx + 1] = wl.H

    def pad(a, val=0.0):
        out = np.full((ny, nx), val, dtype=a.dtype)
        out[r:r + wl.ny, r:r + wl.nx] = a
        return out

    return _wl_with(wl, nx=nx, ny=ny, H=H, eta=pad(wl.eta), hu=pad(wl.hu), hv=pad(wl.hv),
                    f=pad(wl.f, 1e-4), theta=pad(wl.theta))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = max(np.abs(a).max(), np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / s)


def max_filter(a, r):
    """(2r+1)^2 maximum filter (periodic at the edges, fine for masks that
    stay away from them)."""
    out = a.copy()
    for dj in range(-r, r + 1):
        for di in range(-r, r + 1):
            out = np.maximum(out, np.roll(np.roll(a, dj, axis=0), di, axis=1))
    return out


def ulp_perturbed(wl, seed=1):
    """The workload with eta and the wet corner depths moved by one float32
    ulp in random directions (FP64 values)."""
    from paper_1912_02457_gb300 import synth
    rng = np.random.default_rng(seed)
    w2 = wl.copy()
    w2.eta = wl.eta.astype(np.float64) * (1 + 6e-8 * rng.choice([-1, 1], wl.eta.shape))
    Hm = wl.H.astype(np.float64)
    w2.H = np.where(wl.H == synth.LAND, Hm, Hm * (1 + 6e-8 * rng.choice([-1, 1], Hm.shape)))
    return w2.astype(np.float64)


def front_set(wl, eta_end, depth=0.01, radius=3):
    """Wet cells dry (hbar <= depth) at the start or at the end, dilated."""
    from paper_1912_02457_gb300 import synth
    Hm = np.where(wl.H == synth.LAND, np.nan, wl.H.astype(np.float64))
    Hbar = 0.25 * (Hm[:-1, :-1] + Hm[1:, :-1] + Hm[:-1, 1:] + Hm[1:, 1:])
    land = wl.land_cells()
    dry = (((wl.eta.astype(np.float64) + Hbar) <= depth) | ((eta_end + Hbar) <= depth)) & ~land
    return max_filter(dry.astype(np.int8), radius).astype(bool) & ~land


def periodic_rough(nx, ny, seed=0, land=False, periodic=(True, True), dtype=np.float64):
    """Rough domain for periodic boundaries: a periodic random bathymetry
    (its last corner row / column repeats the first along each periodic
    axis), optional land blobs, varying f and north angle; walls on the
    non-periodic axes. No forcing."""
    from paper_1912_02457_gb300 import synth
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(ny)[:, None] ** 2 + np.fft.fftfreq(nx)[None, :] ** 2
    spec = (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))) / np.maximum(k, 2e-3) ** 1.0
    z = np.real(np.fft.ifft2(spec))
    z = (z - z.min()) / (z.max() - z.min())
    Hc = np.empty((ny + 1, nx + 1))
    Hc[:ny, :nx] = 20.0 + 200.0 * z
    Hc[ny, :nx] = Hc[0, :nx] if periodic[1] else Hc[ny - 1, :nx]
    Hc[:, nx] = Hc[:, 0] if periodic[0] else Hc[:, nx - 1]
    if land:
        lm = np.zeros((ny, nx), dtype=bool)
        lm[ny // 3: ny // 3 + 4, nx // 4: nx // 4 + 5] = True
        lm[-3:, -4:] = True                      # touches the seams
        lm = synth.open_mask_2x2(lm)
        Hc = synth.encode_land(Hc, lm)
        if periodic[0]:
            Hc[:, nx] = Hc[:, 0]
        if periodic[1]:
            Hc[ny, :] = Hc[0, :]
    f = 1.0e-4 + 2e-5 * rng.standard_normal((ny, nx))
    th = rng.uniform(-0.5, 0.5, (ny, nx))
    bc = (synth.BC_PERIODIC if periodic[1] else synth.BC_WALL,) * 2 + \
         (synth.BC_PERIODIC if periodic[0] else synth.BC_WALL,) * 2
    z0 = np.zeros((ny, nx))
    wl = synth.Workload(name=f"periodic{nx}x{ny}", nx=nx, ny=ny, dx=1000.0, dy=1000.0,
                        eta=z0.copy(), hu=z0.copy(), hv=z0.copy(), H=Hc, f=f, theta=th,
                        bc=bc, params=synth.Params())
    return wl.astype(dtype)


def gridded_wind(nfx, nfy, hours=3, seed=0, speed=10.0):
    """Hourly wind frames on a coarse nfx x nfy grid (grid axes, m/s): a
    smooth field that turns and strengthens across the grid and changes
    from hour to hour, speeds of roughly 4-16 m/s (both branches of the
    Large & Pond drag law)."""
    rng = np.random.default_rng(seed)
    n = hours + 1
    X = (np.arange(nfx) + 0.5) / nfx
    Y = (np.arange(nfy) + 0.5) / nfy
    fr = np.zeros((n, nfy, nfx, 2), dtype=np.float32)
    for q in range(n):
        a = rng.uniform(-0.6, 0.6)
        ang = a + 1.2 * X[None, :] - 0.8 * Y[:, None]
        sp = speed * (1.0 + 0.5 * np.sin(2.0 * np.pi * (X[None, :] + 0.7 * Y[:, None] + 0.3 * q)))
        fr[q, :, :, 0] = sp * np.cos(ang)
        fr[q, :, :, 1] = sp * np.sin(ang)
    return synth.Forcing(times=3600.0 * np.arange(n, dtype=np.float64), frames=fr, nfx=nfx, nfy=nfy)
