"""The oracle's time step on a decomposed domain (test infrastructure: only
tests and the bench's CPU legs may import the oracle).

Each RK stage of the scheme (Section 3: reconstruction from a cell and its
two neighbours on each side, fluxes across the faces between them, the
semi-implicit update of eq:rk2_semiimp) reads two cells along x and along
y. So a sub-domain that holds its own cells plus a two-cell halo of its
neighbours' cells, refreshed after every stage, updates its own cells with
exactly the values the whole domain would use; and the CFL maximum of
eq:cfl over the whole domain is the maximum of the sub-domains' maxima (an
exact reduction). One step of the decomposed oracle is:

1. dt = courant / 4 / (the largest cell speed of any sub-domain);
2. stage 1 on every sub-domain, then the halo exchange of Q*;
3. stage 2 and the flow relaxation (eq:frs) on every sub-domain, then the
   halo exchange of Q^{n+1}.

The stage arithmetic is written out here with numpy from the oracle's
right-hand side (``Oracle.rhs``: fluxes, bed slope, Coriolis, wind, drag
rate at one time) and relaxation (``Oracle.frs``), in the order of the
whole-domain step of ``swe_oracle.c``; run on a single part it is the
whole-domain step. The exchange is a callable, so the same sub-domain code
runs with all parts in one process (``local_exchange``) or one part per
process with messages between them (the gloo test).
"""
from __future__ import annotations

import numpy as np

from paper_1912_02457_gb300 import synth
from oracle import Oracle


class SubOracle:
    """One window of a ``synth.partition`` of a workload, stepped by the
    oracle in FP64. ``Q`` holds (eta, hu, hv) over the window; the halo
    cells are valid after every exchange."""

    def __init__(self, wl, part):
        self.part = part
        self.win = synth.window(wl, part)
        x0, _, y0, _ = part["win"]
        self.orc = Oracle(self.win, offset=(x0, y0), whole=(wl.nx, wl.ny))
        self.Q = [np.array(a, dtype=np.float64) for a in (self.win.eta, self.win.hu, self.win.hv)]
        self.qs = None
        self.land = self.win.land_cells()

    def max_speed(self):
        """eq:cfl's largest cell speed over the window (own and halo cells:
        all of them hold current values of the whole domain)."""
        return self.orc.max_speed(*self.Q)

    def stage1(self, t, dt):
        """Q* = (Q^n + dt M(Q^n)) / (1 + dt S(Q^n)), S on the momenta only."""
        M, S = self.orc.rhs(*self.Q, t=t)
        eta, hu, hv = self.Q
        self.qs = [eta + dt * M[0],
                   (hu + dt * M[1]) / (1.0 + dt * S),
                   (hv + dt * M[2]) / (1.0 + dt * S)]

    def stage2(self, t, dt):
        """Q^{n+1} = (Q^n + Q* + dt M(Q*)) / 2 / (1 + dt S(Q*) / 2) on water
        cells, then the flow relaxation at t + dt."""
        M, S = self.orc.rhs(*self.qs, t=t + dt)
        eta, hu, hv = self.Q
        qe, qu, qv = self.qs
        ne = 0.5 * (eta + qe + dt * M[0])
        nu = 0.5 * (hu + qu + dt * M[1]) / (1.0 + 0.5 * dt * S)
        nv = 0.5 * (hv + qv + dt * M[2]) / (1.0 + 0.5 * dt * S)
        self.Q = [np.ascontiguousarray(np.where(self.land, old, new))
                  for old, new in ((eta, ne), (hu, nu), (hv, nv))]
        self.orc.frs(*self.Q, t + dt)

    def fields(self, which):
        return self.qs if which == "qs" else self.Q

    def own_slices(self):
        """(rows, cols) of the owned cells within the window."""
        x0, x1, y0, y1 = self.part["own"]
        wx0, _, wy0, _ = self.part["win"]
        return slice(y0 - wy0, y1 - wy0), slice(x0 - wx0, x1 - wx0)


def local_exchange(subs, which, nx, ny):
    """Refresh every window's halo cells from the sub-domains that own
    them (all parts in this process)."""
    whole = [np.full((ny, nx), np.nan) for _ in range(3)]
    for s in subs:
        x0, x1, y0, y1 = s.part["own"]
        r, c = s.own_slices()
        for a, w in zip(s.fields(which), whole):
            w[y0:y1, x0:x1] = a[r, c]
    for s in subs:
        x0, x1, y0, y1 = s.part["win"]
        for a, w in zip(s.fields(which), whole):
            a[...] = w[y0:y1, x0:x1]


def step(subs, n, t, courant, exchange, reduce_max=lambda v: v, t_end=0.0):
    """n steps of the decomposed scheme from time t; ``exchange(subs,
    which)`` refreshes the halos of ``which`` ("qs" after stage 1, "Q"
    after stage 2), ``reduce_max`` combines a local maximum over all
    processes. t_end > 0: a forecast horizon, as in the oracle's run (the
    step that would pass it ends on it, steps past it are no-ops). Returns
    (t, dt of the last step taken)."""
    dt = 0.0
    for _ in range(n):
        if t_end > 0.0 and t >= t_end * (1.0 - 1e-14):
            continue
        speed = reduce_max(max(s.max_speed() for s in subs))
        dt = courant * 0.25 / speed
        if t_end > 0.0 and t + dt > t_end:
            dt = t_end - t
        for s in subs:
            s.stage1(t, dt)
        exchange(subs, "qs")
        for s in subs:
            s.stage2(t, dt)
        exchange(subs, "Q")
        t += dt
    return t, dt


def run_split(wl, px, py, n, t_end=0.0):
    """n steps of ``wl`` split into px x py sub-domains in one process;
    returns the assembled (eta, hu, hv) and (t, dt)."""
    parts = synth.partition(wl.nx, wl.ny, px, py)
    subs = [SubOracle(wl, p) for p in parts]
    t, dt = step(subs, n, wl.t0, wl.params.courant,
                 lambda ss, w: local_exchange(ss, w, wl.nx, wl.ny), t_end=t_end)
    out = [np.zeros((wl.ny, wl.nx)) for _ in range(3)]
    for s in subs:
        x0, x1, y0, y1 = s.part["own"]
        r, c = s.own_slices()
        for a, o in zip(s.Q, out):
            o[y0:y1, x0:x1] = a[r, c]
    return out, (t, dt)
