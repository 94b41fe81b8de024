"""Why depths go negative over moving wet-dry fronts, pinned on the oracle
(CPU only).

Section 3.4 adjusts the reconstruction so that every face depth is
non-negative, after Kurganov & Petrova. Their argument that the cell depths
then stay non-negative needs the time step bounded by the one-sided local
speeds a+, a- of the faces (eq:cfl with the factor 1/4 of two dimensions).
The scheme as read here bounds it by the cell-average velocities and depths
of the current state (the reading of eq:cfl that the CUDA path implements).
The two differ wherever a face is nearly dry: its depth is re-sloped to
zero or near it while its momentum keeps the limited slope of hu, so the
desingularised face velocity (eq:desing_ours) reaches 2 |hu_f| / kappa.
On the drying shelves of the coastal recipe the face speeds then exceed the
cell-average bound by a factor of ten to forty, Kurganov & Petrova's
condition fails, and a cell depth goes negative within a few hundred steps.
Bounding the step by the face speeds instead keeps every depth non-negative
on the same case, at the cost of time steps some forty times shorter (the
small time steps Section 3.4 warns of)."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests import helpers

T_END = 300.0


def _shelf_case():
    """A 32 x 32 domain of the coastal recipe (land, shelves 2 m above to
    5 m below the still level, wind, drag, varying f and north angle) with
    walls on every edge, so no nesting data enters."""
    wl = synth.coastal(32, 32, seed_config=95, member=0, dtype=np.float64)
    wl.bc = (synth.BC_WALL,) * 4
    wl.boundary = None
    return wl


def _min_depth(wl, run):
    land = wl.land_cells()
    Hm = np.where(wl.H == synth.LAND, np.nan, wl.H.astype(np.float64))
    Hbar = 0.25 * (Hm[:-1, :-1] + Hm[1:, :-1] + Hm[:-1, 1:] + Hm[1:, 1:])
    worst = np.inf
    for e in run:
        worst = min(worst, float(np.where(land, np.inf, e + Hbar).min()))
    return worst


def _states(o, wl, chunk):
    st, t, dt, step = (wl.eta, wl.hu, wl.hv), 0.0, 0.0, 0
    while t < T_END * (1.0 - 1e-12):
        e, u, v, t, dt = o.run(chunk, state=st, t=t, dt=dt, step0=step, t_end=T_END)
        step += chunk
        st = (e, u, v)
        yield e, u, v, t, step


def test_face_speeds_closed_form(oracle_mod):
    """Uniform flow over a flat bottom with periodic edges: every x-face has
    the one-sided speed |u| + sqrt(g H), every y-face |v| + sqrt(g H), the
    same as the cell averages."""
    wl = helpers.flat(12, 10, depth=50.0, bc=(synth.BC_PERIODIC,) * 4)
    wl.hu[:] = 2.0 * 50.0
    wl.hv[:] = -1.0 * 50.0
    o = oracle_mod.Oracle(wl)
    ax, ay = o.face_speeds(wl.eta, wl.hu, wl.hv)
    c = np.sqrt(9.81 * 50.0)
    assert abs(ax - (2.0 + c)) < 1e-12 and abs(ay - (1.0 + c)) < 1e-12
    assert abs(o.max_speed(wl.eta, wl.hu, wl.hv) - (2.0 + c) / wl.dx) < 1e-15


def test_cell_average_step_breaks_the_face_condition(oracle_mod):
    """Under the cell-average time step the face speeds of the very states
    it steps exceed the bound of the positivity argument, dt a / dx <= 1/4,
    by an order of magnitude, and a cell depth goes negative."""
    wl = _shelf_case()
    o = oracle_mod.Oracle(wl)
    lam, depths = 0.0, []
    for e, u, v, t, step in _states(o, wl, 25):
        ax, ay = o.face_speeds(e, u, v, t)
        dt = wl.params.courant * 0.25 / o.max_speed(e, u, v)
        lam = max(lam, dt * max(ax / wl.dx, ay / wl.dy))
        depths.append(e)
    assert lam > 10 * 0.25, lam
    assert _min_depth(wl, depths) < -1e-4


def test_face_speed_step_keeps_depths_nonnegative(oracle_mod):
    """The same case with the time step bounded by the face speeds: every
    cell depth stays non-negative over the same 300 s (to round-off), with
    far more steps."""
    wl = _shelf_case()
    o = oracle_mod.Oracle(wl, cfl_faces=True)
    depths, steps = [], 0
    for e, u, v, t, steps in _states(o, wl, 500):
        depths.append(e)
    assert _min_depth(wl, depths) >= -1e-12
    assert steps > 20 * 300       # the cell-average step needs about 300 here
