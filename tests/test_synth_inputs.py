"""Properties of the seeded synthetic inputs (CPU only): what the
generators promise about the workloads they build."""
import numpy as np

from paper_1912_02457_gb300 import synth


def _hbar(wl):
    Hm = np.where(wl.H == synth.LAND, np.nan, wl.H.astype(np.float64))
    return 0.25 * (Hm[:-1, :-1] + Hm[1:, :-1] + Hm[:-1, 1:] + Hm[1:, 1:])


def test_coastal_external_levels_cover_the_bed(oracle_mod):
    """The nesting data of the coastal recipe is an external model's level:
    on raised shelves that reach a nested edge it never lies below the bed,
    so neither the ghost rings nor the flow-relaxation zone (Section 3.6)
    are pulled to a negative depth. Checked at and between the hourly
    frames through the oracle's ghost fill, for every wet cell of each
    edge's relaxation zone."""
    wl = synth.coastal(96, 80, seed_config=92, member=1, dtype=np.float32)
    Hb = _hbar(wl)
    land = wl.land_cells()
    zone = wl.params.frs_width
    need_s = np.where(land[:zone, :], -np.inf, -Hb[:zone, :]).max(axis=0)
    need_n = np.where(land[-zone:, :], -np.inf, -Hb[-zone:, :]).max(axis=0)
    need_w = np.where(land[:, :zone], -np.inf, -Hb[:, :zone]).max(axis=1)
    assert max(need_s.max(), need_n.max(), need_w.max()) > 0.5     # shelves reach the edges
    o = oracle_mod.Oracle(wl)
    tol = 1e-6                                                     # float32 frames
    for t in (0.0, 1800.0, 3600.0, 5000.0, 30000.0):
        G = o.ghosts(wl.eta, wl.hu, wl.hv, t=t)[0]
        for ring in range(2):
            assert np.all(G[1 - ring, 2:-2] >= need_s - tol)
            assert np.all(G[wl.ny + 2 + ring, 2:-2] >= need_n - tol)
            assert np.all(G[2:-2, 1 - ring] >= need_w - tol)
