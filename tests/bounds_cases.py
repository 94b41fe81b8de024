"""Cases run against the bounds-checked library (SWE_LIBRARY points at it):
tiny odd grids with every boundary kind, land across strips, a spatially
varying wind, flow relaxation, a batch of mixed domains, windows of a
decomposed domain, both FP32 modes, each single domain also with the
face-speed time step (its speed pass).
Prints one JSON object: case name -> [status of swe_get_info, error_cell]."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1912_02457_gb300 import swe, synth  # noqa: E402
from tests import helpers  # noqa: E402


def varying_wind(nfx=5, nfy=4):
    rng = np.random.default_rng(3)
    fr = rng.uniform(-12.0, 12.0, (3, nfy, nfx, 2)).astype(np.float32)
    return synth.Forcing(times=np.array([0.0, 3600.0, 1e7]), frames=fr, nfx=nfx, nfy=nfy)


def cases():
    out = []
    for (nx, ny) in [(8, 8), (17, 13), (29, 3), (57, 31), (3, 40), (61, 90)]:
        land = min(nx, ny) >= 8
        w = helpers.rough(nx, ny, seed=nx + ny, land=land, min_depth=5.0, cd=0.002)
        w.eta, w.hu, w.hv = helpers.random_state(w, seed=3, amp=0.2, mom=0.5)
        out.append((f"walls {nx}x{ny}", w))
        n = w.copy()
        n.bc = (synth.BC_NESTED, synth.BC_NESTED, synth.BC_NESTED, synth.BC_NESTED)
        n.boundary = synth.still_boundary(nx, ny, eta=0.05)
        n.wind = varying_wind()
        n.params = synth.Params(frs_width=min(10, nx, ny), cd=0.002)
        out.append((f"nested+varying wind {nx}x{ny}", n))
        p = helpers.periodic_rough(nx, ny, seed=nx * ny, land=land)
        p.eta, p.hu, p.hv = helpers.random_state(p, seed=4, amp=0.2, mom=0.5)
        out.append((f"periodic {nx}x{ny}", p))
    c = synth.coastal(96, 70)
    out.append(("coastal 96x70", c))
    return out


def main():
    res = {}
    for prec in ("f32", "f32_kahan"):
        doms = []
        for name, wl in cases():
            wl = wl.astype(np.float32)
            d = swe.Domain(wl, prec)
            d.step(7)
            i = d.info(check=False)
            st = swe.load().swe_get_info(d.h, swe.C.byref(i))
            res[f"{name} {prec}"] = [int(st), int(i.error_cell)]
            doms.append((name, wl))
            d.close()
            # the face-speed time step (its speed pass reads the same cells)
            wf = wl.copy()
            wf.params.cfl_faces = 1
            d = swe.Domain(wf, prec)
            d.step(7)
            i = d.info(check=False)
            st = swe.load().swe_get_info(d.h, swe.C.byref(i))
            res[f"{name} {prec} faces"] = [int(st), int(i.error_cell)]
            d.close()
        # the same domains in one batch
        b = swe.Batch()
        ds = [swe.Domain(wl, prec) for _, wl in doms]
        for d in ds:
            b.add(d)
        b.set_rows(8)
        b.step(5)
        b.sync()
        for (name, _), d in zip(doms, ds):
            i = d.info(check=False)
            st = swe.load().swe_get_info(d.h, swe.C.byref(i))
            res[f"batch {name} {prec}"] = [int(st), int(i.error_cell)]
        b.close()
        for d in ds:
            d.close()
        # domain decomposition: windows of the coastal domain (own-cell
        # plans, halo columns, cut edges as walls) and of a nested rough
        # domain with gridded wind (sampling at whole-domain positions)
        from paper_1912_02457_gb300.split import SplitDomain
        for name, wl in cases():
            if not (name.startswith("coastal") or name == "nested+varying wind 61x90"):
                continue
            for px, py in ((2, 2), (3, 1)):
                s = SplitDomain(wl.astype(np.float32), px, py, prec)
                s.step(5)
                for k, d in enumerate(s.doms):
                    i = d.info(check=False)
                    st = swe.load().swe_get_info(d.h, swe.C.byref(i))
                    res[f"split {px}x{py} window {k} {name} {prec}"] = [int(st), int(i.error_cell)]
                s.close()
    print(json.dumps(res))


if __name__ == "__main__":
    main()
