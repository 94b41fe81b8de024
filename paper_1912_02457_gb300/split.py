"""A domain stepped as sub-domains that exchange halo cells (the domain
decomposition of the scheme on one device; swe_split_sync / swe_split_step
in swe.h).

Host bookkeeping only: the partition and the windows come from
``synth.partition`` / ``synth.window``, each window is a ``swe.Domain``
created as a window of the whole domain, and every step is one call of the
library (stages, halo copies and the shared clock run on the device).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from paper_1912_02457_gb300 import swe, synth


class SplitDomain:
    """``wl`` split into px x py sub-domains on one stream."""

    def __init__(self, wl, px: int, py: int, precision: str = "f32_kahan", stream: int = 0):
        self.wl = wl
        self.parts = synth.partition(wl.nx, wl.ny, px, py)
        self.doms = []
        try:
            for part in self.parts:
                self.doms.append(swe.Domain(synth.window(wl, part), precision, stream=stream,
                                            window=(part, wl.nx, wl.ny)))
        except Exception:
            self.close()
            raise
        self._handles = (C.c_void_p * len(self.doms))(*[d.h.value for d in self.doms])
        self._L = swe.load()
        self._check(self._L.swe_split_sync(self._handles, len(self.doms)), "swe_split_sync")

    @staticmethod
    def _check(rc, what):
        swe._check(rc, what)

    def step(self, n: int):
        self._check(self._L.swe_split_step(self._handles, len(self.doms), int(n)), "swe_split_step")

    def info(self, check: bool = True):
        return self.doms[0].info(check=check)

    def state(self):
        """(eta, hu, hv) of the whole domain, assembled from the own cells."""
        out = [np.zeros((self.wl.ny, self.wl.nx), dtype=self.doms[0].dtype) for _ in range(3)]
        for part, d in zip(self.parts, self.doms):
            x0, x1, y0, y1 = part["own"]
            wx0, _, wy0, _ = part["win"]
            for o, a in zip(out, d.state()):
                o[y0:y1, x0:x1] = a[y0 - wy0:y1 - wy0, x0 - wx0:x1 - wx0]
        return tuple(out)

    def close(self):
        for d in self.doms:
            d.close()
        self.doms = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
