"""The largest domain the library accepts: 46000 x 46000 cells (~2.1e9; the
padded corner plane still has fewer than 2^31 elements, so every cell and
corner offset fits the kernels' 32-bit index arithmetic). One step of the
fast FP32 path, checked against the oracle on sampled windows: after one
step a cell depends only on cells within four of it (two stages of a
radius-2 stencil), so with the same fixed dt the oracle run on a window
reproduces the window's cells that lie at least four cells inside it, or on
a real edge of the domain."""
import ctypes as C

import numpy as np
import pytest

from paper_1912_02457_gb300 import synth
from tests.test_gpu_parity import swe  # noqa: F401

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 46000
W = 24            # window side; its inner 16 x 16 cells (or up to a real wall) are exact
DT = 4.0


def test_largest_domain_one_step_on_sampled_windows(swe, oracle_mod):
    import torch
    dev = "cuda"
    jj = torch.arange(N, device=dev, dtype=torch.float32)[:, None]
    ii = torch.arange(N, device=dev, dtype=torch.float32)[None, :]
    eta = (0.1 * torch.sin(ii * 0.013) * torch.cos(jj * 0.017)).contiguous()
    hu = (0.2 * torch.cos(ii * 0.011) * torch.sin(jj * 0.007 + 0.3)).contiguous()
    hv = (0.15 * torch.sin(ii * 0.009 + 0.5) * torch.cos(jj * 0.012)).contiguous()
    Ji = torch.arange(N + 1, device=dev, dtype=torch.float32)[:, None]
    Ii = torch.arange(N + 1, device=dev, dtype=torch.float32)[None, :]
    H = (60.0 + 20.0 * torch.sin(Ii * 0.004) * torch.cos(Ji * 0.003)).contiguous()
    del jj, ii, Ji, Ii
    torch.cuda.synchronize()

    d = swe.DomainDesc()
    d.nx = d.ny = N
    d.dx = d.dy = 800.0
    d.precision = 0                                # plain FP32: fewer planes
    for k in range(4):
        d.bc[k] = synth.BC_WALL
    d.eta, d.hu, d.hv, d.H = eta.data_ptr(), hu.data_ptr(), hv.data_ptr(), H.data_ptr()
    d.f = d.theta = None
    d.f_const, d.theta_const = 1.1e-4, 0.2
    d.src_is_device = 1
    p = swe.default_params()
    p.dt_fixed = DT
    p.cd = 0.0
    L = swe.load()
    h = C.c_void_p()
    swe._check(L.swe_create_domain(C.byref(d), C.byref(p), None, C.byref(h)), "swe_create_domain")
    try:
        # the inputs are copied: keep host copies of the windows, free the rest
        starts = [(N // 2, N // 2), (N - W - 9, N - W - 11), (N - W, N - W), (0, N - W), (123457 % N, 2 ** 15)]
        win = {}
        for (j0, i0) in starts:
            win[(j0, i0)] = tuple(t[j0:j0 + W, i0:i0 + W].cpu().numpy() for t in (eta, hu, hv)) + \
                (H[j0:j0 + W + 1, i0:i0 + W + 1].cpu().numpy(),)
        del eta, hu, hv, H
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        swe._check(L.swe_step(h, 1), "swe_step")
        out = torch.empty((N, N), dtype=torch.float32, device=dev)
        got = {k: [] for k in win}
        for field in (swe.ETA, swe.HU, swe.HV):
            swe._check(L.swe_read_state(h, field, C.c_void_p(out.data_ptr()), 1), "swe_read_state")
            torch.cuda.synchronize()
            for (j0, i0) in win:
                got[(j0, i0)].append(out[j0:j0 + W, i0:i0 + W].cpu().numpy())
        del out
        info = swe.Info()
        swe._check(L.swe_get_info(h, C.byref(info)), "swe_get_info")
        assert info.step == 1 and info.error == 0
    finally:
        L.swe_destroy_domain(h)

    for (j0, i0), (e, u, v, Hw) in win.items():
        wl = synth.Workload(name="window", nx=W, ny=W, dx=800.0, dy=800.0, eta=e, hu=u, hv=v, H=Hw,
                            f=None, theta=None, f_const=1.1e-4, theta_const=0.2,
                            bc=(synth.BC_WALL,) * 4, params=synth.Params(dt_fixed=DT, cd=0.0))
        ref = oracle_mod.Oracle(wl).run(1, dt_fixed=DT)
        # exact region: four cells in from an artificial window edge, up to a real domain wall
        ja = 0 if j0 == 0 else 4
        ia = 0 if i0 == 0 else 4
        jb = W if j0 + W == N else W - 4
        ib = W if i0 + W == N else W - 4
        # the bound of the one-step kernel checks: 16 ulp of the largest state
        # component in the window (the state fields share one flux scale)
        gs = [g[ja:jb, ia:ib].astype(np.float64) for g in got[(j0, i0)]]
        rs = [r[ja:jb, ia:ib] for r in ref[:3]]
        scale = max(float(np.abs(r).max()) for r in rs)
        dev = max(float(np.abs(g - r).max()) for g, r in zip(gs, rs))
        assert dev <= 16 * float(np.spacing(np.float32(scale))), ((j0, i0), dev, scale)
