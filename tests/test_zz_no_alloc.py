"""swe_diagnostics_noalloc: the same mass and energy as swe_diagnostics,
from caller-owned device buffers and without any device allocation by the
library (for callers that cannot allocate: graph capture, framework-owned
memory pools, real-time loops). Collected last so that a first-failure stop
has already run every other test; it must also pass alone in a fresh
process."""
import numpy as np
import pytest

from paper_1912_02457_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swe():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1912_02457_gb300 import build, swe as S
    build.build()
    S.load()
    return S


def _close(a, b, rel=1e-12):
    return abs(a - b) <= rel * max(abs(b), 1.0)


def test_noalloc_matches_diagnostics_twice(swe):
    import torch
    wl = synth.coastal(300, 220, seed_config=96, dtype=np.float32)
    nx, ny = wl.nx, wl.ny
    H = torch.from_numpy(np.ascontiguousarray(wl.H)).cuda()
    with swe.Domain(wl, "f32") as d:
        for n_steps in (7, 13):                  # two calls in a row, different states
            d.step(n_steps)
            want = d.diagnostics()
            planes = [torch.empty((ny, nx), dtype=torch.float32, device="cuda") for _ in range(3)]
            for field, t in zip((swe.ETA, swe.HU, swe.HV), planes):
                d.read_device(field, t.data_ptr())
            out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            # an FP32 domain holds g and kappa rounded to float32: pass the same
            swe.diagnostics_noalloc(planes[0].data_ptr(), planes[1].data_ptr(), planes[2].data_ptr(),
                                    H.data_ptr(), nx, ny, nx, nx + 1, wl.dx, wl.dy, out.data_ptr(),
                                    g=float(np.float32(wl.params.g)),
                                    kappa=float(np.float32(wl.params.kappa)))
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert _close(got[0], want[0]) and _close(got[1], want[1]), (got, want)


def _device_planes(swe, d, nx, ny):
    import torch
    planes = [torch.empty((ny, nx), dtype=torch.float32, device="cuda") for _ in range(3)]
    for field, t in zip((swe.ETA, swe.HU, swe.HV), planes):
        d.read_device(field, t.data_ptr())
    torch.cuda.synchronize()
    return planes


def test_noalloc_and_domain_diagnostics_match_oracle(swe, oracle_mod):
    """An FP32 coastal state: the domain's own diagnostics (which use the
    domain's float32 g and kappa) against the oracle given the same two
    values, and the allocation-free call with the exact g and kappa against
    the oracle as configured by the workload, both to 1e-12. Free device
    memory does not move across a call (after the first, which loads the
    library's module)."""
    import torch
    wl = synth.coastal(300, 220, seed_config=96, member=1, dtype=np.float32)
    nx, ny = wl.nx, wl.ny
    H = torch.from_numpy(np.ascontiguousarray(wl.H)).cuda()
    with swe.Domain(wl, "f32") as d:
        d.step(9)
        state = d.state()
        dom = d.diagnostics()
        planes = _device_planes(swe, d, nx, ny)
    w32 = wl.copy()
    w32.params.g = float(np.float32(wl.params.g))
    w32.params.kappa = float(np.float32(wl.params.kappa))
    om32 = oracle_mod.Oracle(w32).diagnostics(*state)
    assert _close(dom[0], om32[0]) and _close(dom[1], om32[1]), (dom, om32)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")

    def call():
        swe.diagnostics_noalloc(planes[0].data_ptr(), planes[1].data_ptr(), planes[2].data_ptr(),
                                H.data_ptr(), nx, ny, nx, nx + 1, wl.dx, wl.dy, out.data_ptr(),
                                g=wl.params.g, kappa=wl.params.kappa)
        torch.cuda.synchronize()

    call()
    free0, _ = torch.cuda.mem_get_info()
    out.fill_(float("nan"))
    call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    got = out.cpu().numpy()
    om = oracle_mod.Oracle(wl).diagnostics(*state)
    assert _close(got[0], om[0]) and _close(got[1], om[1]), (got, om)


def test_noalloc_rejects_too_many_rows(swe):
    import torch
    ny = swe.NOALLOC_MAX_ROWS + 1
    buf = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(swe.SweError) as ei:
        swe.diagnostics_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                1, ny, 1, 2, 1.0, 1.0, out.data_ptr())
    assert ei.value.status == swe.ERR_INVALID_ARG
