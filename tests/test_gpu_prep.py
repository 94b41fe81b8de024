"""Grid pre-processing on the GPU (swe_prep.cu, through the C ABI) against
the FP64 oracle (oracle/prep.py) on the same FP32 inputs: corner bathymetry
and refinement / coarsening (FP32 arithmetic: tolerances in units of the
FP32 spacing of the largest value), land erosion (bit-exact)."""
import ctypes as C

import numpy as np
import pytest

from oracle import prep
from paper_1912_02457_gb300 import swe, synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1912_02457_gb300 import build
    build.build()


def _rough(nx, ny, seed):
    """Cell-average depths of the coastal recipe's kind: a spectral field
    with an eastward ramp, 5 - 3000 m."""
    rng = np.random.default_rng(1912_02457 + 7000 + seed)
    z = synth.spectral_field(rng, ny, nx).astype(np.float64)
    z = z + 1.5 * np.linspace(-1, 1, nx)[None, :]
    z = (z - z.min()) / max(z.max() - z.min(), 1e-12)
    return 5.0 + 2995.0 * z ** 2


def _dev(a, dtype, pad=0):
    """Device copy of a 2-D array with `pad` extra columns of row pitch."""
    a = np.asarray(a, dtype=dtype)
    ny, nx = a.shape
    t = torch.zeros((ny, nx + pad), dtype=getattr(torch, np.dtype(dtype).name), device="cuda")
    t[:, :nx] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t


def _host(t, nx):
    torch.cuda.synchronize()
    return t[:, :nx].cpu().numpy()


SHAPES = [(70, 45), (1, 9), (33, 1), (2, 2), (129, 67)]


def _ulp(x):
    return float(np.spacing(np.float32(np.abs(x).max())))


def _bathy_gpu(Hm32, nx, ny, n_iter, pad=(3, 5)):
    Hm_d = _dev(Hm32, np.float32, pad=pad[0])
    Hc_d = _dev(np.zeros((ny + 1, nx + 1)), np.float32, pad=pad[1])
    work = torch.empty(swe.bathymetry_work_bytes(nx, ny), dtype=torch.uint8, device="cuda")
    stats = swe.bathymetry_reconstruct(Hm_d.data_ptr(), Hm_d.stride(0), nx, ny, Hc_d.data_ptr(),
                                       Hc_d.stride(0), work.data_ptr(), n_iter=n_iter,
                                       stream=torch.cuda.current_stream().cuda_stream)
    return _host(Hc_d, nx + 1).astype(np.float64), stats


# FP32 against FP64 on the same inputs: the initial guess is within ~1 ulp of
# the largest depth, each iteration adds at most a few (measured: 2.5 ulp
# after ten); 16 ulp bounds ten iterations with margin, and is ~1e-6 of the
# depth range, far below any misfit the iteration itself leaves
ULPS = 16


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("n_iter", [0, 10])
def test_bathymetry_matches_oracle(nx, ny, n_iter):
    Hm = _rough(nx, ny, nx * 131 + ny).astype(np.float32)
    got, stats = _bathy_gpu(Hm, nx, ny, n_iter)
    if n_iter == 0:
        ref = prep.initial_corners(Hm.astype(np.float64))
    else:
        ref, misfit, change = prep.reconstruct_bathymetry(Hm.astype(np.float64), n_iter=n_iter)
        np.testing.assert_allclose(stats[:, 0], misfit, rtol=0, atol=ULPS * _ulp(ref))
        np.testing.assert_allclose(stats[:, 1], change, rtol=0, atol=ULPS * _ulp(ref))
    np.testing.assert_allclose(got, ref, rtol=0, atol=ULPS * _ulp(ref))


@pytest.mark.gpu
def test_bathymetry_full_size_4096():
    """The size the bench times, every corner against the oracle."""
    nx = ny = 4096
    Hm = _rough(nx, ny, 1).astype(np.float32)
    got, stats = _bathy_gpu(Hm, nx, ny, 10, pad=(0, 0))
    ref, misfit, change = prep.reconstruct_bathymetry(Hm.astype(np.float64), n_iter=10)
    np.testing.assert_allclose(got, ref, rtol=0, atol=ULPS * _ulp(ref))
    np.testing.assert_allclose(stats[:, 0], misfit, rtol=0, atol=ULPS * _ulp(ref))


@pytest.mark.gpu
@pytest.mark.parametrize("aligned", [False, True])
@pytest.mark.parametrize("nx,ny", [(64, 48), (1, 7), (130, 3), (67, 33), (8192, 64)])
def test_land_erosion_is_bit_exact(nx, ny, aligned):
    """Both kernels: one cell per thread (a pitch that is not a multiple of
    4) and four cells per thread with vector loads (pitch a multiple of 4;
    a row length that is not is finished cell by cell)."""
    rng = np.random.default_rng(nx + 17 * ny)
    land = rng.random((ny, nx)) < 0.5
    eta = rng.standard_normal((ny, nx)).astype(np.float32)
    Hm = rng.uniform(5.0, 300.0, (ny, nx)).astype(np.float32)
    pad = 8 - nx % 4 if aligned else (6 if (nx + 6) % 4 else 5)
    assert ((nx + pad) % 4 == 0) == aligned
    L_d = _dev(land.astype(np.uint8), np.uint8, pad)
    e_d, H_d = _dev(eta, np.float32, pad), _dev(Hm, np.float32, pad)
    Lo, eo, Ho = torch.zeros_like(L_d), torch.zeros_like(e_d), torch.zeros_like(H_d)
    swe.land_erode(L_d.data_ptr(), e_d.data_ptr(), H_d.data_ptr(), nx + pad, nx, ny,
                   Lo.data_ptr(), eo.data_ptr(), Ho.data_ptr(), land_depth=5.0,
                   stream=torch.cuda.current_stream().cuda_stream)
    stays, eta2, H2, _ = prep.erode_land(land, eta.astype(np.float64), Hm.astype(np.float64), 5.0)
    np.testing.assert_array_equal(_host(Lo, nx).astype(bool), stays)
    np.testing.assert_array_equal(_host(eo, nx).astype(np.float64), eta2)
    np.testing.assert_array_equal(_host(Ho, nx).astype(np.float64), H2)


def _coastal_small(nx, ny, seed):
    wl = synth.coastal(nx, ny, seed_config=95, member=seed, land_frac=0.3)
    rng = np.random.default_rng(seed)
    land = wl.land_cells()
    q = [np.where(land, 0.0, rng.standard_normal((ny, nx))).astype(np.float32) for _ in range(3)]
    return q, wl.H.astype(np.float32)


def _refine_gpu(q, H, nx, ny, vec=False):
    """vec: an even coarse pitch and a fine pitch that is a multiple of 4
    (the two-cell kernel with vector loads and stores); else an odd coarse
    pitch (the one-cell kernel)."""
    st = torch.cuda.current_stream().cuda_stream
    qd = [_dev(a, np.float32, pad=4 + nx % 2 if vec else 5 - nx % 2) for a in q]
    assert (qd[0].stride(0) % 2 == 0) == vec
    Hd = _dev(H, np.float32, pad=3)
    fp, fcp = (2 * nx + 4 + 3) // 4 * 4 if vec else 2 * nx + 4, 2 * nx + 3
    qf = [torch.zeros((2 * ny, fp), dtype=torch.float32, device="cuda") for _ in range(3)]
    Hf = torch.zeros((2 * ny + 1, fcp), dtype=torch.float32, device="cuda")
    swe.refine2([t.data_ptr() for t in qd], qd[0].stride(0), Hd.data_ptr(), Hd.stride(0), nx, ny,
                [t.data_ptr() for t in qf], fp, Hf.data_ptr(), fcp, stream=st)
    return qf, Hf, fp, fcp


def _small_case(nx, ny):
    return _coastal_small(nx, ny, nx + ny) if min(nx, ny) > 4 else (
        [np.random.default_rng(3).standard_normal((ny, nx)).astype(np.float32) for _ in range(3)],
        np.random.default_rng(4).uniform(5, 50, (ny + 1, nx + 1)).astype(np.float32))


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny", [(70, 46), (33, 9), (1, 1), (2, 5), (257, 31)])
def test_refine_kernels_agree_bitwise(nx, ny):
    """The two-cell kernel (vector loads and stores, odd last cell of a row
    by the one-cell code) gives the one-cell kernel's bits."""
    q, H = _small_case(nx, ny)
    a, _, _, _ = _refine_gpu(q, H, nx, ny, vec=False)
    b, _, _, _ = _refine_gpu(q, H, nx, ny, vec=True)
    for x, y in zip(a, b):
        assert np.array_equal(_host(x, 2 * nx), _host(y, 2 * nx))


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny", [(70, 46), (33, 9), (1, 1), (2, 5), (257, 31)])
def test_coarsen_kernels_agree_bitwise(nx, ny):
    """The two-cell coarsening kernel (fine pitch a multiple of 4, even
    coarse pitch; the odd last cell of a row by the one-cell code) gives the
    one-cell kernel's bits."""
    q, H = _small_case(nx, ny)
    qf, Hf, fp, fcp = _refine_gpu(q, H, nx, ny, vec=True)
    st = torch.cuda.current_stream().cuda_stream
    got = []
    for cpad in (nx % 2 + 2, nx % 2 + 1):          # even, then odd coarse pitch
        cq = [torch.zeros((ny, nx + cpad), dtype=torch.float32, device="cuda") for _ in range(3)]
        cH = torch.zeros((ny + 1, nx + 3), dtype=torch.float32, device="cuda")
        assert (cq[0].stride(0) % 2 == 0) == (cpad == nx % 2 + 2)
        swe.coarsen2([t.data_ptr() for t in qf], fp, Hf.data_ptr(), fcp, nx, ny,
                     [t.data_ptr() for t in cq], cq[0].stride(0), cH.data_ptr(), nx + 3, stream=st)
        got.append([_host(t, nx) for t in cq])
    for a, b in zip(*got):
        assert np.array_equal(a, b)


@pytest.mark.gpu
@pytest.mark.parametrize("vec", [False, True])
@pytest.mark.parametrize("nx,ny", [(70, 46), (33, 9), (1, 1), (2, 5)])
def test_refine_and_coarsen_match_oracle(nx, ny, vec):
    q, H = _small_case(nx, ny)
    qf, Hf, fp, fcp = _refine_gpu(q, H, nx, ny, vec=vec)
    ref = prep.refine2(*(a.astype(np.float64) for a in q), H.astype(np.float64))
    scale = max(float(np.abs(np.stack(q)).max()), 1e-30)
    for t, r in zip(qf, ref[:3]):
        np.testing.assert_allclose(_host(t, 2 * nx), r, rtol=0, atol=8 * 2.0 ** -24 * scale)
    got_H = _host(Hf, 2 * nx + 1)
    land_ref = ref[3] == prep.LAND
    np.testing.assert_array_equal(got_H == np.float32(prep.LAND), land_ref)
    # a mean of two or four FP32 corners rounds up to three times
    np.testing.assert_allclose(got_H[~land_ref], ref[3][~land_ref], rtol=0,
                               atol=4 * _ulp(ref[3][~land_ref]))

    # coarsen the GPU's fine fields back, on the GPU, against the oracle
    cq = [torch.zeros((ny, nx + 2), dtype=torch.float32, device="cuda") for _ in range(3)]
    cH = torch.zeros((ny + 1, nx + 3), dtype=torch.float32, device="cuda")
    swe.coarsen2([t.data_ptr() for t in qf], fp, Hf.data_ptr(), fcp, nx, ny,
                 [t.data_ptr() for t in cq], nx + 2, cH.data_ptr(), nx + 3,
                 stream=torch.cuda.current_stream().cuda_stream)
    fine_host = [_host(t, 2 * nx).astype(np.float64) for t in qf]
    cref = prep.coarsen2(*fine_host, got_H.astype(np.float64))
    for t, r, orig in zip(cq, cref[:3], q):
        got = _host(t, nx)
        np.testing.assert_allclose(got, r, rtol=0, atol=4 * 2.0 ** -24 * scale)
        # and coarsening undoes the refinement up to FP32 rounding
        np.testing.assert_allclose(got, orig, rtol=0, atol=8 * 2.0 ** -24 * scale)
    np.testing.assert_array_equal(_host(cH, nx + 1), H)


@pytest.mark.gpu
def test_refine_full_size_4096_sampled():
    nx = ny = 4096
    q, H = _coastal_small(nx, ny, 9)
    qf, Hf, fp, fcp = _refine_gpu(q, H, nx, ny, vec=True)    # the layout the bench times
    # sampled rows against the oracle on the slab of rows j-1..j+1 that
    # decides them (a slab edge is a domain edge only where it is one)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([[0, ny - 1], rng.integers(1, ny - 1, 24)]))
    scale = float(np.abs(np.stack(q)).max())
    for j in rows:
        lo, hi = max(j - 1, 0), min(j + 2, ny)
        sub = prep.refine2(*(a[lo:hi].astype(np.float64) for a in q), H[lo:hi + 1].astype(np.float64))
        k = j - lo
        for t, r in zip(qf, sub[:3]):
            got = t[2 * j:2 * j + 2, :2 * nx].cpu().numpy()
            ref = r[2 * k:2 * k + 2]
            np.testing.assert_allclose(got, ref, rtol=0, atol=8 * 2.0 ** -24 * scale)
