"""Host-side validation of swe_create_domain (no GPU needed: every case below
is rejected before the first CUDA call): empty and oversized grids, bad
spacing, precision, boundary kinds, unpaired periodic edges, a periodic
corner plane whose last line does not repeat its first, and out-of-range
parameters."""
import ctypes as C

import numpy as np
import pytest

from paper_1912_02457_gb300 import swe

INVALID = -1


@pytest.fixture(scope="module")
def L():
    from paper_1912_02457_gb300 import build
    build.build()
    return swe.load()


def _desc(nx=8, ny=6, bc=(0, 0, 0, 0), H=None, keep=None):
    d = swe.DomainDesc()
    d.nx, d.ny, d.dx, d.dy = nx, ny, 800.0, 800.0
    d.precision = 0
    for k in range(4):
        d.bc[k] = bc[k]
    buf = np.zeros(64, dtype=np.float32)       # never read: every case fails validation
    Hb = np.full(((ny + 1) * (nx + 1),), 10.0, dtype=np.float32) if H is None else H
    keep.extend([buf, Hb])
    d.eta = d.hu = d.hv = buf.ctypes.data
    d.H = Hb.ctypes.data
    d.f = d.theta = None
    d.f_const, d.theta_const = 1e-4, 0.0
    d.src_is_device = 0
    return d


def _create(L, d, p=None):
    p = swe.default_params() if p is None else p
    h = C.c_void_p()
    rc = L.swe_create_domain(C.byref(d), C.byref(p), None, C.byref(h))
    assert not h.value
    return rc


@pytest.mark.parametrize("nx,ny", [(0, 5), (5, 0), (-3, 4), (65537, 2)])
def test_empty_or_negative_grids(L, nx, ny):
    keep = []
    assert _create(L, _mk(nx, ny, keep)) == INVALID


def _mk(nx, ny, keep):
    d = _desc(nx=1, ny=1, keep=keep)
    d.nx, d.ny = nx, ny
    return d


def test_grids_beyond_32_bit_offsets(L):
    keep = []
    # nx * ny < 2^31 but the padded corner plane is not: rejected before allocation
    d = _mk(46400, 46400, keep)
    assert _create(L, d) == INVALID
    d = _mk(65536, 32769, keep)                  # nx * ny >= 2^31
    assert _create(L, d) == INVALID


def test_bad_spacing_precision_and_boundaries(L):
    keep = []
    d = _desc(keep=keep)
    d.dx = 0.0
    assert _create(L, d) == INVALID
    d = _desc(keep=keep)
    d.precision = 7
    assert _create(L, d) == INVALID
    d = _desc(bc=(0, 0, 0, 5), keep=keep)
    assert _create(L, d) == INVALID
    d = _desc(bc=(2, 0, 0, 0), keep=keep)        # periodic S without periodic N
    assert _create(L, d) == INVALID
    d = _desc(bc=(0, 0, 1, 0), keep=keep)        # nested W on a one-cell-wide domain
    d.nx = 1
    assert _create(L, d) == INVALID


def test_periodic_corner_plane_must_repeat_its_first_line(L):
    keep = []
    nx, ny = 8, 6
    H = np.full(((ny + 1) * (nx + 1),), 10.0, dtype=np.float32)
    H[3 * (nx + 1) + nx] = 11.0                  # row 3: last column differs from the first
    d = _desc(nx=nx, ny=ny, bc=(0, 0, 2, 2), H=H, keep=keep)
    assert _create(L, d) == INVALID
    H2 = np.full(((ny + 1) * (nx + 1),), 10.0, dtype=np.float32)
    H2[ny * (nx + 1) + 2] = 9.0                  # last row differs from the first
    d = _desc(nx=nx, ny=ny, bc=(2, 2, 0, 0), H=H2, keep=keep)
    assert _create(L, d) == INVALID


@pytest.mark.parametrize("field,value", [("g", 0.0), ("kappa", -1.0), ("courant", 0.0),
                                         ("theta_mm", 0.5), ("theta_mm", 2.5), ("frs_width", 33),
                                         ("frs_d0", 0.0), ("cd", -0.1), ("dt_fixed", -1.0),
                                         ("rho_water", 0.0), ("kernel", 3), ("cfl_faces", 2)])
def test_out_of_range_parameters(L, field, value):
    keep = []
    p = swe.default_params()
    setattr(p, field, value)
    assert _create(L, _desc(keep=keep), p) == INVALID


@pytest.mark.parametrize("precision,kernel", [(2, 0), (0, 1), (1, 1)])
def test_face_speed_step_needs_the_fp32_default_kernels(L, precision, kernel):
    """The face-speed time step exists on the FP32 default kernels only."""
    keep = []
    d = _desc(keep=keep)
    d.precision = precision
    if precision == 2:                           # FP64 inputs are doubles
        H = np.full(((d.ny + 1) * (d.nx + 1),), 10.0)
        keep.append(H)
        d.H = H.ctypes.data
    p = swe.default_params()
    p.kernel = kernel
    p.cfl_faces = 1
    assert _create(L, d, p) == swe.ERR_UNSUPPORTED
