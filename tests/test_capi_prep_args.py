"""Host-side argument checks of the pre-processing entry points: every bad
argument is rejected with SWE_ERR_INVALID_ARG before any CUDA call (so these
run without a GPU)."""
import ctypes as C

import pytest

from paper_1912_02457_gb300 import swe

INVALID = -1
FAKE = C.c_void_p(0x10000)          # never dereferenced: the checks reject first


@pytest.fixture(scope="module")
def L():
    from paper_1912_02457_gb300 import build
    build.build()
    return swe.load()


def test_work_bytes(L):
    assert L.swe_bathymetry_work_bytes(0, 5) == 0
    small = L.swe_bathymetry_work_bytes(10, 10)
    big = L.swe_bathymetry_work_bytes(1000, 1000)
    assert 0 < small < big and big >= 1000 * 1001 * 4          # a corner plane at least


def test_bathymetry_rejects(L):
    f = L.swe_bathymetry_reconstruct
    assert f(None, 10, 10, 10, FAKE, 11, FAKE, 1, 1.3, 0.1, None, None) == INVALID
    assert f(FAKE, 9, 10, 10, FAKE, 11, FAKE, 1, 1.3, 0.1, None, None) == INVALID      # pitch < nx
    assert f(FAKE, 10, 10, 10, FAKE, 10, FAKE, 1, 1.3, 0.1, None, None) == INVALID     # cpitch < nx+1
    assert f(FAKE, 10, 10, 10, FAKE, 11, FAKE, -1, 1.3, 0.1, None, None) == INVALID    # n_iter
    assert f(FAKE, 10, 10, 10, FAKE, 11, FAKE, 5000, 1.3, 0.1, None, None) == INVALID  # > max
    assert f(FAKE, 10, 10, 10, FAKE, 11, FAKE, 1, 0.9, 0.1, None, None) == INVALID     # theta
    assert f(FAKE, 10, 10, 10, FAKE, 11, FAKE, 1, 1.3, 1.5, None, None) == INVALID     # smooth
    assert f(FAKE, 10, 10, 10, FAKE, 11, C.c_void_p(0x10010), 1, 1.3, 0.1, None, None) == INVALID  # work alignment


def test_erode_rejects(L):
    f = L.swe_land_erode
    assert f(None, FAKE, FAKE, 10, 10, 10, 5.0, FAKE, FAKE, FAKE, None) == INVALID
    assert f(FAKE, FAKE, FAKE, 9, 10, 10, 5.0, FAKE, C.c_void_p(0x20000), C.c_void_p(0x30000), None) == INVALID
    assert f(FAKE, C.c_void_p(0x20000), C.c_void_p(0x30000), 10, 10, 10, 5.0, FAKE,
             C.c_void_p(0x40000), C.c_void_p(0x50000), None) == INVALID            # land_out aliases land
    assert f(FAKE, C.c_void_p(0x20000), C.c_void_p(0x30000), 10, 10, 10, -1.0, C.c_void_p(0x60000),
             C.c_void_p(0x40000), C.c_void_p(0x50000), None) == INVALID            # negative depth


def test_refine_and_coarsen_reject(L):
    P = [C.c_void_p(0x10000 * k) for k in range(1, 9)]
    r = L.swe_refine2
    assert r(P[0], P[1], P[2], 10, P[3], 11, 10, 10, 1.3, P[4], P[5], P[6], 21, P[7], 21, None) == INVALID  # odd fpitch
    assert r(P[0], P[1], P[2], 10, P[3], 11, 10, 10, 1.3, P[4], P[5], P[6], 18, P[7], 21, None) == INVALID  # fpitch < 2nx
    assert r(P[0], P[1], P[2], 10, P[3], 11, 10, 10, 1.3, C.c_void_p(0x10004), P[5], P[6], 20, P[7], 21,
             None) == INVALID                                                                      # misaligned
    assert r(P[0], P[1], P[2], 10, P[3], 11, 10, 10, 2.5, P[4], P[5], P[6], 20, P[7], 21, None) == INVALID  # theta
    c = L.swe_coarsen2
    assert c(P[0], P[1], P[2], 20, P[3], 20, 10, 10, P[4], P[5], P[6], 10, P[7], 11, None) == INVALID      # fcpitch
    assert c(None, P[1], P[2], 20, P[3], 21, 10, 10, P[4], P[5], P[6], 10, P[7], 11, None) == INVALID
