"""FP64 CPU oracle of the rotating shallow-water scheme (TEST INFRASTRUCTURE).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference arm may import this package. It shares no code with
the CUDA library: the arithmetic lives in ``swe_oracle.c``; this module
only compiles it with gcc and marshals ``Workload`` arrays into it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swe_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C99 + OpenMP, no fast-math, no FMA
    contraction) into oracle/_build/liboracle.so."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Domain(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double),
        ("g", C.c_double), ("theta_mm", C.c_double), ("kappa", C.c_double),
        ("cd", C.c_double), ("rho_air", C.c_double), ("rho_water", C.c_double),
        ("frs_d0", C.c_double), ("frs_width", C.c_int),
        ("bc", C.c_int * 4),
        ("H", C.POINTER(C.c_double)), ("f", C.POINTER(C.c_double)),
        ("theta", C.POINTER(C.c_double)),
        ("wind_n", C.c_int), ("wind_nfx", C.c_int), ("wind_nfy", C.c_int),
        ("wind_t", C.POINTER(C.c_double)), ("wind", C.POINTER(C.c_double)),
        ("bnd_n", C.c_int), ("bnd_nbx", C.c_int), ("bnd_nby", C.c_int),
        ("bnd_t", C.POINTER(C.c_double)), ("bnd", C.POINTER(C.c_double)),
        ("round_state_f32", C.c_int),
        ("cfl_faces", C.c_int),
        ("off_x", C.c_int), ("off_y", C.c_int), ("gnx", C.c_int), ("gny", C.c_int),
    ]


_dp = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_desing.restype = C.c_double
            L.orc_desing.argtypes = [C.c_double, C.c_double]
            L.orc_minmod.restype = C.c_double
            L.orc_minmod.argtypes = [C.c_double] * 3
            L.orc_wind_stress.restype = None
            L.orc_wind_stress.argtypes = [C.c_double] * 4 + [_dp, _dp]
            L.orc_rhs.restype = C.c_int
            L.orc_rhs.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp, C.c_double, _dp, _dp]
            L.orc_recon_x.restype = C.c_int
            L.orc_recon_x.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp, C.c_double, _dp]
            L.orc_face_speeds.restype = C.c_int
            L.orc_face_speeds.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp, C.c_double, _dp]
            L.orc_ghosts.restype = C.c_int
            L.orc_ghosts.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp, C.c_double, _dp]
            L.orc_step.restype = C.c_int
            L.orc_step.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp, C.c_double, C.c_double]
            L.orc_frs.restype = None
            L.orc_frs.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp, C.c_double]
            L.orc_max_speed.restype = C.c_double
            L.orc_max_speed.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp]
            L.orc_cfl_dt.restype = C.c_double
            L.orc_cfl_dt.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp, C.c_double]
            L.orc_run.restype = C.c_int
            L.orc_run.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp, _dp, _dp,
                                  C.c_long, C.c_int, C.c_double, C.c_double,
                                  C.c_int, _dp, C.c_double]
            L.orc_diagnostics.restype = None
            L.orc_diagnostics.argtypes = [C.POINTER(_Domain), _dp, _dp, _dp, _dp, _dp]
            L.orc_face_flux.restype = None
            L.orc_face_flux.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double,
                                        C.c_int, _dp]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_threads.restype = None
            L.orc_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_dp)


class Oracle:
    """The oracle bound to one workload's statics and forcing."""

    def __init__(self, wl, round_state_f32: bool = False, cfl_faces: bool = False,
                 offset=(0, 0), whole=None):
        """``offset``, ``whole``: the workload is the window of a larger
        domain of ``whole`` = (nx, ny) cells whose cell (0, 0) is the whole
        domain's cell ``offset`` (forcing sampled at the whole domain's
        positions); by default the workload is the whole domain."""
        self.wl = wl
        p = wl.params
        nx, ny = wl.nx, wl.ny
        self._keep = []

        def keep(a):
            a = _d(a)
            self._keep.append(a)
            return a

        H = keep(wl.H)
        f = keep(wl.f if wl.f is not None else np.full((ny, nx), wl.f_const))
        th = keep(wl.theta if wl.theta is not None else np.full((ny, nx), wl.theta_const))
        D = _Domain()
        D.nx, D.ny, D.dx, D.dy = nx, ny, wl.dx, wl.dy
        D.g, D.theta_mm, D.kappa, D.cd = p.g, p.theta_mm, p.kappa, p.cd
        D.rho_air, D.rho_water = p.rho_air, p.rho_water
        D.frs_d0, D.frs_width = p.frs_d0, p.frs_width
        for k in range(4):
            D.bc[k] = int(wl.bc[k])
        D.H, D.f, D.theta = _p(H), _p(f), _p(th)
        if wl.wind is not None:
            wt, wv = keep(wl.wind.times), keep(wl.wind.frames)
            D.wind_n, D.wind_nfx, D.wind_nfy = len(wt), wl.wind.nfx, wl.wind.nfy
            D.wind_t, D.wind = _p(wt), _p(wv)
        if wl.boundary is not None:
            bt, bv = keep(wl.boundary.times), keep(wl.boundary.frames)
            D.bnd_n, D.bnd_nbx, D.bnd_nby = len(bt), wl.boundary.nfx, wl.boundary.nfy
            D.bnd_t, D.bnd = _p(bt), _p(bv)
        D.round_state_f32 = int(bool(round_state_f32))
        D.cfl_faces = int(bool(cfl_faces or getattr(p, "cfl_faces", 0)))
        D.off_x, D.off_y = int(offset[0]), int(offset[1])
        if whole is not None:
            D.gnx, D.gny = int(whole[0]), int(whole[1])
        self.D = D
        self.L = lib()

    # -- single evaluations ------------------------------------------------
    def rhs(self, eta, hu, hv, t=0.0):
        e, u, v = _d(eta), _d(hu), _d(hv)
        ny, nx = e.shape
        M = np.empty((3, ny, nx))
        S = np.empty((ny, nx))
        rc = self.L.orc_rhs(C.byref(self.D), _p(e), _p(u), _p(v), t, _p(M), _p(S))
        if rc:
            raise MemoryError("oracle rhs failed")
        return M, S

    def recon_x(self, eta, hu, hv, t=0.0):
        e, u, v = _d(eta), _d(hu), _d(hv)
        ny, nx = e.shape
        out = np.empty((4, ny, nx))
        if self.L.orc_recon_x(C.byref(self.D), _p(e), _p(u), _p(v), t, _p(out)):
            raise MemoryError("oracle recon failed")
        return out

    def ghosts(self, eta, hu, hv, t=0.0):
        """The state padded with two ghost rings, filled at time t: shape
        (3, ny + 4, nx + 4), interior cell (i, j) at [:, j + 2, i + 2]."""
        e, u, v = _d(eta), _d(hu), _d(hv)
        ny, nx = e.shape
        out = np.empty((3, ny + 4, nx + 4))
        if self.L.orc_ghosts(C.byref(self.D), _p(e), _p(u), _p(v), t, _p(out)):
            raise MemoryError("oracle ghost fill failed")
        return out

    def face_speeds(self, eta, hu, hv, t=0.0):
        """The largest one-sided local speed max(a+, -a-) over the x-faces
        and over the y-faces of the reconstruction of a state at time t."""
        e, u, v = _d(eta), _d(hu), _d(hv)
        out = np.empty(2)
        if self.L.orc_face_speeds(C.byref(self.D), _p(e), _p(u), _p(v), t, _p(out)):
            raise MemoryError("oracle face speeds failed")
        return float(out[0]), float(out[1])

    def frs(self, eta, hu, hv, t):
        """The flow relaxation of eq:frs at time t, applied in place to
        float64 C-contiguous arrays."""
        for a in (eta, hu, hv):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        self.L.orc_frs(C.byref(self.D), _p(eta), _p(hu), _p(hv), float(t))

    def max_speed(self, eta, hu, hv):
        e, u, v = _d(eta), _d(hu), _d(hv)
        return self.L.orc_max_speed(C.byref(self.D), _p(e), _p(u), _p(v))

    def diagnostics(self, eta, hu, hv):
        e, u, v = _d(eta), _d(hu), _d(hv)
        m, en = C.c_double(), C.c_double()
        self.L.orc_diagnostics(C.byref(self.D), _p(e), _p(u), _p(v), C.byref(m), C.byref(en))
        return m.value, en.value

    # -- time stepping -----------------------------------------------------
    def run(self, n_steps, state=None, t=None, dt=0.0, step0=0, dt_fixed=None,
            courant=None, dt_every=None, return_dts=False, t_end=0.0):
        """Advance ``n_steps`` from ``state`` (default: the workload's initial
        state) and return (eta, hu, hv, t, dt[, dts])."""
        wl = self.wl
        p = wl.params
        if state is None:
            state = (wl.eta, wl.hu, wl.hv)
        e, u, v = (np.array(a, dtype=np.float64, order="C", copy=True) for a in state)
        tt = C.c_double(wl.t0 if t is None else t)
        dd = C.c_double(dt)
        dts = np.zeros(max(n_steps, 1))
        rc = self.L.orc_run(C.byref(self.D), _p(e), _p(u), _p(v), C.byref(tt), C.byref(dd),
                            int(step0), int(n_steps),
                            p.courant if courant is None else courant,
                            p.dt_fixed if dt_fixed is None else dt_fixed,
                            p.dt_update_every if dt_every is None else dt_every,
                            _p(dts), float(t_end))
        if rc:
            raise RuntimeError(f"oracle run failed (rc={rc})")
        out = (e, u, v, tt.value, dd.value)
        if return_dts:
            out = out + (dts[:n_steps],)
        return out


def desing(h, kappa):
    return lib().orc_desing(float(h), float(kappa))


def minmod(a, b, c):
    return lib().orc_minmod(float(a), float(b), float(c))


def wind_stress(wx, wy, rho_air=1.225, rho_water=1025.0):
    tx, ty = C.c_double(), C.c_double()
    lib().orc_wind_stress(wx, wy, rho_air, rho_water, C.byref(tx), C.byref(ty))
    return tx.value, ty.value


def face_flux(left, right, Hf, dir, g=9.81, kappa=1e-2):
    """Flux across one face from raw (h, eta, hu, hv) states on each side."""
    a, b = _d(left), _d(right)
    out = np.empty(3)
    lib().orc_face_flux(_p(a), _p(b), float(Hf), g, kappa, int(dir), _p(out))
    return out


def num_threads():
    return lib().orc_num_threads()


def set_threads(n):
    """Threads of the oracle's parallel loops from now on."""
    lib().orc_set_threads(int(n))
