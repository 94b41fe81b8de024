"""Thin ctypes binding of libswe (include/swe.h).

Argument marshalling only: every step of the scheme runs in the library's
CUDA kernels. Loading fails loudly when the library has not been built;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SWE_LIBRARY may point at another build of the same library (tuning builds)
LIB_PATH = os.environ.get("SWE_LIBRARY") or os.path.join(_HERE, "_build", "libswe.so")

F32, F32_KAHAN, F64 = 0, 1, 2
PRECISIONS = {"f32": F32, "f32_kahan": F32_KAHAN, "f64": F64}
WIND, BOUNDARY = 0, 1
ETA, HU, HV, COMP_ETA, COMP_HU, COMP_HV = range(6)

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NUMERIC, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5


class SweError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = f"{what}: {_status_string(status)}"
        if status == ERR_CUDA and _lib is not None:
            msg += f" ({_lib.swe_last_cuda_error().decode()})"
        super().__init__(msg)


class Params(C.Structure):
    _fields_ = [("g", C.c_double), ("theta_mm", C.c_double), ("kappa", C.c_double),
                ("cd", C.c_double), ("courant", C.c_double), ("frs_d0", C.c_double),
                ("frs_width", C.c_int), ("dt_update_every", C.c_int),
                ("dt_fixed", C.c_double), ("rho_air", C.c_double),
                ("rho_water", C.c_double), ("t0", C.c_double), ("kernel", C.c_int),
                ("cfl_faces", C.c_int),
                ("window_x0", C.c_int), ("window_y0", C.c_int), ("whole_nx", C.c_int),
                ("whole_ny", C.c_int), ("own_x0", C.c_int), ("own_x1", C.c_int),
                ("own_y0", C.c_int), ("own_y1", C.c_int)]


class DomainDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("precision", C.c_int), ("bc", C.c_int * 4),
                ("eta", C.c_void_p), ("hu", C.c_void_p), ("hv", C.c_void_p),
                ("H", C.c_void_p), ("f", C.c_void_p), ("theta", C.c_void_p),
                ("f_const", C.c_double), ("theta_const", C.c_double),
                ("src_is_device", C.c_int)]


class Info(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("step", C.c_longlong),
                ("error", C.c_int), ("error_cell", C.c_int), ("error_step", C.c_longlong),
                ("max_speed", C.c_double), ("launches", C.c_longlong),
                ("done", C.c_int), ("t_end", C.c_double)]


_lib = None
_lock = threading.Lock()
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# every exported symbol of include/swe.h with its (restype, argtypes)
SIGNATURES = {
    "swe_abi_version": (C.c_int, []),
    "swe_last_cuda_error": (C.c_char_p, []),
    "swe_status_string": (C.c_char_p, [C.c_int]),
    "swe_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
    "swe_default_params": (None, [C.POINTER(Params)]),
    "swe_create_domain": (C.c_int, [C.POINTER(DomainDesc), C.POINTER(Params), C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    "swe_set_forcing": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_int, C.c_int]),
    "swe_step": (C.c_int, [C.c_void_p, C.c_int]),
    "swe_set_end_time": (C.c_int, [C.c_void_p, C.c_double]),
    "swe_launches_per_step": (C.c_int, [C.c_void_p]),
    "swe_launch_name": (C.c_char_p, [C.c_void_p, C.c_int]),
    "swe_step_profiled": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "swe_read_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "swe_write_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "swe_set_clock": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_longlong]),
    "swe_get_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "swe_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "swe_destroy_domain": (C.c_int, [C.c_void_p]),
    "swe_batch_create": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "swe_batch_add": (C.c_int, [C.c_void_p, C.c_void_p]),
    "swe_batch_remove": (C.c_int, [C.c_void_p, C.c_void_p]),
    "swe_batch_size": (C.c_int, [C.c_void_p]),
    "swe_batch_set_rows": (C.c_int, [C.c_void_p, C.c_int]),
    "swe_batch_rows": (C.c_int, [C.c_void_p]),
    "swe_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "swe_batch_step_serial": (C.c_int, [C.c_void_p, C.c_int]),
    "swe_batch_sync": (C.c_int, [C.c_void_p]),
    "swe_batch_poll": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "swe_batch_launches": (C.c_longlong, [C.c_void_p]),
    "swe_batch_destroy": (C.c_int, [C.c_void_p]),
    "swe_split_sync": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "swe_split_step": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int]),
    "swe_diagnostics_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_int, C.c_int, C.c_longlong, C.c_longlong,
                                          C.c_double, C.c_double, C.c_double, C.c_double,
                                          C.c_void_p, C.c_void_p]),
    "swe_bathymetry_work_bytes": (C.c_size_t, [C.c_int, C.c_int]),
    "swe_bathymetry_reconstruct": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_void_p,
                                             C.c_longlong, C.c_void_p, C.c_int, C.c_double, C.c_double,
                                             C.c_void_p, C.c_void_p]),
    "swe_land_erode": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_int, C.c_int,
                                 C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "swe_refine2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p,
                              C.c_longlong, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_longlong, C.c_void_p, C.c_longlong, C.c_void_p]),
    "swe_coarsen2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p,
                               C.c_longlong, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_longlong, C.c_void_p, C.c_longlong, C.c_void_p]),
}

NOALLOC_MAX_ROWS = 16384


# ---- grid pre-processing: device pointers and pitches in elements (swe.h)

def bathymetry_work_bytes(nx, ny):
    return int(load().swe_bathymetry_work_bytes(int(nx), int(ny)))


def bathymetry_reconstruct(Hm_ptr, pitch, nx, ny, Hc_ptr, cpitch, work_ptr, n_iter=10,
                           theta=1.3, smooth=0.125, stats=True, stream=0):
    """Corner bathymetry from FP64 cell averages; returns, when `stats`, an
    (n_iter, 2) array of the per-iteration midpoint misfit and corner change."""
    out = np.zeros(2 * max(int(n_iter), 1), dtype=np.float64) if stats else None
    _check(load().swe_bathymetry_reconstruct(
        C.c_void_p(Hm_ptr), int(pitch), int(nx), int(ny), C.c_void_p(Hc_ptr), int(cpitch),
        C.c_void_p(work_ptr), int(n_iter), float(theta), float(smooth),
        out.ctypes.data_as(C.c_void_p) if stats else None, C.c_void_p(stream)),
        "swe_bathymetry_reconstruct")
    return out[:2 * int(n_iter)].reshape(-1, 2) if stats else None


def land_erode(land_ptr, eta_ptr, Hm_ptr, pitch, nx, ny, land_out_ptr, eta_out_ptr, Hm_out_ptr,
               land_depth=5.0, stream=0):
    _check(load().swe_land_erode(C.c_void_p(land_ptr), C.c_void_p(eta_ptr), C.c_void_p(Hm_ptr),
                                 int(pitch), int(nx), int(ny), float(land_depth),
                                 C.c_void_p(land_out_ptr), C.c_void_p(eta_out_ptr),
                                 C.c_void_p(Hm_out_ptr), C.c_void_p(stream)), "swe_land_erode")


def refine2(q_ptrs, pitch, H_ptr, cpitch, nx, ny, qf_ptrs, fpitch, Hf_ptr, fcpitch, theta=1.3,
            stream=0):
    """q_ptrs / qf_ptrs: device pointers of (eta, hu, hv), coarse / fine."""
    _check(load().swe_refine2(*(C.c_void_p(p) for p in q_ptrs), int(pitch), C.c_void_p(H_ptr),
                              int(cpitch), int(nx), int(ny), float(theta),
                              *(C.c_void_p(p) for p in qf_ptrs), int(fpitch), C.c_void_p(Hf_ptr),
                              int(fcpitch), C.c_void_p(stream)), "swe_refine2")


def coarsen2(qf_ptrs, fpitch, Hf_ptr, fcpitch, nx, ny, q_ptrs, pitch, H_ptr, cpitch, stream=0):
    """nx, ny: the coarse size; the fine planes are 2ny x 2nx."""
    _check(load().swe_coarsen2(*(C.c_void_p(p) for p in qf_ptrs), int(fpitch), C.c_void_p(Hf_ptr),
                               int(fcpitch), int(nx), int(ny), *(C.c_void_p(p) for p in q_ptrs),
                               int(pitch), C.c_void_p(H_ptr), int(cpitch), C.c_void_p(stream)),
           "swe_coarsen2")


def diagnostics_noalloc(eta_ptr, hu_ptr, hv_ptr, H_ptr, nx, ny, pitch, cpitch, dx, dy,
                        out_ptr, g=9.81, kappa=1e-2, stream=0):
    """Mass and energy of caller-owned FP32 device planes into a caller-owned
    device buffer of 2 doubles, without any device allocation (see swe.h)."""
    _check(load().swe_diagnostics_noalloc(C.c_void_p(eta_ptr), C.c_void_p(hu_ptr),
                                          C.c_void_p(hv_ptr), C.c_void_p(H_ptr), int(nx), int(ny),
                                          int(pitch), int(cpitch), float(dx), float(dy), float(g),
                                          float(kappa), C.c_void_p(out_ptr), C.c_void_p(stream)),
           "swe_diagnostics_noalloc")


def load(path: str = LIB_PATH):
    """Load libswe. Raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libswe not built ({path} missing): run "
                                   "`python -m paper_1912_02457_gb300.build`")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                try:
                    fn = getattr(L, name)
                except AttributeError:
                    # another build given by SWE_LIBRARY (a tuning build of an
                    # earlier version) may lack later entry points; the
                    # in-tree library exports every one (checked by the tests)
                    if path == LIB_PATH and "SWE_LIBRARY" not in os.environ:
                        raise
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _status_string(s):
    try:
        return load().swe_status_string(s).decode()
    except Exception:
        return str(s)


def _check(rc, what):
    if rc != OK:
        raise SweError(rc, what)


def default_params() -> Params:
    p = Params()
    load().swe_default_params(C.byref(p))
    return p


def params_from(wl_params, t0=0.0, kernel=0) -> Params:
    p = default_params()
    for k in ("g", "theta_mm", "kappa", "cd", "courant", "frs_d0", "frs_width",
              "dt_update_every", "dt_fixed", "rho_air", "rho_water"):
        setattr(p, k, getattr(wl_params, k))
    p.t0 = t0
    p.kernel = kernel
    p.cfl_faces = int(getattr(wl_params, "cfl_faces", 0))
    return p


_torch_alloc_refs = None


def use_torch_allocator():
    """Route libswe's device allocations through PyTorch's caching allocator."""
    global _torch_alloc_refs
    import torch

    def _alloc(nbytes, stream, ctx):
        dev = torch.cuda.current_device()
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(load().swe_set_allocator(refs[0], refs[1], None), "swe_set_allocator")
    _torch_alloc_refs = refs


def use_default_allocator():
    """Domains created from now on allocate with cudaMalloc again (domains
    created under another allocator keep returning their buffers to it)."""
    _check(load().swe_set_allocator(C.cast(None, ALLOC_FN), C.cast(None, FREE_FN), None),
           "swe_set_allocator")


class Domain:
    """One simulated domain held by libswe.

    ``wl`` is a synth.Workload with host numpy arrays; ``precision`` one of
    'f32', 'f32_kahan', 'f64'; ``stream`` a cudaStream_t as an int (0: the
    legacy default stream, which is also PyTorch's default stream)."""

    def __init__(self, wl, precision: str = "f32", stream: int = 0, kernel: str = "fast",
                 window=None):
        """``window``: (part, whole_nx, whole_ny) with ``part`` an entry of
        ``synth.partition``: ``wl`` is that window of a larger domain (see
        swe_params in swe.h), stepped with its sub-domains by ``split``."""
        L = load()
        self.wl = wl
        self.prec = PRECISIONS[precision]
        self.dtype = np.float64 if self.prec == F64 else np.float32
        self.nx, self.ny = wl.nx, wl.ny
        keep = []

        def arr(a):
            a = np.ascontiguousarray(a, dtype=self.dtype)
            keep.append(a)
            return a.ctypes.data

        d = DomainDesc()
        d.nx, d.ny, d.dx, d.dy = wl.nx, wl.ny, wl.dx, wl.dy
        d.precision = self.prec
        for k in range(4):
            d.bc[k] = int(wl.bc[k])
        d.eta, d.hu, d.hv, d.H = arr(wl.eta), arr(wl.hu), arr(wl.hv), arr(wl.H)
        d.f = arr(wl.f) if wl.f is not None else None
        d.theta = arr(wl.theta) if wl.theta is not None else None
        d.f_const, d.theta_const = wl.f_const, wl.theta_const
        d.src_is_device = 0
        p = params_from(wl.params, wl.t0, {"fast": 0, "reference": 1}[kernel])
        if window is not None:
            part, p.whole_nx, p.whole_ny = window
            wx0, _, wy0, _ = part["win"]
            x0, x1, y0, y1 = part["own"]
            p.window_x0, p.window_y0 = wx0, wy0
            p.own_x0, p.own_x1, p.own_y0, p.own_y1 = x0 - wx0, x1 - wx0, y0 - wy0, y1 - wy0
        h = C.c_void_p()
        _check(L.swe_create_domain(C.byref(d), C.byref(p), C.c_void_p(stream), C.byref(h)),
               "swe_create_domain")
        self.h = h
        self._L = L
        if wl.wind is not None:
            self.set_forcing(WIND, wl.wind)
        if wl.boundary is not None:
            self.set_forcing(BOUNDARY, wl.boundary)

    def set_forcing(self, kind, forcing):
        t = np.ascontiguousarray(forcing.times, dtype=np.float64)
        fr = np.ascontiguousarray(forcing.frames, dtype=np.float32)
        _check(self._L.swe_set_forcing(self.h, kind, len(t), t.ctypes.data, fr.ctypes.data,
                                       forcing.nfx, forcing.nfy), "swe_set_forcing")

    def step(self, n: int):
        _check(self._L.swe_step(self.h, int(n)), "swe_step")

    def set_end_time(self, t_end: float):
        _check(self._L.swe_set_end_time(self.h, float(t_end)), "swe_set_end_time")

    def launches_per_step(self) -> int:
        return self._L.swe_launches_per_step(self.h)

    def launch_names(self):
        return [self._L.swe_launch_name(self.h, k).decode() for k in range(self.launches_per_step())]

    def step_profiled(self, n: int) -> np.ndarray:
        """Step n times; return per-launch device times (ms), shape (n, parts)."""
        parts = self.launches_per_step()
        ms = np.zeros(n * parts, dtype=np.float32)
        _check(self._L.swe_step_profiled(self.h, int(n), ms.ctypes.data, ms.size), "swe_step_profiled")
        return ms.reshape(n, parts)

    def read(self, field: int) -> np.ndarray:
        out = np.empty((self.ny, self.nx), dtype=self.dtype)
        _check(self._L.swe_read_state(self.h, field, out.ctypes.data, 0), "swe_read_state")
        return out

    def read_device(self, field: int, ptr: int):
        _check(self._L.swe_read_state(self.h, field, C.c_void_p(ptr), 1), "swe_read_state")

    def state(self):
        return tuple(self.read(k) for k in (ETA, HU, HV))

    def write(self, field: int, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=self.dtype)
        _check(self._L.swe_write_state(self.h, field, a.ctypes.data, 0), "swe_write_state")

    def write_device(self, field: int, ptr: int):
        _check(self._L.swe_write_state(self.h, field, C.c_void_p(ptr), 1), "swe_write_state")

    def set_clock(self, t: float, dt: float = 0.0, step: int = 0):
        _check(self._L.swe_set_clock(self.h, t, dt, step), "swe_set_clock")

    def info(self, check: bool = True) -> Info:
        i = Info()
        rc = self._L.swe_get_info(self.h, C.byref(i))
        if check:
            _check(rc, "swe_get_info")
        return i

    def diagnostics(self):
        out = (C.c_double * 2)()
        _check(self._L.swe_diagnostics(self.h, out), "swe_diagnostics")
        return out[0], out[1]

    def close(self):
        if getattr(self, "h", None):
            self._L.swe_destroy_domain(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many FP32 domains advanced by one launch per stage."""

    def __init__(self, stream: int = 0, max_domains: int = 4096):
        self._L = load()
        h = C.c_void_p()
        _check(self._L.swe_batch_create(C.c_void_p(stream), int(max_domains), C.byref(h)),
               "swe_batch_create")
        self.h = h
        self.domains = []

    def add(self, dom: "Domain"):
        _check(self._L.swe_batch_add(self.h, dom.h), "swe_batch_add")
        self.domains.append(dom)

    def remove(self, dom: "Domain"):
        _check(self._L.swe_batch_remove(self.h, dom.h), "swe_batch_remove")
        self.domains.remove(dom)

    def set_rows(self, rows: int):
        _check(self._L.swe_batch_set_rows(self.h, int(rows)), "swe_batch_set_rows")

    def rows(self) -> int:
        return self._L.swe_batch_rows(self.h)

    def step(self, n: int):
        _check(self._L.swe_batch_step(self.h, int(n)), "swe_batch_step")

    def step_serial(self, n: int):
        _check(self._L.swe_batch_step_serial(self.h, int(n)), "swe_batch_step_serial")

    def sync(self):
        _check(self._L.swe_batch_sync(self.h), "swe_batch_sync")

    def poll(self):
        n = len(self.domains)
        done = np.zeros(max(n, 1), dtype=np.int32)
        t = np.zeros(max(n, 1), dtype=np.float64)
        _check(self._L.swe_batch_poll(self.h, done.ctypes.data, t.ctypes.data, max(n, 1)),
               "swe_batch_poll")
        return done[:n].astype(bool), t[:n]

    def launches(self) -> int:
        return self._L.swe_batch_launches(self.h)

    def close(self):
        if getattr(self, "h", None):
            self._L.swe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
