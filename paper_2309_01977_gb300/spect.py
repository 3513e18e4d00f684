"""Thin ctypes binding of libspect (include/spect.h).

Argument marshalling only: every step of the projector and of OSEM runs in
the library's CUDA kernels.  Tensors must be CUDA float32 (double for the
diagnostics), contiguous and 16-byte aligned; the binding passes their data
pointers and the current torch stream.  There is no CPU fallback: a missing
library raises ``SpectError``.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspect.so")

SPECT_OK = 0
SPECT_EINVAL = -1
SPECT_ENOMEM = -2
SPECT_ECUDA = -3
SPECT_EBUDGET = -4
SPECT_ETIMEDOUT = -5
SPECT_ECANCELLED = -6
SPECT_ESTATE = -7
SPECT_ENOTFOUND = -8

SPECT_FLAG_ATTEN = 1
SPECT_FLAG_PSF = 2
SPECT_FLAG_PSF_BF16 = 4
SPECT_FLAG_ATTEN_F64 = 8

SPECT_PRIOR_NONE, SPECT_PRIOR_QUADRATIC, SPECT_PRIOR_RDP = 0, 1, 2
SPECT_ALG_OSMAPOSL, SPECT_ALG_BSREM = 1, 2
PRIORS = {"none": SPECT_PRIOR_NONE, "quadratic": SPECT_PRIOR_QUADRATIC, "rdp": SPECT_PRIOR_RDP}
ALGORITHMS = {"osmaposl": SPECT_ALG_OSMAPOSL, "bsrem": SPECT_ALG_BSREM}

# Every symbol include/spect.h declares (checked by the CPU test suite).
EXPORTED = [
    "spect_plan_create", "spect_plan_destroy", "spect_plan_query", "spect_subset_size", "spect_subset_angles",
    "spect_forward", "spect_back", "spect_sensitivity", "spect_osem_run", "spect_poisson_ll",
    "spect_status_str", "spect_last_error", "spect_version",
    "spect_profile_enable", "spect_profile_read", "spect_kernel_launches",
    "spect_poisson_ll_noalloc", "spect_plan_check", "spect_plan_set_mu", "spect_osem_run_dev",
    "spect_map_run", "spect_prior_grad", "spect_multi_osem_run", "spect_plan_selftest_timeout",
    "spect_plan_reserve_stream", "spect_plan_release_stream",
    "spect_serve_create", "spect_serve_submit", "spect_serve_poll", "spect_serve_wait",
    "spect_serve_cancel", "spect_serve_stats_get", "spect_serve_destroy",
]


class SpectError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


class _MapParams(ctypes.Structure):
    _fields_ = [("algorithm", ctypes.c_int), ("prior", ctypes.c_int), ("beta", ctypes.c_float),
                ("delta", ctypes.c_float), ("gamma", ctypes.c_float), ("alpha0", ctypes.c_float)]


class _Geom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("voxel_cm", ctypes.c_float),
        ("n_angles", ctypes.c_int),
        ("angles_rad", ctypes.POINTER(ctypes.c_double)),
        ("psf_sigma0", ctypes.c_float), ("psf_slope", ctypes.c_float),
        ("psf_nsigma", ctypes.c_float), ("det_offset", ctypes.c_float),
        ("n_subsets", ctypes.c_int),
        ("flags", ctypes.c_uint),
        ("det_offsets", ctypes.POINTER(ctypes.c_float)),
        ("det_shifts", ctypes.POINTER(ctypes.c_float)),
        ("fov_mask", ctypes.POINTER(ctypes.c_float)),
    ]


class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_ulonglong), ("total_ms", ctypes.c_double)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("nz", ctypes.c_int), ("n_angles", ctypes.c_int), ("n_subsets", ctypes.c_int),
        ("max_subset_size", ctypes.c_int), ("psf_rmax", ctypes.c_int),
        ("device_bytes", ctypes.c_size_t), ("atten_cache_bytes", ctypes.c_size_t),
        ("ztile", ctypes.c_int), ("n_ztiles", ctypes.c_int), ("threads", ctypes.c_int), ("smem_bytes", ctypes.c_int),
    ]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libspect.so (built by ``paper_2309_01977_gb300.build``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise SpectError(SPECT_ECUDA, "libspect.so not found at %s: build it with "
                                          "paper_2309_01977_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        vp, i, f, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
        lib.spect_plan_create.argtypes = [ctypes.POINTER(_Geom), vp, vp, ctypes.POINTER(vp)]
        lib.spect_plan_destroy.argtypes = [vp]
        lib.spect_plan_query.argtypes = [vp, ctypes.POINTER(_PlanInfo)]
        lib.spect_plan_check.argtypes = [vp]
        lib.spect_plan_selftest_timeout.argtypes = [vp, ctypes.c_longlong, vp]
        lib.spect_plan_reserve_stream.argtypes = [vp, vp]
        lib.spect_plan_release_stream.argtypes = [vp, vp]
        lib.spect_subset_size.argtypes = [vp, i]
        lib.spect_subset_angles.argtypes = [vp, i, ctypes.POINTER(ctypes.c_int)]
        lib.spect_forward.argtypes = [vp, vp, vp, i, i, vp]
        lib.spect_back.argtypes = [vp, vp, vp, i, i, vp]
        lib.spect_sensitivity.argtypes = [vp, i, vp, vp]
        lib.spect_osem_run.argtypes = [vp, vp, f, vp, i, i, vp, vp]
        lib.spect_map_run.argtypes = [vp, vp, f, vp, i, i, ctypes.POINTER(_MapParams), vp]
        lib.spect_prior_grad.argtypes = [vp, i, i, i, f, f, vp, vp]
        lib.spect_multi_osem_run.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(f), i, ctypes.POINTER(vp),
                                             ctypes.POINTER(f), vp, i, i, vp]
        lib.spect_osem_run_dev.argtypes = [vp, vp, vp, vp, i, i, vp, vp]
        lib.spect_plan_set_mu.argtypes = [vp, vp, vp]
        lib.spect_poisson_ll.argtypes = [vp, vp, vp, f, ctypes.c_size_t, vp, vp, vp]
        lib.spect_poisson_ll_noalloc.argtypes = [vp, vp, f, ctypes.c_size_t, vp, vp, vp]
        for name in ("spect_status_str",):
            getattr(lib, name).restype = ctypes.c_char_p
            getattr(lib, name).argtypes = [i]
        lib.spect_last_error.restype = ctypes.c_char_p
        lib.spect_last_error.argtypes = []
        lib.spect_version.restype = ctypes.c_char_p
        lib.spect_version.argtypes = []
        lib.spect_profile_enable.argtypes = [vp, i]
        lib.spect_profile_read.argtypes = [vp, ctypes.POINTER(_KernelTime), i, i]
        lib.spect_kernel_launches.restype = ctypes.c_ulonglong
        lib.spect_kernel_launches.argtypes = []
        _lib = lib
        _ = d
        return lib


def _check(rc: int) -> int:
    if rc < 0:
        lib = load()
        raise SpectError(rc, "%s: %s" % (lib.spect_status_str(rc).decode(), lib.spect_last_error().decode()))
    return rc


def _stream(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dptr(t: Optional[torch.Tensor], dtype=torch.float32) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise SpectError(SPECT_EINVAL, "expected a CUDA tensor")
    if t.dtype != dtype:
        raise SpectError(SPECT_EINVAL, "expected %s, got %s" % (dtype, t.dtype))
    if not t.is_contiguous():
        raise SpectError(SPECT_EINVAL, "expected a contiguous tensor")
    return t.data_ptr()


@dataclass
class Geometry:
    """Python mirror of ``spect_geom`` (voxel units unless stated)."""

    n: int
    nz: int
    n_angles: int
    n_subsets: int = 1
    voxel_cm: float = 0.48
    attenuation: bool = True
    psf: bool = True
    psf_sigma0: float = 0.5
    psf_slope: float = 0.03
    psf_nsigma: float = 3.0
    det_offset: float = 0.0
    atten_f64: bool = False
    psf_bf16: bool = False
    angles_rad: Optional[Sequence[float]] = None
    det_offsets: Optional[Sequence[float]] = None  # per-angle detector offsets (non-circular orbit)
    det_shifts: Optional[Sequence[float]] = None   # per-angle shifts along the detector axis (T_trans)
    fov_mask: Optional[object] = None              # [n_angles][n][nz] projection weights (T_fov)

    def to_c(self):
        g = _Geom()
        g.nx = g.ny = int(self.n)
        g.nz = int(self.nz)
        g.voxel_cm = float(self.voxel_cm)
        g.n_angles = int(self.n_angles)
        keep = []
        if self.angles_rad is not None:
            arr = (ctypes.c_double * len(self.angles_rad))(*[float(a) for a in self.angles_rad])
            keep.append(arr)
            g.angles_rad = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        if self.det_offsets is not None:
            if len(self.det_offsets) != self.n_angles:
                raise SpectError(SPECT_EINVAL, "det_offsets needs one value per angle")
            arr = (ctypes.c_float * len(self.det_offsets))(*[float(v) for v in self.det_offsets])
            keep.append(arr)
            g.det_offsets = ctypes.cast(arr, ctypes.POINTER(ctypes.c_float))
        if self.det_shifts is not None:
            if len(self.det_shifts) != self.n_angles:
                raise SpectError(SPECT_EINVAL, "det_shifts needs one value per angle")
            arr = (ctypes.c_float * len(self.det_shifts))(*[float(v) for v in self.det_shifts])
            keep.append(arr)
            g.det_shifts = ctypes.cast(arr, ctypes.POINTER(ctypes.c_float))
        if self.fov_mask is not None:
            import numpy as np
            m = np.ascontiguousarray(np.asarray(self.fov_mask, dtype=np.float32))
            if m.shape != (self.n_angles, self.n, self.nz):
                raise SpectError(SPECT_EINVAL, "fov_mask must be [n_angles][n][nz]")
            keep.append(m)
            g.fov_mask = m.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        g.psf_sigma0 = float(self.psf_sigma0)
        g.psf_slope = float(self.psf_slope)
        g.psf_nsigma = float(self.psf_nsigma)
        g.det_offset = float(self.det_offset)
        g.n_subsets = int(self.n_subsets)
        g.flags = ((SPECT_FLAG_ATTEN if self.attenuation else 0) | (SPECT_FLAG_PSF if self.psf else 0)
                   | (SPECT_FLAG_ATTEN_F64 if self.atten_f64 else 0) | (SPECT_FLAG_PSF_BF16 if self.psf_bf16 else 0))
        return g, keep


# ---------------------------------------------------------------- C-named calls

def spect_plan_create(geom: Geometry, mu: Optional[torch.Tensor] = None, stream=None) -> int:
    lib = load()
    g, keep = geom.to_c()
    out = ctypes.c_void_p()
    _check(lib.spect_plan_create(ctypes.byref(g), _dptr(mu), _stream(stream), ctypes.byref(out)))
    del keep
    return out.value


def spect_plan_destroy(plan: int) -> None:
    _check(load().spect_plan_destroy(plan))


def spect_plan_check(plan: int) -> None:
    """Raise if a kernel of the plan gave up a bounded wait (synchronises)."""
    _check(load().spect_plan_check(plan))


def spect_plan_selftest_timeout(plan: int, limit_cycles: int, stream=None) -> None:
    """Run the bounded-wait failure path once: a kernel waits on a barrier that
    nothing arrives on for limit_cycles SM cycles and records SPECT_ETIMEDOUT
    in the plan's status word (read it with spect_plan_check)."""
    _check(load().spect_plan_selftest_timeout(plan, int(limit_cycles), _stream(stream)))


def spect_plan_reserve_stream(plan: int, stream=None) -> None:
    """Create the plan's scratch for `stream` now (before a graph capture on it)."""
    _check(load().spect_plan_reserve_stream(plan, _stream(stream)))


def spect_plan_release_stream(plan: int, stream=None) -> None:
    """Wait for `stream` and free the plan's scratch for it."""
    _check(load().spect_plan_release_stream(plan, _stream(stream)))


def spect_plan_query(plan: int) -> dict:
    info = _PlanInfo()
    _check(load().spect_plan_query(plan, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in _PlanInfo._fields_}


def spect_subset_size(plan: int, subset: int) -> int:
    return _check(load().spect_subset_size(plan, subset))


def spect_subset_angles(plan: int, subset: int) -> list:
    n = spect_subset_size(plan, subset)
    buf = (ctypes.c_int * n)()
    _check(load().spect_subset_angles(plan, subset, buf))
    return list(buf)


def spect_forward(plan: int, x: torch.Tensor, proj: torch.Tensor, subset: int = -1, batch: int = 1, stream=None):
    _check(load().spect_forward(plan, _dptr(x), _dptr(proj), subset, batch, _stream(stream)))


def spect_back(plan: int, proj: torch.Tensor, x_out: torch.Tensor, subset: int = -1, batch: int = 1, stream=None):
    _check(load().spect_back(plan, _dptr(proj), _dptr(x_out), subset, batch, _stream(stream)))


def spect_sensitivity(plan: int, subset: int, out: torch.Tensor, stream=None):
    _check(load().spect_sensitivity(plan, subset, _dptr(out), _stream(stream)))


def spect_osem_run(plan: int, y: torch.Tensor, s: float, x: torch.Tensor, first_subiter: int, n_subiters: int,
                   diag: Optional[torch.Tensor] = None, stream=None):
    _check(load().spect_osem_run(plan, _dptr(y), float(s), _dptr(x), first_subiter, n_subiters,
                                 _dptr(diag, torch.float64), _stream(stream)))


def spect_osem_run_dev(plan: int, y: torch.Tensor, s_dev: torch.Tensor, x: torch.Tensor, first_subiter: int,
                       n_subiters: int, diag: Optional[torch.Tensor] = None, stream=None):
    _check(load().spect_osem_run_dev(plan, _dptr(y), _dptr(s_dev), _dptr(x), first_subiter, n_subiters,
                                     _dptr(diag, torch.float64), _stream(stream)))


def spect_map_run(plan: int, y: torch.Tensor, s: float, x: torch.Tensor, first_subiter: int, n_subiters: int,
                  algorithm: str, prior: str, beta: float, delta: float = 1.0, gamma: float = 2.0,
                  alpha0: float = 1.0, stream=None):
    mp = _MapParams(ALGORITHMS[algorithm], PRIORS[prior], beta, delta, gamma, alpha0)
    _check(load().spect_map_run(plan, _dptr(y), float(s), _dptr(x), first_subiter, n_subiters, ctypes.byref(mp),
                                _stream(stream)))


def spect_multi_osem_run(plans, scales, ys, ss, x: torch.Tensor, first_subiter: int, n_subiters: int, stream=None):
    """OSEM over several photopeaks (include/spect.h): plans, scales, ys, ss per peak."""
    P = len(plans)
    if not (len(scales) == len(ys) == len(ss) == P):
        raise SpectError(SPECT_EINVAL, "plans, scales, ys and ss must have one entry per peak")
    ph = (ctypes.c_void_p * P)(*[p.handle if isinstance(p, Plan) else p for p in plans])
    sc = (ctypes.c_float * P)(*[float(v) for v in scales])
    yp = (ctypes.c_void_p * P)(*[_dptr(y) for y in ys])
    sp = (ctypes.c_float * P)(*[float(v) for v in ss])
    _check(load().spect_multi_osem_run(ph, sc, P, yp, sp, _dptr(x), first_subiter, n_subiters, _stream(stream)))


def spect_prior_grad(x: torch.Tensor, prior: str, grad: torch.Tensor, delta: float = 1.0, gamma: float = 2.0,
                     stream=None):
    if x.dim() != 3 or x.shape[0] != x.shape[1] or grad.shape != x.shape:
        raise SpectError(SPECT_EINVAL, "x must be [n][n][nz] and grad the same shape")
    _check(load().spect_prior_grad(_dptr(x), x.shape[0], x.shape[2], PRIORS[prior], float(delta), float(gamma),
                                   _dptr(grad), _stream(stream)))


def spect_plan_set_mu(plan: int, mu: Optional[torch.Tensor], stream=None):
    _check(load().spect_plan_set_mu(plan, _dptr(mu), _stream(stream)))


def spect_poisson_ll(plan: int, y: torch.Tensor, p: torch.Tensor, s: float, ll: torch.Tensor,
                     grad: Optional[torch.Tensor] = None, stream=None):
    if y.numel() != p.numel() or (grad is not None and grad.numel() != p.numel()):
        raise SpectError(SPECT_EINVAL, "y, p and grad must have the same size")
    _check(load().spect_poisson_ll(plan, _dptr(y), _dptr(p), float(s), p.numel(), _dptr(ll, torch.float64),
                                   _dptr(grad), _stream(stream)))


def spect_poisson_ll_noalloc(y: torch.Tensor, p: torch.Tensor, s: float, ll: torch.Tensor,
                             grad: Optional[torch.Tensor] = None, stream=None):
    """Poisson log-likelihood without a plan, for callers that cannot allocate
    device memory: the library's built-in scratch holds the partial sums (up to
    67,108,864 bins); calls on one device must not overlap on the GPU."""
    if y.numel() != p.numel() or (grad is not None and grad.numel() != p.numel()):
        raise SpectError(SPECT_EINVAL, "y, p and grad must have the same size")
    _check(load().spect_poisson_ll_noalloc(_dptr(y), _dptr(p), float(s), p.numel(), _dptr(ll, torch.float64),
                                           _dptr(grad), _stream(stream)))


def spect_version() -> str:
    return load().spect_version().decode()


def spect_profile_enable(plan: int, on: bool) -> None:
    _check(load().spect_profile_enable(plan, int(bool(on))))


def spect_profile_read(plan: int, reset: bool = False) -> dict:
    """{kernel name: (launches, total ms)} from the plan's CUDA-event records (synchronises)."""
    buf = (_KernelTime * 32)()
    n = _check(load().spect_profile_read(plan, buf, 32, int(bool(reset))))
    return {buf[k].name.decode(): (int(buf[k].launches), float(buf[k].total_ms)) for k in range(n)}


def spect_kernel_launches() -> int:
    return int(load().spect_kernel_launches())


# ---------------------------------------------------------------- convenience

class Plan:
    """Owning wrapper of a ``spect_plan``: allocates outputs and frees the plan."""

    def __init__(self, geom: Geometry, mu: Optional[torch.Tensor] = None, stream=None):
        self.geom = geom
        if geom.attenuation and mu is None:
            raise SpectError(SPECT_EINVAL, "attenuation needs a mu map")
        self.device = (mu.device if mu is not None else torch.device("cuda", torch.cuda.current_device()))
        self.handle = spect_plan_create(geom, mu.contiguous() if mu is not None else None, stream)

    def close(self):
        if getattr(self, "handle", None):
            spect_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return spect_plan_query(self.handle)

    def check(self) -> None:
        spect_plan_check(self.handle)

    def subset_angles(self, subset: int) -> list:
        return spect_subset_angles(self.handle, subset)

    def forward(self, x: torch.Tensor, subset: int = -1, out: Optional[torch.Tensor] = None, stream=None):
        g = self.geom
        batch = x.numel() // (g.n * g.n * g.nz)
        na = spect_subset_size(self.handle, subset)
        if out is None:
            out = torch.empty((batch, na, g.n, g.nz) if x.dim() == 4 else (na, g.n, g.nz), device=x.device,
                              dtype=torch.float32)
        spect_forward(self.handle, x, out, subset, batch, stream)
        return out

    def back(self, proj: torch.Tensor, subset: int = -1, out: Optional[torch.Tensor] = None, stream=None):
        g = self.geom
        na = spect_subset_size(self.handle, subset)
        batch = proj.numel() // (na * g.n * g.nz)
        if out is None:
            out = torch.empty((batch, g.n, g.n, g.nz) if proj.dim() == 4 else (g.n, g.n, g.nz),
                              device=proj.device, dtype=torch.float32)
        spect_back(self.handle, proj, out, subset, batch, stream)
        return out

    def sensitivity(self, subset: int, stream=None):
        g = self.geom
        out = torch.empty((g.n, g.n, g.nz), device=self.device, dtype=torch.float32)
        spect_sensitivity(self.handle, subset, out, stream)
        return out

    def osem(self, y: torch.Tensor, s: float, x: torch.Tensor, first: int, count: int, diag: bool = False,
             stream=None):
        d = torch.zeros((max(count, 1), 3), device=x.device, dtype=torch.float64) if diag else None
        spect_osem_run(self.handle, y, s, x, first, count, d, stream)
        return d

    def map(self, y: torch.Tensor, s: float, x: torch.Tensor, first: int, count: int, algorithm: str = "bsrem",
            prior: str = "rdp", beta: float = 0.3, delta: float = 1.0, gamma: float = 2.0, alpha0: float = 1.0,
            stream=None):
        """OSMAPOSL / BSREM subiterations with a nearest-neighbour prior (include/spect.h)."""
        spect_map_run(self.handle, y, s, x, first, count, algorithm, prior, beta, delta, gamma, alpha0, stream)

    def poisson_ll(self, y: torch.Tensor, p: torch.Tensor, s: float, grad: bool = False, stream=None):
        ll = torch.zeros(1, device=p.device, dtype=torch.float64)
        gr = torch.empty_like(p) if grad else None
        spect_poisson_ll(self.handle, y, p, s, ll, gr, stream)
        return ll, gr


def uniform_angles(n_angles: int) -> list:
    return [2.0 * math.pi * a / n_angles for a in range(n_angles)]


# ---------------------------------------------------------------- serving (include/spect_serve.h)

SPECT_REQ_QUEUED, SPECT_REQ_RUNNING, SPECT_REQ_DONE, SPECT_REQ_FAILED, SPECT_REQ_CANCELLED = range(5)

SERVE_EXPORTED = ["spect_serve_create", "spect_serve_submit", "spect_serve_poll", "spect_serve_wait",
                  "spect_serve_cancel", "spect_serve_stats_get", "spect_serve_destroy"]


class _ServeCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("n_streams", ctypes.c_int),
                ("wait_timeout_ms", ctypes.c_int)]


class _Request(ctypes.Structure):
    _fields_ = [("geom", _Geom), ("mu_host", ctypes.c_void_p), ("y_host", ctypes.c_void_p), ("s", ctypes.c_float),
                ("n_iters", ctypes.c_int), ("tag", ctypes.c_uint64)]


class _ServeStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "admitted", "completed", "failed", "cancelled",
                                                "rejected", "queued", "active", "peak_active", "bytes_in_use",
                                                "peak_bytes", "slots_created", "graph_slots")] + \
               [(k, ctypes.c_double) for k in ("p50_ms", "p99_ms", "max_ms", "recon_per_s")]


def _serve_lib():
    lib = load()
    if not getattr(lib, "_serve_bound", False):
        vp = ctypes.c_void_p
        lib.spect_serve_create.argtypes = [ctypes.POINTER(_ServeCfg), ctypes.POINTER(vp)]
        lib.spect_serve_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]
        lib.spect_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
        lib.spect_serve_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double)]
        lib.spect_serve_cancel.argtypes = [vp, ctypes.c_uint64]
        lib.spect_serve_stats_get.argtypes = [vp, ctypes.POINTER(_ServeStats)]
        lib.spect_serve_destroy.argtypes = [vp]
        lib._serve_bound = True
    return lib


class Server:
    """Continuous-batching reconstruction server (host numpy float32 in and out)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 8, n_streams: int = 8, wait_timeout_ms: int = 600000):
        lib = _serve_lib()
        cfg = _ServeCfg(int(hbm_budget_bytes), int(max_slots), int(n_streams), int(wait_timeout_ms))
        h = ctypes.c_void_p()
        _check(lib.spect_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self._shapes = {}

    def submit(self, geom: Geometry, mu, y, s: float, n_iters: int, tag: int = 0) -> int:
        import numpy as np
        lib = _serve_lib()
        g, keep = geom.to_c()
        y = np.ascontiguousarray(y, dtype=np.float32)
        mu = None if mu is None else np.ascontiguousarray(mu, dtype=np.float32)
        req = _Request(g, None if mu is None else mu.ctypes.data, y.ctypes.data, float(s), int(n_iters), int(tag))
        rid = ctypes.c_uint64()
        _check(lib.spect_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(rid)))
        self._shapes[rid.value] = (geom.n, geom.n, geom.nz)
        del keep
        return rid.value

    def poll(self, rid: int) -> int:
        st = ctypes.c_int()
        _check(_serve_lib().spect_serve_poll(self.handle, rid, ctypes.byref(st)))
        return st.value

    def wait(self, rid: int, timeout_ms: int = 0):
        """(image [n][n][nz] float32, latency ms)."""
        import numpy as np
        x = np.empty(self._shapes[rid], dtype=np.float32)
        lat = ctypes.c_double()
        rc = _serve_lib().spect_serve_wait(self.handle, rid, int(timeout_ms), x.ctypes.data, ctypes.byref(lat))
        if rc != SPECT_ETIMEDOUT:
            self._shapes.pop(rid, None)
        _check(rc)
        return x, lat.value

    def cancel(self, rid: int) -> None:
        _check(_serve_lib().spect_serve_cancel(self.handle, rid))

    def stats(self) -> dict:
        st = _ServeStats()
        _check(_serve_lib().spect_serve_stats_get(self.handle, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in _ServeStats._fields_}

    def close(self) -> None:
        if getattr(self, "handle", None):
            _serve_lib().spect_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
