"""ctypes front end of the FP64 listmode PET oracle (``pet_oracle.c``).

TEST INFRASTRUCTURE.  The plain definition of the PET system matrix of
PyTomography (arXiv 2309.01977), Sec. 2.1.1, Eq. (2): H = T_eta T_omega
P_Sigma T_rr with Joseph line integrals over a list of lines of response, its
transpose, and listmode OSEM (Table 1).  Only tests, the smoke check and the
benchmark's CPU legs may use it.  Readings where the paper is silent are
listed in ``pet_oracle.c``.

Pins (``tests/test_oracle_pet.py``): a dense system matrix built from scipy's
linear interpolation (``ndimage.map_coordinates``) at the plane samples;
chord lengths through a uniform box (axis-aligned and oblique lines);
exp(-mu L) through a uniform box; the Gaussian resolution model against
scipy's ``convolve1d`` with scipy window taps; <Hx, y> = <x, H^T y>;
listmode count conservation; listmode OSEM on repeated lines equal to the
binned MLEM step of the dense matrix.  Time of flight: a point source's
projection per bin against scipy's normal CDF; bins that cover the line add
up to the non-TOF projection; the dense TOF matrix from scipy routines; the
TOF listmode EM step against the binned MLEM step.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from .oracle import _f64, _load, _ptr

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_ready = False


def _lib():
    global _ready
    lib = _load()
    if not _ready:
        L, I = ctypes.c_long, ctypes.c_int
        D = ctypes.c_double
        lib.or_pet_planes.restype = None
        lib.or_pet_planes.argtypes = [_dp, L, I, I, I, _dp, _ip]
        lib.or_joseph_fwd.restype = None
        lib.or_joseph_fwd.argtypes = [_dp, I, I, I, _dp, _dp, L, _dp]
        lib.or_joseph_back.restype = None
        lib.or_joseph_back.argtypes = [_dp, _dp, L, I, I, I, _dp, _dp]
        lib.or_pet_rr_radius.restype = I
        lib.or_pet_rr_radius.argtypes = [D, D]
        lib.or_pet_rr_taps.restype = None
        lib.or_pet_rr_taps.argtypes = [D, D, _dp]
        lib.or_pet_blur.restype = None
        lib.or_pet_blur.argtypes = [_dp, I, I, I, _dp, D, D, _dp]
        lib.or_pet_mult.restype = None
        lib.or_pet_mult.argtypes = [_dp, I, I, I, _dp, _dp, L, _dp, _dp]
        lib.or_pet_forward.restype = None
        lib.or_pet_forward.argtypes = [_dp, I, I, I, _dp, D, D, _dp, _dp, L, _dp]
        lib.or_pet_back.restype = None
        lib.or_pet_back.argtypes = [_dp, I, I, I, _dp, D, D, _dp, _dp, L, _dp]
        lib.or_pet_set_tof.restype = None
        lib.or_pet_set_tof.argtypes = [I, D, D, D, _ip]
        lib.or_pet_lm_osem.restype = None
        lib.or_pet_lm_osem.argtypes = [_dp, _dp, _dp, L, _dp, I, I, I, _dp, D, D, I, _dp, I, I, _dp]
        _ready = True
    return lib


@dataclass
class PetGeom:
    """Image grid of the PET oracle.

    shape: (nx, ny, nz), z fastest; voxel: (vx, vy, vz) in mm; the image is
    centred on the scanner axis.  rr_sigma_mm: standard deviation of the
    Gaussian resolution model T_rr (0 = off); rr_nsigma: its truncation
    (radius ceil(nsigma * sigma / v) voxels per axis).
    """

    shape: Sequence[int]
    voxel: Sequence[float]
    rr_sigma_mm: float = 0.0
    rr_nsigma: float = 3.0

    def dims(self):
        nx, ny, nz = (int(v) for v in self.shape)
        self._v = _f64(self.voxel)
        return nx, ny, nz, _ptr(self._v)


@dataclass
class Tof:
    """Time-of-flight model: n_bins bins of bin_mm centred on the line's
    midpoint, Gaussian timing kernel of sigma_mm truncated at nsigma, and
    the bin index of every line."""

    n_bins: int
    bin_mm: float
    sigma_mm: float
    bins: Sequence[int]
    nsigma: float = 3.0


class _tof_scope:
    def __init__(self, tof: Optional[Tof]):
        self.tof = tof

    def __enter__(self):
        lib = _lib()
        if self.tof is None:
            lib.or_pet_set_tof(0, 0.0, 0.0, 0.0, ctypes.cast(None, _ip))
        else:
            self.bins = np.ascontiguousarray(np.asarray(self.tof.bins, dtype=np.int32))
            lib.or_pet_set_tof(int(self.tof.n_bins), float(self.tof.bin_mm), float(self.tof.sigma_mm),
                               float(self.tof.nsigma), self.bins.ctypes.data_as(_ip))
        return self

    def __exit__(self, *exc):
        _lib().or_pet_set_tof(0, 0.0, 0.0, 0.0, ctypes.cast(None, _ip))
        return False


def _lors(lors) -> np.ndarray:
    a = _f64(lors).reshape(-1, 6)
    return np.ascontiguousarray(a)


def planes(lors, g: PetGeom) -> np.ndarray:
    """[n][3] int: principal axis, first and last plane of each LOR."""
    L = _lors(lors)
    out = np.zeros((L.shape[0], 3), dtype=np.int32)
    _lib().or_pet_planes(_ptr(L), L.shape[0], *g.dims(), out.ctypes.data_as(_ip))
    return out


def joseph_fwd(f, lors, g: PetGeom, tof: Optional[Tof] = None) -> np.ndarray:
    f, L = _f64(f), _lors(lors)
    out = np.zeros(L.shape[0])
    with _tof_scope(tof):
        _lib().or_joseph_fwd(_ptr(f), *g.dims(), _ptr(L), L.shape[0], _ptr(out))
    return out


def joseph_back(vals, lors, g: PetGeom, tof: Optional[Tof] = None) -> np.ndarray:
    v, L = _f64(vals), _lors(lors)
    out = np.zeros(tuple(int(s) for s in g.shape))
    with _tof_scope(tof):
        _lib().or_joseph_back(_ptr(v), _ptr(L), L.shape[0], *g.dims(), _ptr(out))
    return out


def rr_taps(sigma_vox: float, nsigma: float = 3.0) -> np.ndarray:
    lib = _lib()
    r = lib.or_pet_rr_radius(float(sigma_vox), float(nsigma))
    w = np.zeros(2 * r + 1)
    lib.or_pet_rr_taps(float(sigma_vox), float(nsigma), _ptr(w))
    return w


def blur(f, g: PetGeom) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    _lib().or_pet_blur(_ptr(f), *g.dims(), float(g.rr_sigma_mm), float(g.rr_nsigma), _ptr(out))
    return out


def mult(lors, g: PetGeom, mu=None, eta=None) -> np.ndarray:
    """eta * exp(-(P_Sigma mu)) per LOR (mu in 1/mm)."""
    L = _lors(lors)
    m = None if mu is None else _f64(mu)
    e = None if eta is None else _f64(eta)
    out = np.zeros(L.shape[0])
    _lib().or_pet_mult(_ptr(m), *g.dims(), _ptr(L), L.shape[0], _ptr(e), _ptr(out))
    return out


def forward(f, lors, g: PetGeom, mult_: Optional[np.ndarray] = None, tof: Optional[Tof] = None) -> np.ndarray:
    """mult * (P_Sigma T_rr f) per LOR (time of flight when tof is given)."""
    f, L = _f64(f), _lors(lors)
    m = None if mult_ is None else _f64(mult_)
    out = np.zeros(L.shape[0])
    with _tof_scope(tof):
        _lib().or_pet_forward(_ptr(f), *g.dims(), float(g.rr_sigma_mm), float(g.rr_nsigma), _ptr(L), _ptr(m),
                              L.shape[0], _ptr(out))
    return out


def back(q, lors, g: PetGeom, mult_: Optional[np.ndarray] = None, tof: Optional[Tof] = None) -> np.ndarray:
    """T_rr P_Sigma^T (mult * q) (time of flight when tof is given)."""
    q, L = _f64(q), _lors(lors)
    m = None if mult_ is None else _f64(mult_)
    out = np.zeros(tuple(int(s) for s in g.shape))
    with _tof_scope(tof):
        _lib().or_pet_back(_ptr(q), *g.dims(), float(g.rr_sigma_mm), float(g.rr_nsigma), _ptr(L), _ptr(m),
                           L.shape[0], _ptr(out))
    return out


def lm_osem(lors, mult_, s, sens, g: PetGeom, n_subsets: int, x0=None, first: int = 0, count: int = 1,
            tof: Optional[Tof] = None):
    """Listmode OSEM (time of flight when tof is given); returns (image,
    diag [count][2]: sum p/(p+s), events used)."""
    L = _lors(lors)
    m = _f64(mult_)
    sv = None if s is None else _f64(np.broadcast_to(np.asarray(s, dtype=np.float64), (L.shape[0],)))
    sens = _f64(sens)
    x = np.ones(tuple(int(v) for v in g.shape)) if x0 is None else _f64(x0).copy()
    diag = np.zeros((count, 2))
    with _tof_scope(tof):
        _lib().or_pet_lm_osem(_ptr(L), _ptr(m), _ptr(sv), L.shape[0], _ptr(sens), *g.dims(), float(g.rr_sigma_mm),
                              float(g.rr_nsigma), int(n_subsets), _ptr(x), int(first), int(count), _ptr(diag))
    return x, diag
