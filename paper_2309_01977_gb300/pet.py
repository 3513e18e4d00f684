"""ctypes binding of the listmode PET calls of libspect.so (include/pet.h).

Argument marshalling only: every step runs in the library's CUDA kernels and
a missing library raises.  H = T_eta T_omega P_Sigma T_rr (Sec. 2.1.1,
Eq. (2)) with Joseph line integrals over lines of response (6 floats each:
both ends in mm), and listmode OSEM (Table 1).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import spect
from .spect import SPECT_EINVAL, SpectError, _check, _dptr, _KernelTime, _stream

# Every symbol include/pet.h declares (checked by the CPU test suite).
PET_EXPORTED = ["pet_plan_create", "pet_plan_destroy", "pet_mult", "pet_forward", "pet_back", "pet_lm_osem_run",
                "pet_profile_enable", "pet_profile_read"]


class _PetGeom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("vx", ctypes.c_float), ("vy", ctypes.c_float), ("vz", ctypes.c_float),
                ("rr_sigma_mm", ctypes.c_float), ("rr_nsigma", ctypes.c_float), ("n_subsets", ctypes.c_int),
                ("n_tof_bins", ctypes.c_int), ("tof_bin_mm", ctypes.c_float), ("tof_sigma_mm", ctypes.c_float),
                ("tof_nsigma", ctypes.c_float)]


_ready = False


def load() -> ctypes.CDLL:
    global _ready
    lib = spect.load()
    if not _ready:
        vp, i, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.pet_plan_create.argtypes = [ctypes.POINTER(_PetGeom), vp, vp, ctypes.POINTER(vp)]
        lib.pet_plan_destroy.argtypes = [vp]
        lib.pet_mult.argtypes = [vp, vp, vp, L, vp, vp]
        lib.pet_forward.argtypes = [vp, vp, vp, vp, vp, L, vp, vp]
        lib.pet_back.argtypes = [vp, vp, vp, vp, vp, L, vp, vp]
        lib.pet_lm_osem_run.argtypes = [vp, vp, vp, vp, vp, L, vp, vp, i, i, ctypes.POINTER(ctypes.c_double), vp]
        lib.pet_profile_enable.argtypes = [vp, i]
        lib.pet_profile_read.argtypes = [vp, ctypes.POINTER(_KernelTime), i, i]
        _ready = True
    return lib


@dataclass
class PetGeometry:
    """Image grid: shape (nx, ny, nz), z fastest; voxel sizes in mm; T_rr
    Gaussian standard deviation in mm (0 = off) and truncation; subsets;
    time of flight: bins (0 = off), bin width, kernel sigma (mm), truncation."""

    shape: Sequence[int]
    voxel: Sequence[float]
    rr_sigma_mm: float = 0.0
    rr_nsigma: float = 3.0
    n_subsets: int = 1
    n_tof_bins: int = 0
    tof_bin_mm: float = 0.0
    tof_sigma_mm: float = 0.0
    tof_nsigma: float = 3.0

    def to_c(self) -> _PetGeom:
        nx, ny, nz = (int(v) for v in self.shape)
        vx, vy, vz = (float(v) for v in self.voxel)
        return _PetGeom(nx, ny, nz, vx, vy, vz, float(self.rr_sigma_mm), float(self.rr_nsigma), int(self.n_subsets),
                        int(self.n_tof_bins), float(self.tof_bin_mm), float(self.tof_sigma_mm),
                        float(self.tof_nsigma))


def _lors(lors: torch.Tensor) -> int:
    if lors.dim() != 2 or lors.shape[1] != 6:
        raise SpectError(SPECT_EINVAL, "lors must be [n][6]")
    return lors.shape[0]


def _bins(tof_bin: Optional[torch.Tensor], n: int):
    if tof_bin is None:
        return None
    if tof_bin.numel() != n:
        raise SpectError(SPECT_EINVAL, "tof_bin needs one bin per line")
    return _dptr(tof_bin, torch.int32)


class PetPlan:
    """A listmode PET plan (owns the library handle)."""

    def __init__(self, geom: PetGeometry, mu: Optional[torch.Tensor] = None, stream=None):
        self.geom = geom
        self.shape = tuple(int(v) for v in geom.shape)
        if mu is not None and tuple(mu.shape) != self.shape:
            raise SpectError(SPECT_EINVAL, "mu must have the image shape")
        g = geom.to_c()
        out = ctypes.c_void_p()
        _check(load().pet_plan_create(ctypes.byref(g), _dptr(mu), _stream(stream), ctypes.byref(out)))
        self.handle = out.value

    def close(self):
        if self.handle:
            load().pet_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _img(self, x: torch.Tensor, what: str) -> int:
        if tuple(x.shape) != self.shape:
            raise SpectError(SPECT_EINVAL, "%s must have the image shape %s" % (what, self.shape))
        return _dptr(x)

    def mult(self, lors: torch.Tensor, eta: Optional[torch.Tensor] = None, out=None, stream=None) -> torch.Tensor:
        n = _lors(lors)
        out = torch.empty(n, device=lors.device) if out is None else out
        _check(load().pet_mult(self.handle, _dptr(lors), _dptr(eta), n, _dptr(out), _stream(stream)))
        return out

    def forward(self, x: torch.Tensor, lors: torch.Tensor, mult: Optional[torch.Tensor] = None,
                tof_bin: Optional[torch.Tensor] = None, out=None, stream=None) -> torch.Tensor:
        n = _lors(lors)
        out = torch.empty(n, device=lors.device) if out is None else out
        _check(load().pet_forward(self.handle, self._img(x, "x"), _dptr(lors), _dptr(mult), _bins(tof_bin, n), n,
                                  _dptr(out), _stream(stream)))
        return out

    def back(self, q: torch.Tensor, lors: torch.Tensor, mult: Optional[torch.Tensor] = None,
             tof_bin: Optional[torch.Tensor] = None, out=None, stream=None) -> torch.Tensor:
        n = _lors(lors)
        out = torch.empty(self.shape, device=lors.device) if out is None else out
        _check(load().pet_back(self.handle, _dptr(q), _dptr(lors), _dptr(mult), _bins(tof_bin, n), n,
                               self._img(out, "x_out"), _stream(stream)))
        return out

    def lm_osem(self, lors: torch.Tensor, mult: torch.Tensor, s: Optional[torch.Tensor], sens: torch.Tensor,
                x: torch.Tensor, first: int, count: int, diag: bool = False, tof_bin: Optional[torch.Tensor] = None,
                stream=None):
        """Listmode OSEM subiterations in place on x (time of flight when
        tof_bin is given); returns the FP64 diagnostics [count][2] (sum
        p/(p+s), events used) when diag is set."""
        n = _lors(lors)
        buf = (ctypes.c_double * (2 * max(count, 1)))() if diag else None
        _check(load().pet_lm_osem_run(self.handle, _dptr(lors), _dptr(mult), _dptr(s), _bins(tof_bin, n), n,
                                      self._img(sens, "sens"), self._img(x, "x"), int(first), int(count), buf,
                                      _stream(stream)))
        if diag:
            return [(buf[2 * k], buf[2 * k + 1]) for k in range(count)]
        return None

    def profile_enable(self, on: bool = True):
        _check(load().pet_profile_enable(self.handle, int(bool(on))))

    def profile_read(self, reset: bool = False) -> dict:
        buf = (_KernelTime * 16)()
        n = _check(load().pet_profile_read(self.handle, buf, 16, int(bool(reset))))
        return {buf[k].name.decode(): (int(buf[k].launches), float(buf[k].total_ms)) for k in range(n)}
