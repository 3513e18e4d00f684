"""ctypes front end of the FP64 CPU oracle (``spect_oracle.c``).

TEST INFRASTRUCTURE.  This is the plain, slow definition of the parallel-hole
SPECT operator of PyTomography (arXiv 2309.01977), Sec. 2.1.1, Eq. (1), its
transpose, and OSEM with the Poisson gradient (Table 1).  Only tests, the smoke
check and the benchmark's CPU-baseline leg may use it.

Pins (all in ``tests/test_oracle_*.py``): brute-force dense H built from
scipy.ndimage library routines at 8^3; 90/180/270 degree rotations as exact
index permutations; rotation against scipy's bilinear affine transform;
exp(-mu L) through a uniform slab; PSF sum, centre and second moment against
the continuous Gaussian (sigma_i^2); <Hx, y> = <x, H^T y>; OSEM count
conservation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spect_oracle.c")
_SRC_PET = os.path.join(_HERE, "pet_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math).  Returns the .so path."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_PET))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, _SRC_PET, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.or_psf_rmax.restype = ctypes.c_int
            lib.or_psf_rmax.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4
            lib.or_psf_taps.restype = None
            lib.or_psf_taps.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [ctypes.c_int, _dp, _ip, _dp]
            lib.or_rotate.restype = None
            lib.or_rotate.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
            lib.or_rotate_adjoint.restype = None
            lib.or_rotate_adjoint.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
            lib.or_attenuation.restype = None
            lib.or_attenuation.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
            geom_args = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp, ctypes.c_int,
                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.or_forward.restype = None
            lib.or_forward.argtypes = [_dp] + geom_args + [_ip, ctypes.c_int, _dp]
            lib.or_back.restype = None
            lib.or_back.argtypes = [_dp] + geom_args + [_ip, ctypes.c_int, _dp]
            lib.or_osem.restype = None
            lib.or_osem.argtypes = [_dp, ctypes.c_double] + geom_args + [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                                         _dp, _dp]
            lib.or_poisson_ll.restype = ctypes.c_double
            lib.or_poisson_ll.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_size_t]
            lib.or_prior_value.restype = ctypes.c_double
            lib.or_prior_value.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.or_prior_grad.restype = None
            lib.or_prior_grad.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
            lib.or_set_orbit.restype = None
            lib.or_set_orbit.argtypes = [_dp, ctypes.c_int]
            lib.or_set_trans.restype = None
            lib.or_set_trans.argtypes = [_dp, ctypes.c_int]
            lib.or_set_fov.restype = None
            lib.or_set_fov.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.or_rotate_shift.restype = None
            lib.or_rotate_shift.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
            lib.or_rotate_adjoint_shift.restype = None
            lib.or_rotate_adjoint_shift.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                    _dp]
            lib.or_map.restype = None
            lib.or_map.argtypes = ([_dp, ctypes.c_double] + geom_args + [ctypes.c_int] * 5 +
                                   [ctypes.c_double] * 4 + [_dp])
            lib.or_n_threads.restype = ctypes.c_int
            lib.or_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.cast(None, _dp)
    return a.ctypes.data_as(_dp)


@dataclass
class Geom:
    """Acquisition geometry (voxel units unless stated).

    n: transaxial size (nx == ny); nz: axial size; n_angles: projections;
    angles: optional explicit angles in radians (default 2*pi*k/n_angles);
    voxel_cm: voxel edge (cm), scales mu into per-voxel optical depth;
    mu: optional attenuation map [n][n][nz] in 1/cm;
    use_psf: depth-dependent Gaussian blur on/off;
    sigma0, slope: sigma_i = sigma0 + slope * d_i with d_i = n - i - 0.5 + det_offset;
    nsigma: truncation radius R_i = ceil(nsigma * sigma_i);
    det_offsets: optional per-angle detector offsets (a non-circular orbit):
    d_i(a) = n - i - 0.5 + det_offsets[a] replaces det_offset for angle a.
    trans: optional per-angle shifts (voxels) of the rotated frame along the
    detector's transaxial axis (T_trans, non-central projections).
    fov: optional per-angle projection-space weights [n_angles][n][nz]
    (T_fov, the field-of-view mask).
    """

    n: int
    nz: int
    n_angles: int
    angles: Optional[Sequence[float]] = None
    voxel_cm: float = 0.48
    mu: Optional[np.ndarray] = None
    use_psf: bool = True
    sigma0: float = 0.5
    slope: float = 0.03
    nsigma: float = 3.0
    det_offset: float = 0.0
    det_offsets: Optional[Sequence[float]] = None
    trans: Optional[Sequence[float]] = None
    fov: Optional[np.ndarray] = None

    def _args(self):
        # the orbit, T_trans and T_fov travel through the oracle's module
        # state, set for every call
        orb = None if self.det_offsets is None else _f64(self.det_offsets)
        if orb is not None:
            assert orb.size == self.n_angles
        _load().or_set_orbit(_ptr(orb), int(self.n_angles))
        tr = None if self.trans is None else _f64(self.trans)
        if tr is not None:
            assert tr.size == self.n_angles
        _load().or_set_trans(_ptr(tr), int(self.n_angles))
        fv = None if self.fov is None else _f64(self.fov)
        if fv is not None:
            assert fv.shape == (self.n_angles, self.n, self.nz)
        _load().or_set_fov(_ptr(fv), int(self.n_angles), int(self.n), int(self.nz))
        self._keep_state = (orb, tr, fv)
        ang = None if self.angles is None else _f64(self.angles)
        mu = None if self.mu is None else _f64(self.mu).reshape(self.n, self.n, self.nz)
        self._keep = (ang, mu)  # keep the buffers alive for the call
        return (self.n, self.nz, self.n_angles, _ptr(ang), float(self.voxel_cm), _ptr(mu), int(bool(self.use_psf)),
                float(self.sigma0), float(self.slope), float(self.nsigma), float(self.det_offset))


def subset_angles(n_angles: int, n_subsets: int, m: int) -> list:
    """Subset S_m = {n : n mod M == m} in ascending order (interleaved subsets)."""
    return [a for a in range(n_angles) if a % n_subsets == m]


def n_threads() -> int:
    return _load().or_n_threads()


def set_threads(t: int) -> None:
    _load().or_set_threads(int(t))


def psf_rmax(n, sigma0=0.5, slope=0.03, nsigma=3.0, det_offset=0.0) -> int:
    return _load().or_psf_rmax(n, sigma0, slope, nsigma, det_offset)


def psf_taps(n, sigma0=0.5, slope=0.03, nsigma=3.0, det_offset=0.0):
    """Per-plane (sigma [n], radius [n], taps [n][2*rmax+1] centred at rmax)."""
    lib = _load()
    rmax = lib.or_psf_rmax(n, sigma0, slope, nsigma, det_offset)
    sig = np.zeros(n)
    rad = np.zeros(n, dtype=np.int32)
    taps = np.zeros((n, 2 * rmax + 1))
    lib.or_psf_taps(n, sigma0, slope, nsigma, det_offset, rmax, _ptr(sig), rad.ctypes.data_as(_ip), _ptr(taps))
    return sig, rad, taps


def rotate(f, theta: float, shift: float = 0.0) -> np.ndarray:
    """T_trans T_rot: bilinear rotation by theta, the rotated frame shifted by
    `shift` voxels along the detector's transaxial axis."""
    f = _f64(f)
    n, _, nz = f.shape
    out = np.empty_like(f)
    if shift == 0.0:
        _load().or_rotate(_ptr(f), n, nz, float(theta), _ptr(out))
    else:
        _load().or_rotate_shift(_ptr(f), n, nz, float(theta), float(shift), _ptr(out))
    return out


def rotate_adjoint(v, theta: float, shift: float = 0.0) -> np.ndarray:
    v = _f64(v)
    n, _, nz = v.shape
    out = np.empty_like(v)
    if shift == 0.0:
        _load().or_rotate_adjoint(_ptr(v), n, nz, float(theta), _ptr(out))
    else:
        _load().or_rotate_adjoint_shift(_ptr(v), n, nz, float(theta), float(shift), _ptr(out))
    return out


def attenuation(mu, theta: float, voxel_cm: float) -> np.ndarray:
    mu = _f64(mu)
    n, _, nz = mu.shape
    out = np.empty_like(mu)
    _load().or_attenuation(_ptr(mu), n, nz, float(theta), float(voxel_cm), _ptr(out))
    return out


def _sel(g: Geom, sel):
    if sel is None:
        sel = range(g.n_angles)
    s = np.ascontiguousarray(np.asarray(list(sel), dtype=np.int32))
    if s.size and (s.min() < 0 or s.max() >= g.n_angles):
        raise ValueError("angle index out of range")
    return s


def forward(f, g: Geom, sel=None) -> np.ndarray:
    """H f restricted to angles ``sel`` (default all): [len(sel)][n][nz]."""
    f = _f64(f).reshape(g.n, g.n, g.nz)
    s = _sel(g, sel)
    out = np.zeros((len(s), g.n, g.nz))
    _load().or_forward(_ptr(f), *g._args(), s.ctypes.data_as(_ip), len(s), _ptr(out))
    return out


def back(proj, g: Geom, sel=None) -> np.ndarray:
    """H^T proj restricted to angles ``sel``: [n][n][nz]."""
    s = _sel(g, sel)
    proj = _f64(proj).reshape(len(s), g.n, g.nz)
    out = np.zeros((g.n, g.n, g.nz))
    _load().or_back(_ptr(proj), *g._args(), s.ctypes.data_as(_ip), len(s), _ptr(out))
    return out


def osem(y, s: float, g: Geom, n_subsets: int, first: int, count: int, f0=None):
    """Run OSEM subiterations first..first+count-1 from f0 (default ones).

    Returns (f, diag) with diag [count][3] = sums over the subset's bins of
    (H_m f + s), y and y * H_m f / (H_m f + s), taken before each update.
    """
    y = _f64(y).reshape(g.n_angles, g.n, g.nz)
    f = np.ones((g.n, g.n, g.nz)) if f0 is None else _f64(f0).reshape(g.n, g.n, g.nz).copy()
    diag = np.zeros((max(count, 0), 3))
    _load().or_osem(_ptr(y), float(s), *g._args(), int(n_subsets), int(first), int(count), _ptr(f), _ptr(diag))
    return f, diag


def poisson_ll(y, p, s: float) -> float:
    """Poisson log-likelihood sum y log(p+s) - (p+s) (log y! dropped)."""
    y = _f64(y).ravel()
    p = _f64(p).ravel()
    assert y.size == p.size
    return _load().or_poisson_ll(_ptr(y), _ptr(p), float(s), y.size)


PRIORS = {"none": 0, "quadratic": 1, "rdp": 2}
ALGORITHMS = {"osmaposl": 1, "bsrem": 2}


def prior_value(f, prior: str, delta: float = 1.0, gamma: float = 2.0) -> float:
    """V(f) = sum_r sum_s w_rs phi(f_r, f_s) over 26-neighbourhoods, w = 1/distance (Table 1)."""
    f = _f64(f)
    n, n2, nz = f.shape
    assert n == n2
    return _load().or_prior_value(_ptr(f), n, nz, PRIORS[prior], float(delta), float(gamma))


def prior_grad(f, prior: str, delta: float = 1.0, gamma: float = 2.0):
    """dV/df for the prior of prior_value."""
    f = _f64(f)
    n, n2, nz = f.shape
    assert n == n2
    g = np.zeros_like(f)
    _load().or_prior_grad(_ptr(f), n, nz, PRIORS[prior], float(delta), float(gamma), _ptr(g))
    return g


def map_recon(y, s: float, g: Geom, n_subsets: int, first: int, count: int, algorithm: str, prior: str,
              beta: float, delta: float = 1.0, gamma: float = 2.0, alpha0: float = 1.0, f0=None):
    """OSMAPOSL or BSREM subiterations first..first+count-1 (Eq. PGA, Table 1) from f0 (default ones)."""
    y = _f64(y).reshape(g.n_angles, g.n, g.nz)
    f = np.ones((g.n, g.n, g.nz)) if f0 is None else _f64(f0).reshape(g.n, g.n, g.nz).copy()
    _load().or_map(_ptr(y), float(s), *g._args(), int(n_subsets), int(first), int(count), ALGORITHMS[algorithm],
                   PRIORS[prior], float(beta), float(delta), float(gamma), float(alpha0), _ptr(f))
    return f



def osem_multi(ys, ss, geoms, scales, n_subsets: int, first: int, count: int, f0=None):
    """OSEM for a multi-photopeak extended system matrix (Sec. 2.1.1, Eq.
    extended_sm): H' = sum_n v_n (x) a_n H_n, one system matrix H_n per peak
    (its own attenuation map and PSF) scaled by a_n (detector sensitivity and
    branching ratio), B_n the identity.  With the Poisson gradient of Table 1
    for the stacked data, each subiteration is
        r_n = y_n / (a_n H_n,m f + s_n),
        f <- f * (sum_n a_n H_n,m^T r_n) / (sum_n a_n H_n,m^T 1)   (unchanged where the sum is 0).
    Built from the FP64 forward and back projections of each peak."""
    f = np.ones((geoms[0].n, geoms[0].n, geoms[0].nz)) if f0 is None else _f64(f0).copy()
    for t in range(first, first + count):
        sel = subset_angles(geoms[0].n_angles, n_subsets, t % n_subsets)
        bp = np.zeros_like(f)
        sens = np.zeros_like(f)
        for y, s, g, a in zip(ys, ss, geoms, scales):
            p = a * forward(f, g, sel)
            den = p + s
            yv = _f64(y).reshape(g.n_angles, g.n, g.nz)[sel]
            r = np.where(den > 0, yv / np.where(den > 0, den, 1.0), 0.0)
            bp += a * back(r, g, sel)
            sens += a * back(np.ones_like(r), g, sel)
        pos = sens > 0
        f = np.where(pos, f * bp / np.where(pos, sens, 1.0), f)
    return f
