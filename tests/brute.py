"""Independent dense construction of the SPECT system matrix for tiny sizes.

Built from library primitives only, so that it shares no arithmetic with the
oracle's hand-written loops:
  - T_rot: scipy.ndimage.affine_transform, order 1 (bilinear), mode
    'grid-constant' (taps outside the grid read 0);
  - T_att: numpy cumulative sums along depth and exp;
  - T_cdr: scipy.signal.windows.gaussian taps, normalised, applied with
    scipy.ndimage.correlate1d along the two detector axes, zero padding;
  - P_x: numpy sum over depth.
Eq. (1) of PyTomography (arXiv 2309.01977) fixes the order of the steps.
The dense H is assembled column by column from unit vectors.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage
from scipy.signal import windows


def rotate_lib(vol: np.ndarray, theta: float, shift: float = 0.0) -> np.ndarray:
    """Output voxel o = (i, j, k) reads the input at mat (o - centre - (0, shift, 0)) + centre:
    rotation about the centre of the rotated frame shifted by `shift` along j (T_trans T_rot)."""
    n = vol.shape[0]
    c = 0.5 * (n - 1)
    ct, st = math.cos(theta), math.sin(theta)
    mat = np.array([[ct, -st, 0.0], [st, ct, 0.0], [0.0, 0.0, 1.0]])
    centre = np.array([c, c, 0.0])
    offset = centre - mat @ (centre + np.array([0.0, shift, 0.0]))
    return ndimage.affine_transform(vol, mat, offset=offset, order=1, mode="grid-constant", cval=0.0)


def attenuation_lib(mu: np.ndarray, theta: float, voxel_cm: float, shift: float = 0.0) -> np.ndarray:
    tau = voxel_cm * rotate_lib(mu, theta, shift)
    suffix_incl = np.flip(np.cumsum(np.flip(tau, axis=0), axis=0), axis=0)   # sum_{i' >= i}
    beyond = suffix_incl - tau                                              # sum_{i' > i}
    return np.exp(-(beyond + 0.5 * tau))


def gaussian_taps_lib(sigma: float, nsigma: float) -> np.ndarray:
    r = int(math.ceil(nsigma * sigma))
    w = windows.gaussian(2 * r + 1, std=sigma, sym=True)
    return w / w.sum()


def forward_lib(f, theta, mu, voxel_cm, use_psf, sigma0, slope, nsigma, det_offset=0.0, shift=0.0, fov=None):
    n = f.shape[0]
    p = rotate_lib(f, theta, shift)
    if mu is not None:
        p = p * attenuation_lib(mu, theta, voxel_cm, shift)
    if use_psf:
        out = np.empty_like(p)
        for i in range(n):
            sigma = sigma0 + slope * (n - i - 0.5 + det_offset)
            w = gaussian_taps_lib(sigma, nsigma)
            q = ndimage.correlate1d(p[i], w, axis=1, mode="constant", cval=0.0)
            out[i] = ndimage.correlate1d(q, w, axis=0, mode="constant", cval=0.0)
        p = out
    proj = p.sum(axis=0)
    return proj if fov is None else proj * fov


def dense_h(n, nz, angles, mu, voxel_cm, use_psf, sigma0, slope, nsigma, det_offset=0.0,
            det_offsets=None, trans=None, fov=None) -> np.ndarray:
    """Dense H of shape [len(angles)*n*nz, n*n*nz] (rows: angle, bin y, bin z).
    det_offsets (optional): a detector offset per angle (non-circular orbit);
    trans (optional): a shift of the rotated frame per angle (T_trans);
    fov (optional): projection-space weights per angle [angle][n][nz] (T_fov)."""
    nvox = n * n * nz
    cols = []
    for q in range(nvox):
        e = np.zeros(nvox)
        e[q] = 1.0
        e = e.reshape(n, n, nz)
        col = [forward_lib(e, th, mu, voxel_cm, use_psf, sigma0, slope, nsigma,
                           det_offset if det_offsets is None else det_offsets[a],
                           0.0 if trans is None else trans[a], None if fov is None else fov[a]).ravel()
               for a, th in enumerate(angles)]
        cols.append(np.concatenate(col))
    return np.stack(cols, axis=1)
