"""Dense listmode PET system matrix built from library routines, for pinning
the FP64 oracle (tests only).

Joseph's method (Sec. 2.1.1, Eq. (2), P_Sigma) restated in numpy: per line
of response the principal axis and the sampled voxel planes are decided in
double precision, the sample points are placed in double precision, and
the image is read at them with scipy's linear
interpolation (``ndimage.map_coordinates``, order 1, zero outside the grid
tap by tap), weighted by the line's length between planes.  T_rr is applied
with ``ndimage.convolve1d`` and taps from ``signal.windows.gaussian``.
"""
import numpy as np
from scipy import ndimage
from scipy.signal import windows
from scipy.stats import norm


def decisions(lor, shape, voxel):
    """Principal axis (largest |d_c| / v_c, ties to the lower axis) and the
    planes of that axis between the ends, clipped to the image."""
    lor = np.asarray(lor, dtype=np.float64)
    v = np.asarray(voxel, dtype=np.float64)
    sc = np.abs(lor[3:] - lor[:3]) / v
    a = 0
    for c in (1, 2):
        if sc[c] > sc[a]:
            a = c
    if not sc[a] > 0:
        return a, 1, 0
    org = -0.5 * (shape[a] - 1) * v[a]
    s1 = (lor[a] - org) / v[a]
    s2 = (lor[3 + a] - org) / v[a]
    lo = max(np.ceil(min(s1, s2)), 0.0)
    hi = min(np.floor(max(s1, s2)), float(shape[a] - 1))
    if lo > hi:
        return a, 1, 0
    return a, int(lo), int(hi)


def samples(lor, shape, voxel):
    """Index-space sample points [k][3] and the step length of one LOR."""
    a, q0, q1 = decisions(lor, shape, voxel)
    if q0 > q1:
        return np.zeros((0, 3)), 0.0
    lor = np.asarray(lor, dtype=np.float64)
    v = np.asarray(voxel, dtype=np.float64)
    org = -0.5 * (np.asarray(shape) - 1) * v
    e1 = (lor[:3] - org) / v
    e2 = (lor[3:] - org) / v
    d = lor[3:] - lor[:3]
    step = v[a] * np.linalg.norm(d) / abs(d[a])
    q = np.arange(q0, q1 + 1, dtype=np.float64)
    t = (q - e1[a]) / (e2[a] - e1[a])
    pts = e1[None, :] + t[:, None] * (e2 - e1)[None, :]
    pts[:, a] = q  # exactly on the plane
    return pts, step


def tof_weights(lor, shape, voxel, tof, b):
    """Timing weights of one line's samples for TOF bin b (tof = (n_bins,
    bin_mm, sigma_mm, nsigma)): the Gaussian integrated over the bin, by
    scipy's normal CDF, for samples within nsigma sigma + width / 2 of the
    bin centre, else 0."""
    nb, width, sigma, nsig = tof
    a, q0, q1 = decisions(lor, shape, voxel)
    lor = np.asarray(lor, dtype=np.float64)
    v = np.asarray(voxel, dtype=np.float64)
    org = -0.5 * (np.asarray(shape) - 1) * v
    e1 = (lor[:3] - org) / v
    e2 = (lor[3:] - org) / v
    ln = np.linalg.norm(lor[3:] - lor[:3])
    q = np.arange(q0, q1 + 1, dtype=np.float64)
    ell = ((q - e1[a]) / (e2[a] - e1[a]) - 0.5) * ln
    c = (b - 0.5 * (nb - 1)) * width
    wt = norm.cdf((ell - c + 0.5 * width) / sigma) - norm.cdf((ell - c - 0.5 * width) / sigma)
    return np.where(np.abs(ell - c) <= nsig * sigma + 0.5 * width, wt, 0.0)


def joseph(f, lors, voxel, tof=None, bins=None):
    f = np.asarray(f, dtype=np.float64)
    out = np.zeros(len(lors))
    for e, lor in enumerate(lors):
        pts, step = samples(lor, f.shape, voxel)
        if len(pts):
            vals = ndimage.map_coordinates(f, pts.T, order=1, mode="grid-constant", cval=0.0, prefilter=False)
            if tof is not None:
                vals = vals * tof_weights(lor, f.shape, voxel, tof, bins[e])
            out[e] = step * vals.sum()
    return out


def dense(lors, shape, voxel, tof=None, bins=None):
    """[n_lors][nvox] matrix of P_Sigma (from unit images)."""
    nvox = int(np.prod(shape))
    H = np.zeros((len(lors), nvox))
    for vx in range(nvox):
        b = np.zeros(nvox)
        b[vx] = 1.0
        H[:, vx] = joseph(b.reshape(shape), lors, voxel, tof, bins)
    return H


def gaussian_blur(f, voxel, sigma_mm, nsigma=3.0):
    out = np.asarray(f, dtype=np.float64)
    if not sigma_mm > 0:
        return out.copy()
    for ax in range(3):
        s = sigma_mm / voxel[ax]
        r = int(np.ceil(nsigma * s))
        w = windows.gaussian(2 * r + 1, std=s)
        w = w / w.sum()
        out = ndimage.convolve1d(out, w, axis=ax, mode="constant", cval=0.0)
    return out


def dense_blur(shape, voxel, sigma_mm, nsigma=3.0):
    nvox = int(np.prod(shape))
    B = np.zeros((nvox, nvox))
    for vx in range(nvox):
        b = np.zeros(nvox)
        b[vx] = 1.0
        B[:, vx] = gaussian_blur(b.reshape(shape), voxel, sigma_mm, nsigma).ravel()
    return B
