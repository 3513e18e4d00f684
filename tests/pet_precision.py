"""Lines of response whose integer decisions depend on the precision.

Joseph's method (Sec. 2.1.1, Eq. (2), P_Sigma) decides integers from
floating point: the principal axis, the range of planes and, with time of
flight, the window of samples that count.  The FP64 oracle takes them in
double precision, by definition.  The CUDA kernel takes the axis and the
plane range in single precision from the single-precision ends, and the
time-of-flight window as a range of sample indices computed in double
precision from its set-up values.  Where the two disagree (a rounding tie:
a line at 45 degrees between two axes, an end within single-precision
rounding of a voxel plane, a sample on the edge of the window) both are
valid samplings of the same line but their values differ, so the parity
tests leave those lines out and count them.

kernel_decisions restates the kernel's single-precision operations with
numpy float32 (every operation rounded to nearest like the kernel's); the
double-precision side is the oracle's own decision (oracle.pet.planes).
"""
import numpy as np


def kernel_decisions(lors, shape, voxel):
    """(axis, first plane, last plane, hit) per line, in the kernel's single precision."""
    L = np.asarray(lors, dtype=np.float32).reshape(-1, 6)
    p1, p2 = L[:, :3], L[:, 3:]
    v = np.asarray(voxel, dtype=np.float32)
    n = np.asarray(shape, dtype=np.int64)
    sc = np.abs(p2 - p1) / v
    rows = np.arange(len(L))
    a = np.where(sc[:, 1] > sc[:, 0], 1, 0)
    a = np.where(sc[:, 2] > sc[rows, a], 2, a)
    va = v[a]
    half = np.float32(0.5) * (n[a] - 1).astype(np.float32)
    org = -(half * va)
    s1 = (p1[rows, a] - org) / va
    s2 = (p2[rows, a] - org) / va
    lo = np.maximum(np.ceil(np.minimum(s1, s2)), np.float32(0.0))
    hi = np.minimum(np.floor(np.maximum(s1, s2)), (n[a] - 1).astype(np.float32))
    hit = (sc[rows, a] > 0) & (lo <= hi)
    return a, lo.astype(np.int64), hi.astype(np.int64), hit


def _tof_windows_agree(L, shape, voxel, a, q0, q1, tof):
    """Per line: the kernel's window [i0, i1] of sample indices (double
    precision, its operation order) equals the set of samples within
    nsigma sigma + width / 2 of the bin centre (the definition)."""
    nb, width, sigma, nsig, bins = tof
    v = np.asarray(voxel, dtype=np.float32).astype(np.float64)
    n = np.asarray(shape, dtype=np.float64)
    L64 = np.asarray(L, dtype=np.float32).astype(np.float64)
    org = (-0.5 * (n - 1)) * v
    e1 = (L64[:, :3] - org) / v
    e2 = (L64[:, 3:] - org) / v
    d = L64[:, 3:] - L64[:, :3]
    ln = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
    rows = np.arange(len(L))
    da = e2[rows, a] - e1[rows, a]
    cnt = q1 - q0 + 1
    width = float(np.float32(width))
    c = (np.asarray(bins, dtype=np.float64) - 0.5 * (nb - 1)) * width
    w = float(np.float32(nsig)) * float(np.float32(sigma)) + 0.5 * width
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (q0 - e1[rows, a]) / da
        l0 = (t0 - 0.5) * ln
        dl = ln / da
        lo = ((c - w) - l0) / dl
        hi = ((c + w) - l0) / dl
    lo, hi = np.where(dl < 0, hi, lo), np.where(dl < 0, lo, hi)
    lo = np.minimum(np.maximum(np.ceil(lo), 0.0), cnt)
    hi = np.maximum(np.minimum(np.floor(hi), cnt - 1), -1.0)
    ok = np.ones(len(L), dtype=bool)
    for e in range(len(L)):
        i = np.arange(cnt[e])
        ell = (((q0[e] + i) - e1[e, a[e]]) / da[e] - 0.5) * ln[e]
        inside = np.abs(ell - c[e]) <= w
        ok[e] = np.array_equal(inside, (i >= lo[e]) & (i <= hi[e]))
    return ok


def same_decisions(lors, og, opet, tof=None):
    """Boolean mask of the lines whose axis, planes (and, with `tof` =
    (n_bins, width_mm, sigma_mm, nsigma, bins), time-of-flight window) are
    the same in the kernel's precision and in the oracle's."""
    L = np.asarray(lors, dtype=np.float32).reshape(-1, 6)
    if len(L) == 0:
        return np.zeros(0, dtype=bool)
    a, q0, q1, hit = kernel_decisions(L, og.shape, og.voxel)
    ref = opet.planes(L.astype(np.float64), og)
    ref_hit = ref[:, 1] <= ref[:, 2]
    same = (hit == ref_hit) & (~hit | ((a == ref[:, 0]) & (q0 == ref[:, 1]) & (q1 == ref[:, 2])))
    if tof is not None:
        sel = same & hit
        idx = np.nonzero(sel)[0]
        if len(idx):
            bins = np.asarray(tof[4])[idx]
            ok = _tof_windows_agree(L[idx], og.shape, og.voxel, a[idx], q0[idx], q1[idx],
                                    tuple(tof[:4]) + (bins,))
            same[idx[~ok]] = False
    return same


def keep_alike(lors, og, opet, tof=None, max_frac=0.01):
    """same_decisions, asserting that the lines left out are few."""
    keep = same_decisions(lors, og, opet, tof)
    dropped = int((~keep).sum())
    print("lines left out (decisions differ between FP32 and FP64): %d of %d" % (dropped, len(keep)))
    assert dropped <= max(2, max_frac * len(keep))
    return keep
