"""Host-side checks of the tiled gather's strip-list layout (no GPU).

The tiled gather (csrc/gather_tiled.cu) gives each row y of an 8 x 8 output
tile nine lists of rotated-grid samples, keyed by the sample's lower
bilinear column xa, with kGtMaxList fixed slots per list.  Two facts carry
that layout:

* a list holds the samples with a given xa and ya in {y - 1, y}: a 1 x 2
  cell of the rotated unit grid, which holds at most three samples, so
  three slots suffice (a plan whose tables would need more falls back to
  the per-column gather);
* adding each sample of list xa to column xa with weight (1 - ax) wy and to
  column xa + 1 with ax wy, over the nine lists of a row, is the transpose
  of bilinear interpolation (T_rot of Eq. 1) restricted to that row.

Both are checked here on the geometry alone, in float32 sample points
formed as the kernels form them.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _constant(name: str) -> int:
    text = open(os.path.join(ROOT, "paper_2309_01977_gb300", "csrc", "internal.h")).read()
    m = re.search(r"constexpr int %s = (\d+);" % name, text)
    assert m, name
    return int(m.group(1))


def _sample_points(n: int, theta: float, shift: float = 0.0):
    """u, v of every rotated-frame sample (i, j), float32 as in sample_point:
    u = c + cos (i - c) - sin (j - cj), v = c + sin (i - c) + cos (j - cj)."""
    f = np.float32
    c = f(0.5 * (n - 1))
    ct, st = f(np.cos(theta)), f(np.sin(theta))
    cj = f(0.5 * (n - 1) + shift)
    i, j = np.meshgrid(np.arange(n, dtype=np.float32), np.arange(n, dtype=np.float32), indexing="ij")
    di, dj = (i - c).astype(np.float32), (j - cj).astype(np.float32)
    u = (c + ct * di - st * dj).astype(np.float32)
    v = (c + st * di + ct * dj).astype(np.float32)
    return u, v


@pytest.mark.parametrize("n", [32, 64, 96, 128, 132, 256])
def test_a_list_never_needs_more_than_its_slots(n):
    slots = _constant("kGtMaxList")
    rng = np.random.Generator(np.random.PCG64(n))
    thetas = np.concatenate([2 * np.pi * np.arange(180) / 180, rng.uniform(0, 2 * np.pi, 60)])
    worst = 0
    for k, th in enumerate(thetas):
        shift = float(rng.uniform(-4, 4)) if k % 3 == 0 else 0.0
        u, v = _sample_points(n, th, shift)
        xa = np.floor(u).astype(np.int64) + 2
        ya = np.floor(v).astype(np.int64) + 2
        keep = (xa >= 0) & (xa < n + 4) & (ya >= 0) & (ya < n + 4)
        cells = np.zeros((n + 5, n + 5), dtype=np.int64)
        np.add.at(cells, (xa[keep], ya[keep]), 1)
        pairs = cells[:, 1:] + cells[:, :-1]  # ya in {y - 1, y}
        worst = max(worst, int(pairs.max()))
    assert worst <= slots, "a 1 x 2 cell held %d samples, more than the %d list slots" % (worst, slots)


def _bilinear_transpose(b, u, v, n):
    """x[q] = sum over samples p of w_pq b[p]: the scatter form of the
    transpose of bilinear interpolation at the points (u, v)."""
    x = np.zeros((n, n))
    fu, fv = np.floor(u), np.floor(v)
    ax, by = (u - fu).astype(np.float64), (v - fv).astype(np.float64)
    xa, ya = fu.astype(int), fv.astype(int)
    for dx, wx in ((0, 1 - ax), (1, ax)):
        for dy, wy in ((0, 1 - by), (1, by)):
            xs, ys = xa + dx, ya + dy
            m = (xs >= 0) & (xs < n) & (ys >= 0) & (ys < n)
            np.add.at(x, (xs[m], ys[m]), (wx * wy * b)[m])
    return x


def _strip_gather(b, u, v, n, T=8):
    """The same sums through per-row strip lists, as the tiled gather forms
    them: tile row y, list of lower column xa, weights to xa and xa + 1."""
    x = np.zeros((n, n))
    fu, fv = np.floor(u).ravel(), np.floor(v).ravel()
    ax = (u.ravel() - fu).astype(np.float64)
    by = (v.ravel() - fv).astype(np.float64)
    xa, ya, bb = fu.astype(int), fv.astype(int), b.ravel()
    for y in range(n):
        wy = np.where(ya == y, 1 - by, np.where(ya + 1 == y, by, 0.0))
        for tx in range((n + T - 1) // T):
            for l in range(T + 1):  # list l: lower column tx T + l - 1
                col = tx * T + l - 1
                m = (xa == col) & (wy != 0)
                if not m.any():
                    continue
                if l >= 1 and col < n:
                    x[col, y] += np.sum((1 - ax[m]) * wy[m] * bb[m])
                if l + 1 <= T and col + 1 < n:
                    x[col + 1, y] += np.sum(ax[m] * wy[m] * bb[m])
    return x


@pytest.mark.parametrize("n, theta", [(24, 0.3), (24, 2.0), (20, 4.1)])
def test_strip_lists_are_the_bilinear_transpose(n, theta):
    u, v = _sample_points(n, theta)
    b = np.random.Generator(np.random.PCG64(7)).uniform(0.5, 1.5, size=(n, n))
    ref = _bilinear_transpose(b, u, v, n)
    got = _strip_gather(b, u, v, n)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_table_slices_are_whole_bulk_copies():
    """The issuing warp moves each (angle, tile) strip table and footprint
    descriptor with one cp.async.bulk: sizes and offsets must be multiples
    of 16 bytes, and a footprint row per lane must cover a descriptor."""
    text = open(os.path.join(ROOT, "paper_2309_01977_gb300", "csrc", "internal.h")).read()
    assert "constexpr int kGtLists = kGtT + 1;" in text
    T, hdr, slots = _constant("kGtT"), _constant("kGtHdr"), _constant("kGtMaxList")
    slice_bytes = T * hdr * 4 + T * (T + 1) * slots * 16
    assert slice_bytes % 16 == 0
    assert (T * hdr * 4) % 16 == 0  # entries start 16-byte aligned
    assert hdr >= T + 1
    desc_ints = 4 + 2 * _constant("kFpMaxRows")
    assert (desc_ints * 4) % 16 == 0
    assert _constant("kFpMaxRows") == 32  # one footprint row per lane of the issuing warp
