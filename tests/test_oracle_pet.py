"""Pins of the FP64 listmode PET oracle (Sec. 2.1.1, Eq. (2); Table 1), CPU only.

Each pin is independent of the oracle's code: a dense matrix from scipy's
linear interpolation, closed-form chord lengths and exp(-mu L), scipy's 1-D
convolution, the adjoint identity, count conservation of the listmode EM
step and the binned MLEM step of a dense matrix.
"""
import numpy as np
import pytest

import pet_brute

pet = pytest.importorskip("oracle.pet")

SHAPE = (5, 6, 7)
VOXEL = (2.0, 1.5, 2.5)


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def mixed_lors(seed, count=60, shape=SHAPE, voxel=VOXEL):
    """Lines of every kind: endpoints on a sphere outside the image, inside
    it, axis-parallel, steep in z, and endpoints exactly on voxel planes."""
    rng = _rng(seed)
    ext = 0.5 * np.asarray(shape) * np.asarray(voxel)
    R = 2.0 * np.linalg.norm(ext)
    out = []
    for i in range(count):
        kind = i % 5
        if kind == 0:
            u = rng.normal(size=(2, 3))
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            p = (u * R).ravel()
        elif kind == 1:
            p = rng.uniform(-ext, ext, size=(2, 3)).ravel()
        elif kind == 2:
            ax = rng.integers(3)
            c = rng.uniform(-ext, ext)
            a, b = c.copy(), c.copy()
            a[ax], b[ax] = -R, R
            p = np.concatenate([a, b])
        elif kind == 3:
            c = rng.uniform(-0.5 * ext, 0.5 * ext, size=3)
            d = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 1.0])
            p = np.concatenate([c - R * d, c + R * d])
        else:
            ax = rng.integers(3)
            org = -0.5 * (shape[ax] - 1) * voxel[ax]
            a = rng.uniform(-ext, ext)
            b = rng.uniform(-ext, ext)
            a[ax] = org + voxel[ax] * rng.integers(shape[ax])
            b[ax] = org + voxel[ax] * rng.integers(shape[ax])
            if a[ax] == b[ax]:
                b[ax] = R
            p = np.concatenate([a, b])
        out.append(p)
    return _f32(np.array(out))


def test_planes_match_double_precision_reading():
    lors = mixed_lors(1)
    g = pet.PetGeom(SHAPE, VOXEL)
    got = pet.planes(lors, g)
    for e, lor in enumerate(lors):
        a, q0, q1 = pet_brute.decisions(lor, SHAPE, VOXEL)
        if q0 <= q1:
            assert tuple(got[e]) == (a, q0, q1)
        else:
            assert got[e][1] > got[e][2]


def test_joseph_equals_scipy_linear_interpolation():
    lors = mixed_lors(2)
    g = pet.PetGeom(SHAPE, VOXEL)
    f = _rng(3).uniform(0.0, 2.0, size=SHAPE)
    ref = pet_brute.joseph(f, lors, VOXEL)
    got = pet.joseph_fwd(f, lors, g)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    assert np.count_nonzero(ref) > len(lors) // 2


def test_joseph_back_is_dense_transpose():
    lors = mixed_lors(4, count=40)
    g = pet.PetGeom(SHAPE, VOXEL)
    H = pet_brute.dense(lors, SHAPE, VOXEL)
    v = _rng(5).normal(size=len(lors))
    got = pet.joseph_back(v, lors, g).ravel()
    ref = H.T @ v
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_axis_line_through_uniform_box_is_its_length():
    shape, voxel, c = (8, 9, 10), (2.0, 3.0, 1.5), 1.7
    g = pet.PetGeom(shape, voxel)
    f = np.full(shape, c)
    org = -0.5 * (np.asarray(shape) - 1) * np.asarray(voxel)
    # along x through the centre line of voxel row (j=3, k=4); along y and z too
    y3, z4 = org[1] + 3 * voxel[1], org[2] + 4 * voxel[2]
    x2 = org[0] + 2 * voxel[0]
    lors = np.array([[-100.0, y3, z4, 100.0, y3, z4],
                     [x2, -100.0, z4, x2, 100.0, z4],
                     [x2, y3, -100.0, x2, y3, 100.0],
                     # starting exactly on plane 2 of x: planes 2..7 count
                     [x2, y3, z4, 100.0, y3, z4]])
    got = pet.joseph_fwd(f, _f32(lors), g)
    want = c * np.array([8 * 2.0, 9 * 3.0, 10 * 1.5, 6 * 2.0])
    assert np.allclose(got, want, rtol=1e-13, atol=0)


def test_oblique_line_through_uniform_slab_is_chord_length():
    shape, voxel, c = (12, 64, 4), (2.0, 2.0, 2.0), 0.8
    g = pet.PetGeom(shape, voxel)
    f = np.full(shape, c)
    for dy in (10.0, 37.0, 80.0):
        lor = np.array([[-100.0, -dy / 2, 0.0, 100.0, dy / 2, 0.0]])
        got = pet.joseph_fwd(f, lor, g)[0]
        chord = shape[0] * voxel[0] * np.hypot(200.0, dy) / 200.0
        assert abs(got - c * chord) <= 1e-12 * chord


def test_attenuation_factor_through_uniform_box():
    shape, voxel, mu = (10, 6, 6), (2.0, 2.0, 2.0), 0.0096
    g = pet.PetGeom(shape, voxel)
    lor = np.array([[-300.0, 1.0, 1.0, 300.0, 1.0, 1.0]])
    m = pet.mult(lor, g, mu=np.full(shape, mu), eta=np.array([0.9]))
    assert abs(m[0] - 0.9 * np.exp(-mu * 10 * 2.0)) <= 1e-15


def test_resolution_model_matches_scipy_convolution():
    shape, voxel = (9, 10, 11), (1.25, 1.25, 2.0)
    f = _rng(6).uniform(size=shape)
    for sigma in (0.0, 1.274, 2.9):
        g = pet.PetGeom(shape, voxel, rr_sigma_mm=sigma)
        got = pet.blur(f, g)
        ref = pet_brute.gaussian_blur(f, voxel, sigma)
        assert np.max(np.abs(got - ref)) <= 1e-13


def test_resolution_taps_moments():
    for s in (0.6, 1.02, 2.5):
        w = pet.rr_taps(s)
        r = (len(w) - 1) // 2
        t = np.arange(-r, r + 1)
        assert r == int(np.ceil(3 * s))
        assert abs(w.sum() - 1.0) <= 1e-15
        assert abs((w * t).sum()) <= 1e-15
        # second moment of the truncated sampled Gaussian: within the
        # truncation factor of sigma^2 (3-sigma truncation removes < 3 %)
        m2 = (w * t * t).sum()
        assert 0.95 * s * s <= m2 <= 1.0 * s * s + 1.0 / 12.0


def test_system_matrix_adjoint():
    lors = mixed_lors(7, count=50)
    g = pet.PetGeom(SHAPE, VOXEL, rr_sigma_mm=1.8)
    rng = _rng(8)
    f = rng.uniform(size=SHAPE)
    q = rng.normal(size=len(lors))
    m = rng.uniform(0.5, 1.0, size=len(lors))
    lhs = np.dot(pet.forward(f, lors, g, m), q)
    rhs = np.sum(f * pet.back(q, lors, g, m))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_forward_equals_dense_composition():
    lors = mixed_lors(9, count=30)
    g = pet.PetGeom(SHAPE, VOXEL, rr_sigma_mm=1.8)
    rng = _rng(10)
    f = rng.uniform(size=SHAPE)
    m = rng.uniform(0.5, 1.0, size=len(lors))
    H = m[:, None] * (pet_brute.dense(lors, SHAPE, VOXEL) @ pet_brute.dense_blur(SHAPE, VOXEL, 1.8))
    assert np.allclose(pet.forward(f, lors, g, m), H @ f.ravel(), rtol=0, atol=1e-12)


def _em_case(seed, s_val):
    rng = _rng(seed)
    lines = mixed_lors(seed, count=25)
    g = pet.PetGeom(SHAPE, VOXEL, rr_sigma_mm=1.5)
    m_line = rng.uniform(0.6, 1.0, size=len(lines))
    H = m_line[:, None] * (pet_brute.dense(lines, SHAPE, VOXEL) @ pet_brute.dense_blur(SHAPE, VOXEL, 1.5))
    keep = H.sum(axis=1) > 0
    lines, m_line, H = lines[keep], m_line[keep], H[keep]
    y = rng.integers(0, 4, size=len(lines))
    ev = np.repeat(np.arange(len(lines)), y)
    rng.shuffle(ev)
    return g, lines, m_line, H, y, ev


@pytest.mark.parametrize("s_val", [0.0, 0.05])
def test_listmode_em_equals_binned_mlem_of_dense_matrix(s_val):
    g, lines, m_line, H, y, ev = _em_case(11, s_val)
    sens = H.sum(axis=0)
    x0 = _rng(12).uniform(0.5, 1.5, size=SHAPE)
    x, _ = pet.lm_osem(lines[ev], m_line[ev], np.full(len(ev), s_val), sens.reshape(SHAPE), g, 1, x0=x0)
    p = H @ x0.ravel()
    ref = x0.ravel() * (H.T @ (y / (p + s_val))) / sens
    ref = np.where(sens > 0, ref, x0.ravel())
    assert np.max(np.abs(x.ravel() - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("s_val", [0.0, 0.05])
def test_listmode_osem_conserves_counts(s_val):
    g, lines, m_line, H, y, ev = _em_case(13, s_val)
    M = 3
    sens = H.sum(axis=0).reshape(SHAPE)
    x = np.ones(SHAPE)
    for it in range(4):
        xn, diag = pet.lm_osem(lines[ev], m_line[ev], np.full(len(ev), s_val), sens, g, M, x0=x, first=it, count=1)
        mask = sens > 0
        lhs = np.sum(sens[mask] / M * xn[mask])
        sub = ev[it % M::M]
        p = H[sub] @ x.ravel()
        rhs = np.sum(p / (p + s_val))
        assert abs(lhs - rhs) <= 1e-11 * rhs
        assert abs(diag[0, 0] - rhs) <= 1e-11 * rhs
        if s_val == 0.0:
            assert diag[0, 1] == len(sub)
        x = xn


# ---------------------------------------------------------------- time of flight

TOF = (9, 6.0, 5.0, 3.0)  # bins, bin width (mm), sigma (mm), truncation


def _tof(bins, tof=TOF):
    return pet.Tof(n_bins=tof[0], bin_mm=tof[1], sigma_mm=tof[2], nsigma=tof[3], bins=bins)


def test_tof_point_source_closed_form():
    """A line along x through the centre of one hot voxel: its projection in
    bin b is the step times the Gaussian integrated over the bin at the
    voxel's arc length (scipy's normal CDF)."""
    from scipy.stats import norm
    shape, voxel = (21, 5, 5), (2.0, 2.0, 2.0)
    g = pet.PetGeom(shape, voxel)
    f = np.zeros(shape)
    f[13, 2, 2] = 1.0
    nb, width, sigma, nsig = 11, 4.0, 3.0, 3.0
    lor = np.array([-30.0, 0.0, 0.0, 34.0, 0.0, 0.0])  # midpoint at x = 2 mm
    x_hot = (13 - 10) * 2.0
    ell = x_hot - 2.0
    got = [pet.joseph_fwd(f, lor[None], g, _tof([b], (nb, width, sigma, nsig)))[0] for b in range(nb)]
    for b in range(nb):
        c = (b - 0.5 * (nb - 1)) * width
        want = 2.0 * (norm.cdf((ell - c + width / 2) / sigma) - norm.cdf((ell - c - width / 2) / sigma))
        if abs(ell - c) > nsig * sigma + width / 2:
            want = 0.0
        assert abs(got[b] - want) <= 1e-14


def test_tof_bins_sum_to_non_tof():
    """Bins that cover the line and a window wide enough to cut nothing:
    the bins' projections add up to the non-TOF projection."""
    lors = mixed_lors(21, count=40)
    g = pet.PetGeom(SHAPE, VOXEL)
    f = _rng(22).uniform(size=SHAPE)
    ref = pet.joseph_fwd(f, lors, g)
    nb, width, sigma = 81, 10.0, 4.0
    tot = np.zeros(len(lors))
    for b in range(nb):
        tot += pet.joseph_fwd(f, lors, g, _tof([b] * len(lors), (nb, width, sigma, 40.0)))
    assert np.max(np.abs(tot - ref)) <= 1e-12 * max(1.0, np.max(ref))


def test_tof_joseph_equals_scipy_dense_matrix():
    lors = mixed_lors(23, count=40)
    bins = _rng(24).integers(0, TOF[0], size=len(lors))
    g = pet.PetGeom(SHAPE, VOXEL)
    H = pet_brute.dense(lors, SHAPE, VOXEL, TOF, bins)
    f = _rng(25).uniform(size=SHAPE)
    got = pet.joseph_fwd(f, lors, g, _tof(bins))
    assert np.max(np.abs(got - H @ f.ravel())) <= 1e-12 * max(1.0, np.max(np.abs(got)))
    v = _rng(26).normal(size=len(lors))
    back = pet.joseph_back(v, lors, g, _tof(bins)).ravel()
    assert np.max(np.abs(back - H.T @ v)) <= 1e-12 * max(1.0, np.max(np.abs(back)))
    assert np.count_nonzero(H.sum(axis=1)) > len(lors) // 3


def test_tof_listmode_em_equals_binned_mlem():
    rng = _rng(27)
    lines = mixed_lors(27, count=25)
    g = pet.PetGeom(SHAPE, VOXEL, rr_sigma_mm=1.5)
    bins = rng.integers(0, TOF[0], size=len(lines))
    m_line = rng.uniform(0.6, 1.0, size=len(lines))
    H = m_line[:, None] * (pet_brute.dense(lines, SHAPE, VOXEL, TOF, bins) @
                           pet_brute.dense_blur(SHAPE, VOXEL, 1.5))
    keep = H.sum(axis=1) > 0
    lines, bins, m_line, H = lines[keep], bins[keep], m_line[keep], H[keep]
    y = rng.integers(0, 4, size=len(lines))
    ev = np.repeat(np.arange(len(lines)), y)
    rng.shuffle(ev)
    sens = H.sum(axis=0) + 0.1  # any positive sensitivity image
    x0 = rng.uniform(0.5, 1.5, size=SHAPE)
    s_val = 0.02
    x, diag = pet.lm_osem(lines[ev], m_line[ev], np.full(len(ev), s_val), sens.reshape(SHAPE), g, 1, x0=x0,
                          tof=_tof(bins[ev]))
    p = H @ x0.ravel()
    ref = x0.ravel() * (H.T @ (y / (p + s_val))) / sens
    assert np.max(np.abs(x.ravel() - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert abs(diag[0, 0] - np.sum(y * p / (p + s_val))) <= 1e-11 * diag[0, 0]


def test_planes_are_decided_in_double_precision():
    """An end 1e-9 voxel past plane 2 (below single precision's resolution
    there) starts the walk at plane 3; an end exactly on plane 2 starts it at
    plane 2; |dx| / vx a hair above |dy| / vy picks x."""
    shape, voxel = (8, 8, 8), (2.0, 2.0, 2.0)
    g = pet.PetGeom(shape, voxel)
    org = -0.5 * (shape[0] - 1) * voxel[0]
    x_on = org + 2 * voxel[0]
    x_past = org + (2 + 1e-9) * voxel[0]
    assert np.float32(x_past) == np.float32(x_on)
    lors = np.array([[x_on, 0.3, 0.2, 100.0, 0.3, 0.2],
                     [x_past, 0.3, 0.2, 100.0, 0.3, 0.2],
                     [-50.0, -50.0 + 1e-9, 0.1, 50.0, 50.0, 0.1],
                     [-50.0, -50.0 - 1e-9, 0.1, 50.0, 50.0, 0.1]])
    got = pet.planes(lors, g)
    assert tuple(got[0]) == (0, 2, 7)
    assert tuple(got[1]) == (0, 3, 7)
    assert got[2][0] == 0  # |dx| > |dy|
    assert got[3][0] == 1  # |dy| > |dx|


def test_precision_filter_flags_rounding_ties():
    """The GPU tests leave out lines whose single-precision decisions differ
    from the oracle's, from float32 ends as the kernel reads them: an end one
    float32 step past a plane (p - org rounds onto the plane in float32),
    and a near-45-degree line whose float32 |dx| and |dy| compare the other
    way than in double precision."""
    import pet_precision
    shape, voxel = (8, 8, 8), (2.0, 2.0, 2.0)
    g = pet.PetGeom(shape, voxel)
    x_on = np.float32(-3.0)  # plane 2 of x: org = -7
    x_past = np.nextafter(x_on, np.float32(1.0), dtype=np.float32)
    lors = np.array([[x_on, 0.3, 0.2, 100.0, 0.3, 0.2],
                     [x_past, 0.3, 0.2, 100.0, 0.3, 0.2],
                     [-50.0, 0.7, 0.1, 50.0, 1.3, 0.1],
                     [-57.94597625732422, -36.93305969238281, 0.1, 32.47325897216797, 53.48617935180664, 0.1]],
                    dtype=np.float32)
    ref = pet.planes(lors.astype(np.float64), g)
    a, q0, q1, hit = pet_precision.kernel_decisions(lors, shape, voxel)
    assert (ref[1][1], q0[1]) == (3, 2)
    assert (ref[3][0], a[3]) == (1, 0)
    assert pet_precision.same_decisions(lors, g, pet).tolist() == [True, False, True, False]
