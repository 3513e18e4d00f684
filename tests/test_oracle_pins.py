"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails at least one of them:
  - brute force: dense H assembled from scipy/numpy library routines (8^3);
  - rotation: identity at 0, exact index permutations at 90/180/270 degrees,
    scipy's bilinear affine transform at arbitrary angles;
  - attenuation: exp(-mu L) through a uniform medium (closed form);
  - PSF: unit sum, centre and second moment of a point source against the
    continuous Gaussian sigma_i^2 with sigma_i linear in the depth distance;
  - adjointness <Hx, y> = <x, H^T y>;
  - OSEM count conservation (s = 0) and its s > 0 form;
  - the Poisson gradient of Table 1 against central finite differences of
    the log-likelihood;
  - MAP algorithms: the optimality condition of the MAP objective at the
    limit (one subset, and M identical subsets for the beta / M weight),
    plain MLEM steps and the relaxation schedule of BSREM on identical
    subsets, and BSREM's approach to the MAP point with distinct subsets.
"""
import math

import numpy as np
import pytest

import brute
from paper_2309_01977_gb300 import phantom


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- rotation

def test_rotation_zero_angle_is_identity(oracle_mod):
    f = _rng(1).uniform(size=(9, 9, 4))
    np.testing.assert_array_equal(oracle_mod.rotate(f, 0.0), f)


@pytest.mark.parametrize("quarter", [1, 2, 3])
def test_rotation_quarter_turns_are_permutations(oracle_mod, quarter):
    n, nz = 10, 3
    f = _rng(2).uniform(size=(n, n, nz))
    out = oracle_mod.rotate(f, quarter * math.pi / 2)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    # sample point of rotated voxel (i, j) for cos/sin in {0, +-1}
    ct = [1, 0, -1, 0][quarter]
    st = [0, 1, 0, -1][quarter]
    c2 = n - 1  # 2c
    u2 = c2 + ct * (2 * i - c2) - st * (2 * j - c2)
    v2 = c2 + st * (2 * i - c2) + ct * (2 * j - c2)
    expect = f[u2 // 2, v2 // 2, :]
    np.testing.assert_allclose(out, expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("theta", [0.3, 1.1, 2.5, 4.0, 5.9])
def test_rotation_matches_scipy_bilinear(oracle_mod, theta):
    f = _rng(3).uniform(size=(13, 13, 5))
    np.testing.assert_allclose(oracle_mod.rotate(f, theta), brute.rotate_lib(f, theta), rtol=0, atol=1e-13)


def test_rotation_adjoint_dot(oracle_mod):
    rng = _rng(4)
    x = rng.normal(size=(11, 11, 3))
    y = rng.normal(size=(11, 11, 3))
    for theta in (0.7, 2.0, 3.3):
        lhs = np.vdot(oracle_mod.rotate(x, theta), y)
        rhs = np.vdot(x, oracle_mod.rotate_adjoint(y, theta))
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1)


# ---------------------------------------------------------------- attenuation

@pytest.mark.parametrize("theta_q", [0, 1, 2])
def test_uniform_medium_attenuation_closed_form(oracle_mod, theta_q):
    """A point source behind L = (n-1-i+1/2) voxels of uniform mu reaches the detector with exp(-mu*dx*L)."""
    n, nz, mu0, dx = 12, 5, 0.2, 0.48
    theta = theta_q * math.pi / 2
    mu = np.full((n, n, nz), mu0)
    g = oracle_mod.Geom(n=n, nz=nz, n_angles=1, angles=[theta], voxel_cm=dx, mu=mu, use_psf=False)
    for (x0, y0, z0) in [(2, 3, 1), (9, 6, 4), (5, 11, 0)]:
        f = np.zeros((n, n, nz))
        f[x0, y0, z0] = 1.0
        proj = oracle_mod.forward(f, g)[0]
        # rotated-frame coordinates of the source (quarter turns are permutations)
        if theta_q == 0:
            depth, bin_y = x0, y0
        elif theta_q == 1:
            depth, bin_y = y0, n - 1 - x0
        else:
            depth, bin_y = n - 1 - x0, n - 1 - y0
        expect = math.exp(-mu0 * dx * (n - 1 - depth + 0.5))
        assert proj[bin_y, z0] == pytest.approx(expect, rel=1e-13)
        proj[bin_y, z0] = 0.0
        assert np.abs(proj).max() < 1e-14


def test_attenuation_map_matches_cumulative_sum(oracle_mod):
    mu = _rng(5).uniform(0, 0.3, size=(9, 9, 4))
    for theta in (0.0, 0.9, 4.4):
        np.testing.assert_allclose(oracle_mod.attenuation(mu, theta, 0.48),
                                   brute.attenuation_lib(mu, theta, 0.48), rtol=1e-13, atol=0)


# ---------------------------------------------------------------- PSF

@pytest.mark.parametrize("depth", [0, 10, 20, 40])
def test_psf_point_source_second_moment(oracle_mod, depth):
    """With negligible truncation (12 sigma) the sampled Gaussian of sigma >= 1 has
    variance sigma^2 up to e^(-2 pi^2 sigma^2); sigma_i = sigma0 + slope*(n - i - 1/2)."""
    n, nz = 64, 64
    sigma0, slope = 0.5, 0.03
    g = oracle_mod.Geom(n=n, nz=nz, n_angles=1, angles=[0.0], mu=None, use_psf=True,
                        sigma0=sigma0, slope=slope, nsigma=12.0)
    f = np.zeros((n, n, nz))
    j0, k0 = 31, 33
    f[depth, j0, k0] = 1.0
    p = oracle_mod.forward(f, g)[0]
    sigma = sigma0 + slope * (n - depth - 0.5)
    assert sigma >= 1.0
    jj, kk = np.meshgrid(np.arange(n) - j0, np.arange(nz) - k0, indexing="ij")
    assert p.sum() == pytest.approx(1.0, abs=1e-13)
    assert (p * jj).sum() == pytest.approx(0.0, abs=1e-12)
    assert (p * kk).sum() == pytest.approx(0.0, abs=1e-12)
    assert (p * jj * jj).sum() == pytest.approx(sigma * sigma, rel=1e-7)
    assert (p * kk * kk).sum() == pytest.approx(sigma * sigma, rel=1e-7)
    assert (p * jj * kk).sum() == pytest.approx(0.0, abs=1e-12)


def test_psf_taps_radius_and_normalisation(oracle_mod):
    sig, rad, taps = oracle_mod.psf_taps(128, 0.5, 0.03, 3.0)
    d = 128 - np.arange(128) - 0.5
    np.testing.assert_allclose(sig, 0.5 + 0.03 * d, rtol=1e-15)
    np.testing.assert_array_equal(rad, np.ceil(3 * sig).astype(int))
    assert rad.max() == 13 and rad.min() == 2
    np.testing.assert_allclose(taps.sum(axis=1), 1.0, rtol=1e-14)
    for i in (0, 64, 127):
        np.testing.assert_allclose(taps[i][13 - rad[i]:13 + rad[i] + 1],
                                   brute.gaussian_taps_lib(sig[i], 3.0), rtol=1e-14)


# ---------------------------------------------------------------- whole operator

def test_brute_force_dense_h_8cubed(oracle_mod):
    """H x and H^T y of the oracle equal the library-built dense H at 8^3, 8 angles."""
    n = nz = 8
    rng = _rng(6)
    mu = rng.uniform(0.0, 0.4, size=(n, n, nz))
    angles = [2 * math.pi * a / 8 + 0.05 for a in range(8)]
    kw = dict(voxel_cm=0.48, use_psf=True, sigma0=0.6, slope=0.15, nsigma=3.0)
    H = brute.dense_h(n, nz, angles, mu, **kw)
    g = oracle_mod.Geom(n=n, nz=nz, n_angles=8, angles=angles, mu=mu, **kw)
    x = rng.uniform(size=(n, n, nz))
    y = rng.uniform(size=(8, n, nz))
    hx = oracle_mod.forward(x, g).ravel()
    hty = oracle_mod.back(y, g).ravel()
    ref_hx = H @ x.ravel()
    ref_hty = H.T @ y.ravel()
    assert np.abs(hx - ref_hx).max() <= 1e-12 * np.abs(ref_hx).max()
    assert np.abs(hty - ref_hty).max() <= 1e-12 * np.abs(ref_hty).max()


def test_adjoint_dot_product_composed(oracle_mod):
    n, nz = 16, 12
    rng = _rng(7)
    mu = rng.uniform(0, 0.3, size=(n, n, nz))
    g = oracle_mod.Geom(n=n, nz=nz, n_angles=12, mu=mu, use_psf=True, sigma0=0.5, slope=0.1)
    x = rng.normal(size=(n, n, nz))
    y = rng.normal(size=(12, n, nz))
    lhs = np.vdot(oracle_mod.forward(x, g), y)
    rhs = np.vdot(x, oracle_mod.back(y, g))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_subset_selection_is_interleaved(oracle_mod):
    assert oracle_mod.subset_angles(60, 8, 0) == [0, 8, 16, 24, 32, 40, 48, 56]
    assert oracle_mod.subset_angles(60, 8, 7) == [7, 15, 23, 31, 39, 47, 55]
    sizes = [len(oracle_mod.subset_angles(120, 8, m)) for m in range(8)]
    assert sizes == [15] * 8


def _small_problem(oracle_mod, s_frac, seed=8):
    n = nz = 16
    f_raw, mu = phantom.make_phantom(n, nz, seed)
    g = oracle_mod.Geom(n=n, nz=nz, n_angles=16, mu=mu, use_psf=True, sigma0=0.5, slope=0.05)
    hf = oracle_mod.forward(f_raw, g)
    f_true, y, s, _ = phantom.make_counts(f_raw, hf, 1e5, s_frac, seed)
    return g, y, s


@pytest.mark.parametrize("s_frac", [0.0, 0.05])
def test_osem_count_conservation(oracle_mod, s_frac):
    """sum_{S_m} H_m f_new = sum_{S_m} y * H_m f / (H_m f + s); for s = 0 that is sum y."""
    g, y, s = _small_problem(oracle_mod, s_frac)
    M = 4
    f = np.ones((g.n, g.n, g.nz))
    for t in range(6):
        m = t % M
        sel = oracle_mod.subset_angles(g.n_angles, M, m)
        f_new, diag = oracle_mod.osem(y, s, g, M, t, 1, f)
        lhs = oracle_mod.forward(f_new, g, sel).sum()
        p = oracle_mod.forward(f, g, sel)
        ys = y[sel]
        expect = (ys * p / (p + s)).sum()
        assert lhs == pytest.approx(expect, rel=1e-12)
        assert diag[0, 2] == pytest.approx(expect, rel=1e-12)
        assert diag[0, 1] == pytest.approx(ys.sum(), rel=1e-14)
        assert diag[0, 0] == pytest.approx((p + s).sum(), rel=1e-12)
        if s_frac == 0.0:
            assert lhs == pytest.approx(ys.sum(), rel=1e-12)
        f = f_new


def test_osem_resume_equals_one_call(oracle_mod):
    g, y, s = _small_problem(oracle_mod, 0.05)
    f_all, _ = oracle_mod.osem(y, s, g, 4, 0, 5)
    f_a, _ = oracle_mod.osem(y, s, g, 4, 0, 2)
    f_b, _ = oracle_mod.osem(y, s, g, 4, 2, 3, f_a)
    np.testing.assert_array_equal(f_all, f_b)


def test_poisson_gradient_matches_finite_differences(oracle_mod):
    """Table 1: grad L = H^T(y/(Hf+s)) - H^T 1 for L = sum y log(Hf+s) - (Hf+s)."""
    g, y, s = _small_problem(oracle_mod, 0.05, seed=9)
    f = _rng(10).uniform(0.5, 2.0, size=(g.n, g.n, g.nz)) * (y.sum() / 16 ** 3 / 16)
    p = oracle_mod.forward(f, g)
    grad = oracle_mod.back(y / (p + s), g) - oracle_mod.back(np.ones_like(p), g)
    rng = _rng(11)
    for _ in range(6):
        q = tuple(rng.integers(0, 16, size=3))
        h = 1e-3 * f[q]
        fp = f.copy(); fp[q] += h
        fm = f.copy(); fm[q] -= h
        lp = oracle_mod.poisson_ll(y, oracle_mod.forward(fp, g), s)
        lm = oracle_mod.poisson_ll(y, oracle_mod.forward(fm, g), s)
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(grad[q], rel=1e-5, abs=1e-6 * np.abs(grad).max())


# ---------------------------------------------------------------- priors and MAP (Sec. 2.1.3, Table 1)

def test_prior_value_two_voxels_closed_form(oracle_mod):
    """Two voxels along z (w = 1): V = phi(a, b) + phi(b, a), by hand."""
    f = np.array([[[3.0, 1.0]]])
    # RDP, gamma = 2: (3-1)^2 / (3+1+2*2) = 0.5 per ordered pair
    assert oracle_mod.prior_value(f, "rdp", gamma=2.0) == pytest.approx(1.0, rel=1e-15)
    # quadratic, delta = 2: ((3-1)/2)^2 / 4 = 0.25 per ordered pair
    assert oracle_mod.prior_value(f, "quadratic", delta=2.0) == pytest.approx(0.5, rel=1e-15)


def test_prior_gradient_two_voxels_closed_form(oracle_mod):
    """V(a, b) = 2 (a-b)^2 / (a+b+2|a-b|) at (3, 1): dV/da = 0.625, dV/db = -0.875 (by hand)."""
    g = oracle_mod.prior_grad(np.array([[[3.0, 1.0]]]), "rdp", gamma=2.0)
    assert g[0, 0, 0] == pytest.approx(0.625, rel=1e-14)
    assert g[0, 0, 1] == pytest.approx(-0.875, rel=1e-14)


def test_prior_neighbour_weights_inverse_distance(oracle_mod):
    """2x2x2 block, one corner a, the rest c: the corner has 3 neighbours at
    distance 1, 3 at sqrt 2 and 1 at sqrt 3, each pair counted twice."""
    a, c = 2.0, 0.5
    f = np.full((2, 2, 2), c)
    f[0, 0, 0] = a
    phi = (a - c) ** 2 / (a + c + 2.0 * abs(a - c))
    expect = 2 * phi * (3 + 3 / math.sqrt(2) + 1 / math.sqrt(3))
    assert oracle_mod.prior_value(f, "rdp", gamma=2.0) == pytest.approx(expect, rel=1e-14)


@pytest.mark.parametrize("prior", ["quadratic", "rdp"])
def test_prior_gradient_matches_finite_differences(oracle_mod, prior):
    rng = _rng(21)
    f = rng.uniform(0.2, 3.0, size=(5, 5, 6))
    g = oracle_mod.prior_grad(f, prior, delta=1.5, gamma=2.0)
    for _ in range(12):
        q = tuple(int(v) for v in rng.integers(0, [5, 5, 6]))
        h = 1e-5
        fp = f.copy(); fp[q] += h
        fm = f.copy(); fm[q] -= h
        fd = (oracle_mod.prior_value(fp, prior, 1.5, 2.0) - oracle_mod.prior_value(fm, prior, 1.5, 2.0)) / (2 * h)
        assert fd == pytest.approx(g[q], rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("prior", ["quadratic", "rdp"])
def test_prior_gradient_vanishes_on_constant_image(oracle_mod, prior):
    g = oracle_mod.prior_grad(np.full((4, 4, 5), 1.7), prior)
    assert np.abs(g).max() == 0.0


def test_osmaposl_without_prior_weight_is_osem(oracle_mod):
    """Table 1: OSMAPOSL with beta = 0 has the OSEM preconditioner."""
    g, y, s = _small_problem(oracle_mod, 0.05)
    f_osem, _ = oracle_mod.osem(y, s, g, 4, 0, 5)
    f_map = oracle_mod.map_recon(y, s, g, 4, 0, 5, "osmaposl", "rdp", beta=0.0)
    np.testing.assert_allclose(f_map, f_osem, rtol=1e-13, atol=0)


def test_bsrem_one_subset_first_step_is_mlem(oracle_mod):
    """BSREM with one subset, beta = 0 and alpha = 1: f + f/H^T1 (H^T r - H^T 1) = f H^T r / H^T 1."""
    g, y, s = _small_problem(oracle_mod, 0.05)
    f_mlem, _ = oracle_mod.osem(y, s, g, 1, 0, 1)
    f_map = oracle_mod.map_recon(y, s, g, 1, 0, 1, "bsrem", "rdp", beta=0.0, alpha0=1.0)
    np.testing.assert_allclose(f_map, f_mlem, rtol=1e-12, atol=1e-14 * np.abs(f_mlem).max())


@pytest.mark.parametrize("algorithm", ["osmaposl", "bsrem"])
def test_map_prior_smooths(oracle_mod, algorithm):
    """With the RDP weighted in, the image's own RDP value drops below the unregularised one."""
    g, y, s = _small_problem(oracle_mod, 0.05)
    f0 = oracle_mod.map_recon(y, s, g, 4, 0, 8, algorithm, "rdp", beta=0.0)
    f1 = oracle_mod.map_recon(y, s, g, 4, 0, 8, algorithm, "rdp", beta=0.3)
    assert oracle_mod.prior_value(f1, "rdp") < oracle_mod.prior_value(f0, "rdp")
    assert np.isfinite(f1).all() and f1.min() >= 0.0


# MAP algorithms pinned by the optimality condition of the MAP objective
# Phi(f) = L(f) - beta V(f) (Eq. PGA with the Poisson gradient of Table 1):
# at a maximiser f >= 0, f (grad L(f) - beta grad V(f)) = 0 voxel by voxel.
# grad L comes from the oracle's H and H^T (pinned by the dense H above) and
# grad V from the prior gradient (pinned by finite differences above), so
# the check is independent of or_map's update formulas.  The subset
# scalings are pinned by data sets whose M subsets are identical (every
# angle listed M times): then L = M L_K (L_K the likelihood of one copy), so
# the MAP point of beta is the MAP point of L_K - (beta / M) V, and a
# BSREM step of one subset is a plain MLEM step of L_K.

_MAP_K, _MAP_M = 12, 4


def _map_problem(oracle_mod, copies=1):
    """8^3 x 4 volume, 12 angles (each listed `copies` times in a row), y = H f + s."""
    n, nz, K = 8, 4, _MAP_K
    rng = _rng(7)
    base = [2 * math.pi * k / K + 0.3 for k in range(K)]
    f_true = rng.uniform(0.5, 2.0, size=(n, n, nz))
    mu = np.full((n, n, nz), 0.1)
    kw = dict(n=n, nz=nz, mu=mu, sigma0=0.6, slope=0.05)
    g1 = oracle_mod.Geom(n_angles=K, angles=base, **kw)
    y1 = oracle_mod.forward(f_true, g1)
    s = 0.05 * y1.mean()
    y1 = y1 + s
    if copies == 1:
        return g1, y1, s
    # angle a = k * copies + m: subset m of `copies` subsets holds each base angle once
    g = oracle_mod.Geom(n_angles=K * copies, angles=[base[a // copies] for a in range(K * copies)], **kw)
    return g, np.repeat(y1, copies, axis=0), s


def _kkt(oracle_mod, f, g, y, s, beta, prior):
    """|| f (grad L - beta grad V) || relative to || f H^T 1 ||."""
    p = oracle_mod.forward(f, g)
    ones = np.ones_like(p)
    gl = oracle_mod.back(y / (p + s), g) - oracle_mod.back(ones, g)
    gv = oracle_mod.prior_grad(f, prior, delta=1.0, gamma=2.0)
    return np.linalg.norm(f * (gl - beta * gv)) / np.linalg.norm(f * oracle_mod.back(ones, g))


@pytest.mark.parametrize("prior", ["quadratic", "rdp"])
def test_osmaposl_one_subset_converges_to_the_map_point(oracle_mod, prior):
    """One subset: the one-step-late fixed point satisfies the MAP optimality
    condition of L - beta V; the same image is far from optimal for 2 beta
    (a prior term scaled or signed wrongly would fail)."""
    g, y, s = _map_problem(oracle_mod)
    beta = 0.1
    f = oracle_mod.map_recon(y, s, g, 1, 0, 600, "osmaposl", prior, beta=beta)
    assert _kkt(oracle_mod, f, g, y, s, beta, prior) <= 1e-12
    assert _kkt(oracle_mod, f, g, y, s, 2 * beta, prior) >= 1e-3


def test_osmaposl_identical_subsets_weight_the_prior_by_one_over_m(oracle_mod):
    """M identical subsets: the limit is the MAP point of the whole data set
    for beta (so the per-subset weight is beta / M), not of beta M."""
    g, y, s = _map_problem(oracle_mod, copies=_MAP_M)
    beta = 0.1
    f = oracle_mod.map_recon(y, s, g, _MAP_M, 0, 400 * _MAP_M, "osmaposl", "quadratic", beta=beta)
    assert _kkt(oracle_mod, f, g, y, s, beta, "quadratic") <= 1e-12
    assert _kkt(oracle_mod, f, g, y, s, beta * _MAP_M, "quadratic") >= 1e-3
    # each subiteration is a one-subset step on one copy with the prior weight beta / M
    g1, y1, _ = _map_problem(oracle_mod)
    f1 = oracle_mod.map_recon(y1, s, g1, 1, 0, 400 * _MAP_M, "osmaposl", "quadratic", beta=beta / _MAP_M)
    np.testing.assert_allclose(f, f1, rtol=1e-12, atol=0)


def test_bsrem_identical_subsets_are_mlem_steps_with_the_relaxation_schedule(oracle_mod):
    """M identical subsets, beta = 0, alpha0 = 1: H^T 1 = M H_K^T 1, so with
    c_n = 1/M each subiteration of the first iteration is an MLEM step of one
    copy (alpha = 1); the first subiteration of the second iteration has
    alpha = 1/2 and lands halfway between its start and that MLEM step."""
    g, y, s = _map_problem(oracle_mod, copies=_MAP_M)
    g1, y1, _ = _map_problem(oracle_mod)
    f_b = oracle_mod.map_recon(y, s, g, _MAP_M, 0, _MAP_M, "bsrem", "quadratic", beta=0.0, alpha0=1.0)
    f_m, _ = oracle_mod.osem(y1, s, g1, 1, 0, _MAP_M)
    np.testing.assert_allclose(f_b, f_m, rtol=1e-13, atol=0)
    f_b1 = oracle_mod.map_recon(y, s, g, _MAP_M, 0, _MAP_M + 1, "bsrem", "quadratic", beta=0.0, alpha0=1.0)
    f_m1, _ = oracle_mod.osem(y1, s, g1, 1, 0, 1, f_m)
    np.testing.assert_allclose(f_b1, 0.5 * (f_m + f_m1), rtol=1e-13, atol=0)


def test_bsrem_converges_to_the_map_point(oracle_mod):
    """Distinct subsets: the relaxed BSREM iterates approach the MAP point of
    L - beta V (the OSMAPOSL limit of one subset, pinned above), and get
    closer as the relaxation shrinks; unrelaxed OSMAPOSL with the same
    subsets stalls further away (a limit cycle)."""
    g, y, s = _map_problem(oracle_mod)
    beta, M = 0.1, _MAP_M
    f_map = oracle_mod.map_recon(y, s, g, 1, 0, 600, "osmaposl", "quadratic", beta=beta)

    def dist(f):
        return np.linalg.norm(f - f_map) / np.linalg.norm(f_map)

    f_200 = oracle_mod.map_recon(y, s, g, M, 0, 200 * M, "bsrem", "quadratic", beta=beta, alpha0=1.0)
    f_800 = oracle_mod.map_recon(y, s, g, M, 0, 800 * M, "bsrem", "quadratic", beta=beta, alpha0=1.0)
    f_osl = oracle_mod.map_recon(y, s, g, M, 0, 400 * M, "osmaposl", "quadratic", beta=beta)
    assert dist(f_800) <= 6e-4
    assert dist(f_800) < 0.6 * dist(f_200)
    assert dist(f_osl) > 5 * dist(f_800)
    assert _kkt(oracle_mod, f_800, g, y, s, beta, "quadratic") <= 1e-4
    assert _kkt(oracle_mod, f_800, g, y, s, beta * M, "quadratic") >= 1e-2


# ---------------------------------------------------------------- non-circular orbits

def test_brute_force_dense_h_noncircular_orbit(oracle_mod):
    """Per-angle detector offsets (a non-circular orbit): the oracle's H and
    H^T equal the library-built dense H with each angle's own PSF table."""
    n = nz = 8
    rng = _rng(61)
    mu = rng.uniform(0.0, 0.4, size=(n, n, nz))
    angles = [2 * math.pi * a / 8 + 0.05 for a in range(8)]
    offs = [0.0, 1.5, 3.0, 1.0, 0.5, 2.5, 4.0, 0.2]
    kw = dict(voxel_cm=0.48, use_psf=True, sigma0=0.6, slope=0.15, nsigma=3.0)
    H = brute.dense_h(n, nz, angles, mu, det_offsets=offs, **kw)
    g = oracle_mod.Geom(n=n, nz=nz, n_angles=8, angles=angles, mu=mu, det_offsets=offs, **kw)
    x = rng.uniform(size=(n, n, nz))
    y = rng.uniform(size=(8, n, nz))
    ref_hx = H @ x.ravel()
    ref_hty = H.T @ y.ravel()
    assert np.abs(oracle_mod.forward(x, g).ravel() - ref_hx).max() <= 1e-12 * np.abs(ref_hx).max()
    assert np.abs(oracle_mod.back(y, g).ravel() - ref_hty).max() <= 1e-12 * np.abs(ref_hty).max()
    # a circular orbit given per angle is the scalar offset
    g1 = oracle_mod.Geom(n=n, nz=nz, n_angles=8, angles=angles, mu=mu, det_offset=1.5, **kw)
    g2 = oracle_mod.Geom(n=n, nz=nz, n_angles=8, angles=angles, mu=mu, det_offsets=[1.5] * 8, **kw)
    np.testing.assert_array_equal(oracle_mod.forward(x, g1), oracle_mod.forward(x, g2))


# ---------------------------------------------------------------- multi-photopeak extended system matrix

def _two_peaks(oracle_mod, seed=71):
    n = nz = 12
    f_raw, mu = phantom.make_phantom(n, nz, seed)
    g1 = oracle_mod.Geom(n=n, nz=nz, n_angles=8, mu=mu, use_psf=True, sigma0=0.5, slope=0.05)
    g2 = oracle_mod.Geom(n=n, nz=nz, n_angles=8, mu=0.8 * mu, use_psf=True, sigma0=0.7, slope=0.08)
    rng = _rng(seed)
    y1 = rng.poisson(oracle_mod.forward(f_raw, g1) * 50.0 + 1.0).astype(float)
    y2 = rng.poisson(0.6 * oracle_mod.forward(f_raw, g2) * 50.0 + 1.0).astype(float)
    return g1, g2, y1, y2


def test_multi_peak_with_one_peak_is_osem(oracle_mod):
    g1, g2, y1, y2 = _two_peaks(oracle_mod)
    f_ref, _ = oracle_mod.osem(y1, 1.0, g1, 4, 0, 6)
    f = oracle_mod.osem_multi([y1], [1.0], [g1], [1.0], 4, 0, 6)
    np.testing.assert_allclose(f, f_ref, rtol=1e-12, atol=0)


def test_multi_peak_two_copies_of_one_peak_is_osem(oracle_mod):
    """Two identical peaks observing the same counts: numerator and
    denominator both double, so the update is OSEM's."""
    g1, g2, y1, y2 = _two_peaks(oracle_mod)
    f_ref, _ = oracle_mod.osem(y1, 1.0, g1, 4, 0, 6)
    f = oracle_mod.osem_multi([y1, y1], [1.0, 1.0], [g1, g1], [1.0, 1.0], 4, 0, 6)
    np.testing.assert_allclose(f, f_ref, rtol=1e-12, atol=0)


def test_multi_peak_count_conservation(oracle_mod):
    """s = 0: the subset's predicted counts over all peaks equal its measured counts after the update."""
    g1, g2, y1, y2 = _two_peaks(oracle_mod)
    scales = [1.0, 0.6]
    f = np.ones((12, 12, 12))
    for t in range(4):
        f_new = oracle_mod.osem_multi([y1, y2], [0.0, 0.0], [g1, g2], scales, 4, t, 1, f)
        sel = oracle_mod.subset_angles(8, 4, t % 4)
        pred = sum(a * oracle_mod.forward(f_new, g, sel).sum() for a, g in zip(scales, [g1, g2]))
        meas = y1[sel].sum() + y2[sel].sum()
        assert pred == pytest.approx(meas, rel=1e-11)
        f = f_new


def test_rotation_keeps_a_constant_field_inside_the_grid(oracle_mod):
    """Bilinear weights sum to one: a constant volume stays constant at every
    rotated voxel whose four taps lie inside the grid (the inscribed region),
    for arbitrary angles; voxels whose sample point leaves the grid by a full
    voxel read zero."""
    n, nz, c0 = 20, 3, 2.75
    f = np.full((n, n, nz), c0)
    cen = 0.5 * (n - 1)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for theta in (0.3, 1.1, 2.5, 4.0, 5.9):
        out = oracle_mod.rotate(f, theta)
        u = cen + np.cos(theta) * (ii - cen) - np.sin(theta) * (jj - cen)
        v = cen + np.sin(theta) * (ii - cen) + np.cos(theta) * (jj - cen)
        inside = (u >= 0) & (u <= n - 1) & (v >= 0) & (v <= n - 1)
        np.testing.assert_allclose(out[inside], c0, rtol=0, atol=1e-13)
        outside = (u < -1) | (u > n) | (v < -1) | (v > n)
        assert np.all(out[outside] == 0.0)
        assert inside.sum() > n * n // 2


# ---------------------------------------------------------------- T_trans and T_fov (Eq. 1)

@pytest.mark.parametrize("theta, shift", [(0.3, 0.7), (1.1, -2.3), (2.5, 1.0), (4.0, -0.45), (5.9, 3.2)])
def test_shifted_rotation_matches_scipy_affine(oracle_mod, theta, shift):
    f = _rng(81).uniform(size=(13, 13, 5))
    np.testing.assert_allclose(oracle_mod.rotate(f, theta, shift), brute.rotate_lib(f, theta, shift),
                               rtol=0, atol=1e-13)


def test_shifted_rotation_adjoint_dot(oracle_mod):
    rng = _rng(82)
    x = rng.normal(size=(11, 11, 3))
    y = rng.normal(size=(11, 11, 3))
    for theta, shift in ((0.7, 1.3), (2.0, -0.6), (3.3, 2.0)):
        lhs = np.vdot(oracle_mod.rotate(x, theta, shift), y)
        rhs = np.vdot(x, oracle_mod.rotate_adjoint(y, theta, shift))
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1)


def test_integer_shift_translates_the_projection(oracle_mod):
    """theta = 0, no blur, no attenuation: a shift of 2 voxels moves every
    projection bin by exactly 2 along j (zero where nothing arrives)."""
    n, nz = 12, 4
    f = _rng(83).uniform(size=(n, n, nz))
    g0 = oracle_mod.Geom(n=n, nz=nz, n_angles=1, angles=[0.0], mu=None, use_psf=False)
    g2 = oracle_mod.Geom(n=n, nz=nz, n_angles=1, angles=[0.0], mu=None, use_psf=False, trans=[2.0])
    p0 = oracle_mod.forward(f, g0)[0]
    p2 = oracle_mod.forward(f, g2)[0]
    np.testing.assert_allclose(p2[2:], p0[:-2], rtol=1e-14, atol=0)
    assert np.all(p2[:2] == 0.0)


def test_brute_force_dense_h_with_trans_and_fov(oracle_mod):
    """Per-angle shifts (T_trans) and projection-space weights (T_fov): the
    oracle's H and H^T equal the library-built dense H at 8^3, 8 angles."""
    n = nz = 8
    rng = _rng(84)
    mu = rng.uniform(0.0, 0.4, size=(n, n, nz))
    angles = [2 * math.pi * a / 8 + 0.05 for a in range(8)]
    shifts = list(rng.uniform(-2.0, 2.0, size=8))
    fov = (rng.uniform(size=(8, n, nz)) > 0.25) * rng.uniform(0.5, 1.0, size=(8, n, nz))
    kw = dict(voxel_cm=0.48, use_psf=True, sigma0=0.6, slope=0.15, nsigma=3.0)
    H = brute.dense_h(n, nz, angles, mu, trans=shifts, fov=fov, **kw)
    g = oracle_mod.Geom(n=n, nz=nz, n_angles=8, angles=angles, mu=mu, trans=shifts, fov=fov, **kw)
    x = rng.uniform(size=(n, n, nz))
    y = rng.uniform(size=(8, n, nz))
    ref_hx = H @ x.ravel()
    ref_hty = H.T @ y.ravel()
    assert np.abs(oracle_mod.forward(x, g).ravel() - ref_hx).max() <= 1e-12 * np.abs(ref_hx).max()
    assert np.abs(oracle_mod.back(y, g).ravel() - ref_hty).max() <= 1e-12 * np.abs(ref_hty).max()
    # with both switched off the operator is the central, unmasked one
    g0 = oracle_mod.Geom(n=n, nz=nz, n_angles=8, angles=angles, mu=mu, trans=[0.0] * 8, fov=np.ones((8, n, nz)), **kw)
    g1 = oracle_mod.Geom(n=n, nz=nz, n_angles=8, angles=angles, mu=mu, **kw)
    np.testing.assert_array_equal(oracle_mod.forward(x, g0), oracle_mod.forward(x, g1))


def test_one_hot_projection_from_a_z_slab_equals_the_full_one(oracle_mod):
    """The GPU gradient test at 192^3 takes H e_v from the z slab the voxel's
    blur reaches (tests/helpers.py); at 16 x 16 x 40 it equals the oracle's
    projection of the whole one-hot volume, near both axial edges and inside."""
    from helpers import one_hot_projection
    n, nz = 16, 40
    rng = _rng(91)
    mu = rng.uniform(0.0, 0.3, size=(n, n, nz))
    g = oracle_mod.Geom(n=n, nz=nz, n_angles=6, mu=mu, use_psf=True, sigma0=0.5, slope=0.2)
    rmax = oracle_mod.psf_rmax(n, 0.5, 0.2, 3.0)
    for v in [(3, 7, 0), (8, 2, 20), (12, 12, 39), (5, 9, rmax + 1)]:
        e = np.zeros((n, n, nz))
        e[v] = 1.0
        full = oracle_mod.forward(e, g)
        np.testing.assert_allclose(one_hot_projection(oracle_mod, g, v, rmax), full, rtol=1e-13, atol=1e-16)


def test_uniform_quarter_turns_are_exact_permutations(oracle_mod):
    """theta = 2 pi a / 4: cos and sin are exactly 0 and +-1, so without blur
    and attenuation each projection is the sum over depth of an exact index
    permutation of the volume (bitwise, summed in the same order), with no
    rounding-level weight leaking into neighbouring voxels."""
    n, nz = 10, 3
    f = _rng(92).uniform(size=(n, n, nz))
    g = oracle_mod.Geom(n=n, nz=nz, n_angles=4, mu=None, use_psf=False)
    p = oracle_mod.forward(f, g)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    perms = [(i, j), (n - 1 - j, i), (n - 1 - i, n - 1 - j), (j, n - 1 - i)]  # (u, v) of rotated voxel (i, j)
    for a, (u, v) in enumerate(perms):
        rot = f[u, v, :]
        expect = np.zeros((n, nz))
        for d in range(n):
            expect += rot[d]
        np.testing.assert_array_equal(p[a], expect)
