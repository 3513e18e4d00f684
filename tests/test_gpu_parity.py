"""GPU parity of libspect against the FP64 oracle (through the C ABI).

Tolerances:
  - projections, back projections and sensitivities: relative L2 <= 1e-5
    (FP32 path), and every element within 1e-4 of the largest reference
    value (so that an error confined to one tile or strip shows);
  - adjointness <Hx, y> = <x, H^T y> in FP32: <= 1e-6 relative;
  - OSEM images: relative L2 <= 2e-5 after the full 2 x 8 and 4 x 8 runs
    (rounding of ~1e-7 per step compounds over the subiterations; the
    measured error is an order of magnitude below this);
  - FP64 count sums: conservation holds to FP32 rounding of H x (1e-6).
Sizes span several blur strips and plane tiles with ragged tails (n and nz
not multiples of 16), a 132^2 x 44 geometry whose back projection takes the
tiled gather with partial tiles, a non-circular orbit (per-angle PSF tables),
non-central projections (T_trans) with a field-of-view mask (T_fov), the
64^3 and 128^3 workloads in full, and a 192^3 geometry whose planes are
split into z tiles.
"""
import math

import numpy as np
import pytest

from helpers import assert_close, f32, oracle_geom, phantom_inputs, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(dev)


def _fov_mask(n_angles, n, nz, seed):
    """T_fov test weights: per angle a field of view of random width along y
    and z (1 inside, 0 outside), with a few partial weights at its edge."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = np.zeros((n_angles, n, nz), dtype=np.float32)
    for a in range(n_angles):
        j0, j1 = sorted(rng.integers(0, n, size=2))
        k0, k1 = sorted(rng.integers(0, nz, size=2))
        m[a, j0:j1 + 2, k0:k1 + 2] = 1.0
        m[a, j0, k0:k1 + 2] = 0.5
    return m


def _band_mask(n_angles, n, nz, shifts, half):
    """A detector field of view: bins within `half` of the angle's shifted
    detector centre along y and inside two bins of the axial edges."""
    m = np.zeros((n_angles, n, nz), dtype=np.float32)
    c = 0.5 * (n - 1)
    j = np.arange(n)
    for a in range(n_angles):
        m[a][np.abs(j - c - shifts[a]) <= half, 2:nz - 2] = 1.0
    return m


def _shifts(n_angles, amp, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [float(v) for v in rng.uniform(-amp, amp, size=n_angles)]


CASES = {
    # name: (geometry kwargs, phantom seed)
    # non-central projections (T_trans, sub-voxel shifts per angle) and a
    # field-of-view mask (T_fov), per-column gather
    "trans_fov40x36": (dict(n=40, nz=36, n_angles=12, n_subsets=3, psf_slope=0.1, det_shifts=_shifts(12, 3.5, 41),
                            fov_mask=_fov_mask(12, 40, 36, 42)), 20),
    # the same on the tiled gather (partial tiles) with an orbit
    "trans_tiled132x44": (dict(n=132, nz=44, n_angles=9, n_subsets=3, det_shifts=_shifts(9, 6.0, 43),
                               det_offsets=[1.0 + 0.5 * a for a in range(9)]), 21),
    "ragged40x36": (dict(n=40, nz=36, n_angles=12, n_subsets=3, psf_slope=0.1), 11),
    "osem64": (dict(n=64, nz=64, n_angles=64, n_subsets=8), 1),
    "noatt_nopsf": (dict(n=48, nz=20, n_angles=7, n_subsets=2, attenuation=False, psf=False), 12),
    "psf_only": (dict(n=32, nz=44, n_angles=5, n_subsets=1, attenuation=False, psf_slope=0.15), 13),
    "explicit_angles": (dict(n=24, nz=8, n_angles=6, n_subsets=2, det_offset=3.0, psf_sigma0=0.8,
                             angles_rad=[0.0, 0.4, 1.9, math.pi, 4.0, 6.0]), 14),
    # planes of 128^2 and up take the tiled gather; 132 leaves partial 8x8
    # tiles at the edge and nz = 44 short z rows
    "tiled132x44": (dict(n=132, nz=44, n_angles=9, n_subsets=3), 15),
    # non-circular (elliptical) orbit: every angle has its own PSF table
    "orbit48x40": (dict(n=48, nz=40, n_angles=12, n_subsets=3,
                        det_offsets=[2.0 + 1.5 * math.cos(2 * 2 * math.pi * a / 12) for a in range(12)]), 16),
    # the largest supported PSF radius (R = 20 at the deepest plane), one
    # angle per subset
    "max_radius": (dict(n=48, nz=32, n_angles=6, n_subsets=6, psf_slope=0.129), 17),
    # a single angle
    "one_angle": (dict(n=16, nz=16, n_angles=1, n_subsets=1), 18),
    # a wide plane (256 x 256 rows, tiled gather) with short z rows
    "wide256x32": (dict(n=256, nz=32, n_angles=4, n_subsets=2, psf_slope=0.02), 19),
}


def _setup(spect, oracle, dev, name):
    kw, seed = CASES[name]
    g = spect.Geometry(**kw)
    f, mu = phantom_inputs(g.n, g.nz, seed)
    plan = spect.Plan(g, _t(mu, dev) if g.attenuation else None)
    og = oracle_geom(oracle, g, mu)
    return g, f, mu, plan, og


@pytest.mark.parametrize("name", sorted(CASES))
def test_forward_parity(spect_lib, oracle_mod, cuda, name):
    g, f, mu, plan, og = _setup(spect_lib, oracle_mod, cuda, name)
    for subset in [-1, 0, g.n_subsets - 1]:
        sel = plan.subset_angles(subset)
        assert sel == (list(range(g.n_angles)) if subset < 0 else oracle_mod.subset_angles(g.n_angles, g.n_subsets, subset))
        p = plan.forward(_t(f, cuda), subset).cpu().numpy()
        ref = oracle_mod.forward(f, og, sel)
        assert_close(p, ref, TOL, (name, subset))


@pytest.mark.parametrize("name", sorted(CASES))
def test_back_parity(spect_lib, oracle_mod, cuda, name):
    g, f, mu, plan, og = _setup(spect_lib, oracle_mod, cuda, name)
    rng = np.random.Generator(np.random.PCG64(5))
    for subset in [-1, 0]:
        sel = plan.subset_angles(subset)
        q = f32(rng.uniform(0.0, 2.0, size=(len(sel), g.n, g.nz)))
        b = plan.back(_t(q, cuda), subset).cpu().numpy()
        ref = oracle_mod.back(q, og, sel)
        assert_close(b, ref, TOL, (name, subset))


@pytest.mark.parametrize("name", ["ragged40x36", "osem64", "explicit_angles"])
def test_adjoint_dot_product(spect_lib, oracle_mod, cuda, name):
    g, f, mu, plan, og = _setup(spect_lib, oracle_mod, cuda, name)
    rng = np.random.Generator(np.random.PCG64(6))
    x = _t(rng.normal(size=(g.n, g.n, g.nz)), cuda)
    y = _t(rng.normal(size=(g.n_angles, g.n, g.nz)), cuda)
    hx = plan.forward(x).double()
    hty = plan.back(y).double()
    lhs = float((hx * y.double()).sum())
    rhs = float((x.double() * hty).sum())
    scale = float(hx.abs().sum() * y.abs().max())
    assert abs(lhs - rhs) <= 1e-6 * scale


@pytest.mark.parametrize("name", ["ragged40x36", "osem64", "noatt_nopsf", "trans_fov40x36"])
def test_sensitivity_parity(spect_lib, oracle_mod, cuda, name):
    g, f, mu, plan, og = _setup(spect_lib, oracle_mod, cuda, name)
    for m in range(g.n_subsets):
        sel = oracle_mod.subset_angles(g.n_angles, g.n_subsets, m)
        s = plan.sensitivity(m).cpu().numpy()
        ref = oracle_mod.back(np.ones((len(sel), g.n, g.nz)), og, sel)
        assert_close(s, ref, TOL, (name, m))
    s_all = plan.sensitivity(-1).cpu().numpy()
    ref = oracle_mod.back(np.ones((g.n_angles, g.n, g.nz)), og)
    assert_close(s_all, ref, TOL, (name, "all"))


def _osem_case(spect, oracle, dev, n, n_angles, iters, M, counts, seed):
    from paper_2309_01977_gb300 import phantom
    g = spect.Geometry(n=n, nz=n, n_angles=n_angles, n_subsets=M)
    f_raw, mu = phantom_inputs(n, n, seed)
    og = oracle_geom(oracle, g, mu)
    hf = oracle.forward(f_raw, og)
    _, y, s, _ = phantom.make_counts(f_raw, hf, counts, 0.05, seed)
    s = float(np.float32(s))
    plan = spect.Plan(g, _t(mu, dev))
    return g, plan, og, y, s


@pytest.mark.parametrize("n, n_angles, iters, counts, seed", [
    (64, 64, 2, 2e6, 1),      # the 64^3 workload, full run
    (128, 120, 4, 1e7, 2),    # the 128^3 workload, full run
])
def test_osem_parity_and_conservation(spect_lib, oracle_mod, cuda, n, n_angles, iters, counts, seed):
    M = 8
    g, plan, og, y, s = _osem_case(spect_lib, oracle_mod, cuda, n, n_angles, iters, M, counts, seed)
    yd = _t(y, cuda)
    x = torch.ones((n, n, n), device=cuda)
    total = iters * M
    diag = plan.osem(yd, s, x, 0, total, diag=True).cpu().numpy()
    ref, ref_diag = oracle_mod.osem(y, s, og, M, 0, total)
    assert_close(x.cpu().numpy(), ref, 2e-5, "osem image")
    np.testing.assert_allclose(diag, ref_diag, rtol=2e-5)
    # conservation on the GPU: sum over S_m of H_m x_new equals sum y * p / (p + s)
    x2 = torch.ones((n, n, n), device=cuda)
    for t in range(3):
        d = plan.osem(yd, s, x2, t, 1, diag=True).cpu().numpy()[0]
        p_new = plan.forward(x2, t % M).double().sum().item()
        assert p_new == pytest.approx(d[2], rel=2e-6)
        sel = plan.subset_angles(t % M)
        assert d[1] == pytest.approx(float(y[sel].sum()), rel=1e-12)


def test_osem_resume_is_bitwise(spect_lib, oracle_mod, cuda):
    g, plan, og, y, s = _osem_case(spect_lib, oracle_mod, cuda, 64, 64, 2, 8, 2e6, 1)
    yd = _t(y, cuda)
    a = torch.ones((64, 64, 64), device=cuda)
    plan.osem(yd, s, a, 0, 6)
    b = torch.ones((64, 64, 64), device=cuda)
    plan.osem(yd, s, b, 0, 2)
    plan.osem(yd, s, b, 2, 4)
    assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["ragged40x36", "tiled132x44"])
def test_forward_is_deterministic_and_batched(spect_lib, oracle_mod, cuda, name):
    g, f, mu, plan, og = _setup(spect_lib, oracle_mod, cuda, name)
    rng = np.random.Generator(np.random.PCG64(8))
    xs = _t(rng.uniform(size=(3, g.n, g.n, g.nz)), cuda)
    pb = plan.forward(xs)
    for b in range(3):
        p1 = plan.forward(xs[b].contiguous())
        assert torch.equal(p1, pb[b])
        assert torch.equal(p1, plan.forward(xs[b].contiguous()))
    q = _t(rng.uniform(size=(3, g.n_angles, g.n, g.nz)), cuda)
    bb = plan.back(q)
    for b in range(3):
        assert torch.equal(plan.back(q[b].contiguous()), bb[b])


def test_z_tiled_planes_192(spect_lib, oracle_mod, cuda):
    """192^3 planes do not fit shared memory whole: z tiles with PSF halos."""
    g = spect_lib.Geometry(n=192, nz=192, n_angles=128, n_subsets=32)
    f, mu = phantom_inputs(192, 192, 5)
    plan = spect_lib.Plan(g, _t(mu, cuda))
    og = oracle_geom(oracle_mod, g, mu)
    sel = plan.subset_angles(3)
    p = plan.forward(_t(f, cuda), 3).cpu().numpy()
    assert_close(p, oracle_mod.forward(f, og, sel), TOL, "forward 192")
    q = f32(np.random.Generator(np.random.PCG64(9)).uniform(size=(len(sel), 192, 192)))
    b = plan.back(_t(q, cuda), 3).cpu().numpy()
    assert_close(b, oracle_mod.back(q, og, sel), TOL, "back 192")


def test_poisson_ll_and_gradient(spect_lib, oracle_mod, cuda):
    g, plan, og, y, s = _osem_case(spect_lib, oracle_mod, cuda, 64, 64, 1, 8, 2e6, 1)
    rng = np.random.Generator(np.random.PCG64(10))
    p = f32(rng.uniform(0.0, 5.0, size=y.shape))
    p[0, 0, :5] = 0.0
    ll, grad = plan.poisson_ll(_t(y, cuda), _t(p, cuda), s, grad=True)
    ref = oracle_mod.poisson_ll(y, p, s)
    assert ll.item() == pytest.approx(ref, rel=1e-6)
    ref_g = y / (p + s) - 1.0
    assert rel_l2(grad.cpu().numpy(), ref_g) <= 1e-6


def test_bad_pointers_rejected(spect_lib, cuda):
    g = spect_lib.Geometry(n=16, nz=16, n_angles=4, attenuation=False)
    plan = spect_lib.Plan(g)
    x = torch.zeros(16 * 16 * 16 + 1, device=cuda)
    out = torch.zeros(4 * 16 * 16 + 4, device=cuda)
    with pytest.raises(spect_lib.SpectError) as e:
        spect_lib.spect_forward(plan.handle, x[1:], out[:4 * 256], -1, 1)
    assert e.value.status == spect_lib.SPECT_EINVAL
    with pytest.raises(spect_lib.SpectError):
        spect_lib.spect_forward(plan.handle, x[:4096], out, 5, 1)
    with pytest.raises(spect_lib.SpectError):
        spect_lib.spect_forward(plan.handle, x[:4096], out, 0, 0)


def test_plan_reuse_with_new_mu_and_device_scatter(spect_lib, oracle_mod, cuda):
    """spect_plan_set_mu equals a fresh plan bitwise; spect_osem_run_dev equals spect_osem_run."""
    g = spect_lib.Geometry(n=40, nz=36, n_angles=12, n_subsets=3, psf_slope=0.1)
    f1, mu1 = phantom_inputs(40, 36, 51)
    f2, mu2 = phantom_inputs(40, 36, 52)
    p1 = spect_lib.Plan(g, _t(mu1, cuda))
    p2 = spect_lib.Plan(g, _t(mu2, cuda))
    spect_lib.spect_plan_set_mu(p1.handle, _t(mu2, cuda))
    x = _t(f2, cuda)
    assert torch.equal(p1.forward(x), p2.forward(x))
    assert torch.equal(p1.sensitivity(1), p2.sensitivity(1))
    y = p2.forward(x) + 0.5
    a = torch.ones((40, 40, 36), device=cuda)
    b = torch.ones((40, 40, 36), device=cuda)
    p2.osem(y, 0.25, a, 0, 5)
    spect_lib.spect_osem_run_dev(p1.handle, y, torch.full((1,), 0.25, device=cuda), b, 0, 5)
    assert torch.equal(a, b)


def test_osem_with_trans_and_fov(spect_lib, oracle_mod, cuda):
    """OSEM through T_trans and T_fov: the masked forward feeds the ratio and
    the count sums, the back projection weights the ratio again.  The field
    of view is a detector band that follows each angle's shifted centre (the
    random per-angle masks of the projector cases leave voxels seen only
    through PSF tails at a mask edge, where FP32 rounding of the tiny
    bilinear weights, not the method, decides the OSEM ratio)."""
    from paper_2309_01977_gb300 import phantom
    n, na, M = 48, 24, 4
    shifts = _shifts(na, 2.5, 44)
    g = spect_lib.Geometry(n=n, nz=n, n_angles=na, n_subsets=M, det_shifts=shifts,
                           fov_mask=_band_mask(na, n, n, shifts, 18.0))
    f_raw, mu = phantom_inputs(n, n, 22)
    og = oracle_geom(oracle_mod, g, mu)
    hf = oracle_mod.forward(f_raw, og)
    _, y, s, _ = phantom.make_counts(f_raw, hf, 2e6, 0.05, 22)
    s = float(np.float32(s))
    plan = spect_lib.Plan(g, _t(mu, cuda))
    x = torch.ones((n, n, n), device=cuda)
    diag = plan.osem(_t(y, cuda), s, x, 0, 2 * M, diag=True).cpu().numpy()
    ref, ref_diag = oracle_mod.osem(y, s, og, M, 0, 2 * M)
    assert_close(x.cpu().numpy(), ref, 2e-5, "osem trans+fov")
    np.testing.assert_allclose(diag, ref_diag, rtol=2e-5)


def test_trans_fov_reject_bad_values(spect_lib, cuda):
    bad_mask = np.ones((4, 16, 16), dtype=np.float32)
    bad_mask[1, 2, 3] = -1.0
    for kw in (dict(det_shifts=[0.0, float("nan"), 0.0, 0.0]), dict(det_shifts=[0.0, 100.0, 0.0, 0.0]),
               dict(fov_mask=bad_mask)):
        g = spect_lib.Geometry(n=16, nz=16, n_angles=4, attenuation=False, **kw)
        with pytest.raises(spect_lib.SpectError) as e:
            spect_lib.Plan(g)
        assert e.value.status == spect_lib.SPECT_EINVAL
