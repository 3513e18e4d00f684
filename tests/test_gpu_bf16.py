"""BF16 tensor-core PSF path (SPECT_FLAG_PSF_BF16) against the FP64 oracle.

The PSF runs as banded-Toeplitz BF16 GEMMs with FP32 accumulation; the
rotation, attenuation, ratio and update stay FP32 and the attenuation prefix
sums run in FP64.  Bar (the precision target of this path): relative L2 error
<= 1e-3 against the FP64 oracle for projections, back projections and the
full 128^3 OSEM image.  The measured errors are printed for the record.
"""
import math

import numpy as np
import pytest

from helpers import f32, oracle_geom, phantom_inputs, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_BF16 = 1e-3


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(dev)


@pytest.mark.parametrize("n, nz, na, M, subset, seed", [
    (64, 64, 64, 8, 0, 1),
    (96, 96, 96, 8, 3, 1000),
    (128, 128, 120, 8, 0, 2),
    (64, 40, 12, 3, -1, 7),   # axial size below 128 and not a multiple of 16
    (64, 64, 16, 4, -1, 8),   # non-circular orbit (per-angle Toeplitz tiles)
    (64, 48, 16, 4, -1, 9),   # non-central projections (T_trans) and a field-of-view mask (T_fov)
    (32, 32, 16, 2, 1, 12),   # the smallest plane (n = 32): one 64-column swizzle block
])
def test_bf16_projection_parity(spect_lib, oracle_mod, cuda, n, nz, na, M, subset, seed):
    offs = [3.0 + 2.0 * math.cos(2 * 2 * math.pi * a / na) for a in range(na)] if seed == 8 else None
    kw = {}
    if seed == 9:
        rng = np.random.Generator(np.random.PCG64(9))
        kw["det_shifts"] = [float(v) for v in rng.uniform(-4.0, 4.0, size=na)]
        mask = np.zeros((na, n, nz), dtype=np.float32)
        mask[:, 6:58, 4:44] = 1.0
        kw["fov_mask"] = mask
    g = spect_lib.Geometry(n=n, nz=nz, n_angles=na, n_subsets=M, psf_bf16=True, atten_f64=True, det_offsets=offs,
                           **kw)
    f, mu = phantom_inputs(n, nz, seed)
    plan = spect_lib.Plan(g, _t(mu, cuda))
    og = oracle_geom(oracle_mod, g, mu)
    sel = plan.subset_angles(subset)
    p = plan.forward(_t(f, cuda), subset).cpu().numpy()
    ref = oracle_mod.forward(f, og, sel)
    e_fwd = rel_l2(p, ref)
    q = f32(np.random.Generator(np.random.PCG64(seed)).uniform(0.5, 1.5, size=(len(sel), n, nz)))
    b = plan.back(_t(q, cuda), subset).cpu().numpy()
    e_back = rel_l2(b, oracle_mod.back(q, og, sel))
    plan.check()
    print("bf16 %dx%d: forward %.2e back %.2e" % (n, nz, e_fwd, e_back))
    assert e_fwd <= TOL_BF16 and e_back <= TOL_BF16
    # element-wise: a wrong plane, chunk or tile shows up locally
    bref = oracle_mod.back(q, og, sel)
    assert np.max(np.abs(p - ref)) <= 10 * TOL_BF16 * np.max(np.abs(ref))
    assert np.max(np.abs(b - bref)) <= 10 * TOL_BF16 * np.max(np.abs(bref))


def test_bf16_single_angle_batch(spect_lib, oracle_mod, cuda):
    """One angle per subset (more depth chunks than planes, so some CTAs have
    no plane) and a batch of two volumes / two projection sets."""
    n, nz, na, M = 64, 64, 8, 8
    g = spect_lib.Geometry(n=n, nz=nz, n_angles=na, n_subsets=M, psf_bf16=True, atten_f64=True)
    f0, mu = phantom_inputs(n, nz, 13)
    f1, _ = phantom_inputs(n, nz, 14)
    plan = spect_lib.Plan(g, _t(mu, cuda))
    og = oracle_geom(oracle_mod, g, mu)
    for subset in (0, 5):
        sel = plan.subset_angles(subset)
        assert len(sel) == 1
        p = plan.forward(_t(np.stack([f0, f1]), cuda), subset).cpu().numpy().reshape(2, 1, n, nz)
        q = f32(np.random.Generator(np.random.PCG64(subset)).uniform(0.5, 1.5, size=(2, 1, n, nz)))
        b = plan.back(_t(q, cuda), subset).cpu().numpy().reshape(2, n, n, nz)
        for k, f in enumerate((f0, f1)):
            ref = oracle_mod.forward(f, og, sel)
            bref = oracle_mod.back(q[k], og, sel)
            print("bf16 one angle, entry %d: forward %.2e back %.2e" % (k, rel_l2(p[k], ref), rel_l2(b[k], bref)))
            assert rel_l2(p[k], ref) <= TOL_BF16 and rel_l2(b[k], bref) <= TOL_BF16
            assert np.max(np.abs(p[k] - ref)) <= 10 * TOL_BF16 * np.max(np.abs(ref))
    plan.check()


def test_bf16_adjoint_and_sensitivity(spect_lib, oracle_mod, cuda):
    g = spect_lib.Geometry(n=64, nz=64, n_angles=32, n_subsets=4, psf_bf16=True)
    f, mu = phantom_inputs(64, 64, 3)
    plan = spect_lib.Plan(g, _t(mu, cuda))
    rng = np.random.Generator(np.random.PCG64(4))
    x = _t(rng.uniform(size=(64, 64, 64)), cuda)
    y = _t(rng.uniform(size=(32, 64, 64)), cuda)
    lhs = (plan.forward(x).double() * y.double()).sum().item()
    rhs = (x.double() * plan.back(y).double()).sum().item()
    assert abs(lhs - rhs) <= 1e-3 * abs(lhs)
    og = oracle_geom(oracle_mod, g, mu)
    sel = oracle_mod.subset_angles(32, 4, 1)
    assert rel_l2(plan.sensitivity(1).cpu().numpy(), oracle_mod.back(np.ones((len(sel), 64, 64)), og, sel)) <= TOL_BF16


def test_bf16_osem_128_image_error(spect_lib, oracle_mod, cuda):
    """The 128^3 x 120-angle, 4 x 8 OSEM with the BF16 PSF against the FP64 oracle."""
    from paper_2309_01977_gb300 import phantom
    n, na, M, iters = 128, 120, 8, 4
    f_raw, mu = phantom_inputs(n, n, 2)
    g32 = spect_lib.Geometry(n=n, nz=n, n_angles=na, n_subsets=M)
    og = oracle_geom(oracle_mod, g32, mu)
    hf = oracle_mod.forward(f_raw, og)
    _, y, s, _ = phantom.make_counts(f_raw, hf, 1e7, 0.05, 2)
    s = float(np.float32(s))
    ref, _ = oracle_mod.osem(y, s, og, M, 0, iters * M)
    yd = _t(y, cuda)
    gb = spect_lib.Geometry(n=n, nz=n, n_angles=na, n_subsets=M, psf_bf16=True, atten_f64=True)
    plan = spect_lib.Plan(gb, _t(mu, cuda))
    x = torch.ones((n, n, n), device=cuda)
    plan.osem(yd, s, x, 0, iters * M)
    plan.check()
    err = rel_l2(x.cpu().numpy(), ref)
    print("bf16 OSEM 128^3 4x8: image rel L2 vs FP64 %.3e" % err)
    assert err <= TOL_BF16
    assert math.isfinite(err)
