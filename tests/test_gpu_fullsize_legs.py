"""The benchmark's secondary legs at their full size (128^3 volume, 120
angles, 4 x 8 subiterations, 1e7 counts, seed 2), on the GPU against the
FP64 oracle through the C ABI, in the configurations bench.py times:

  - BSREM with the relative-difference prior, beta 0.3, gamma 2, alpha0 1
    (Eq. PGA, Table 1);
  - two photopeaks (Eq. extended_sm): the second sees 1.25 x mu through a
    sigma = 0.7 + 0.04 d collimator response with relative scale 0.6;
  - an elliptical orbit: detector offsets r(t) - n/2 from 4 to 20 voxels.

Bar: relative L2 of the image 2e-5, as for the OSEM workload.
"""
import numpy as np
import pytest

from helpers import f32, oracle_geom, phantom_inputs, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N, NA, M, ITERS, COUNTS, SEED = 128, 120, 8, 4, 1e7, 2


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(dev)


def _data(spect, oracle, g, f_raw, mu):
    from paper_2309_01977_gb300 import phantom
    og = oracle_geom(oracle, g, mu)
    _, y, s, _ = phantom.make_counts(f_raw, oracle.forward(f_raw, og), COUNTS, 0.05, SEED)
    return og, y, float(np.float32(s))


def test_bsrem_rdp_full_size(spect_lib, oracle_mod, cuda):
    g = spect_lib.Geometry(n=N, nz=N, n_angles=NA, n_subsets=M)
    f_raw, mu = phantom_inputs(N, N, SEED)
    og, y, s = _data(spect_lib, oracle_mod, g, f_raw, mu)
    plan = spect_lib.Plan(g, _t(mu, cuda))
    x = torch.ones((N, N, N), device=cuda)
    plan.map(_t(y, cuda), s, x, 0, ITERS * M, "bsrem", "rdp", beta=0.3, gamma=2.0, alpha0=1.0)
    plan.check()
    ref = oracle_mod.map_recon(y, s, og, M, 0, ITERS * M, "bsrem", "rdp", 0.3, delta=1.0, gamma=2.0, alpha0=1.0)
    err = rel_l2(x.cpu().numpy(), ref)
    print("BSREM-RDP 4x8 at 128^3: image rel L2 vs FP64 %.2e" % err)
    assert err <= 2e-5
    plan.close()


def test_two_photopeaks_full_size(spect_lib, oracle_mod, cuda):
    import dataclasses
    g1 = spect_lib.Geometry(n=N, nz=N, n_angles=NA, n_subsets=M)
    g2 = dataclasses.replace(g1, psf_sigma0=0.7, psf_slope=0.04)
    f_raw, mu = phantom_inputs(N, N, SEED)
    mu2 = f32(1.25 * mu)
    og1, y1, s1 = _data(spect_lib, oracle_mod, g1, f_raw, mu)
    og2 = oracle_geom(oracle_mod, g2, mu2)
    scale2 = 0.6
    # the second peak observes the same activity as the first
    f_scale = COUNTS / float(oracle_mod.forward(f_raw, og1).sum())
    ybar2 = scale2 * oracle_mod.forward(f_raw, og2) * f_scale
    s2 = float(np.float32(0.05 * ybar2.mean()))
    y2 = f32(np.random.Generator(np.random.PCG64(SEED + 104729)).poisson(ybar2 + s2))
    p1 = spect_lib.Plan(g1, _t(mu, cuda))
    p2 = spect_lib.Plan(g2, _t(mu2, cuda))
    x = torch.ones((N, N, N), device=cuda)
    spect_lib.spect_multi_osem_run([p1, p2], [1.0, scale2], [_t(y1, cuda), _t(y2, cuda)], [s1, s2], x, 0, ITERS * M)
    p1.check()
    p2.check()
    ref = oracle_mod.osem_multi([y1, y2], [s1, s2], [og1, og2], [1.0, scale2], M, 0, ITERS * M)
    err = rel_l2(x.cpu().numpy(), ref)
    print("two-photopeak OSEM 4x8 at 128^3: image rel L2 vs FP64 %.2e" % err)
    assert err <= 2e-5
    p1.close()
    p2.close()


def test_elliptical_orbit_full_size(spect_lib, oracle_mod, cuda):
    import dataclasses
    a, b = N / 2 + 4.0, N / 2 + 20.0
    t = 2.0 * np.pi * np.arange(NA) / NA
    r = a * b / np.sqrt((b * np.cos(t)) ** 2 + (a * np.sin(t)) ** 2)
    g = dataclasses.replace(spect_lib.Geometry(n=N, nz=N, n_angles=NA, n_subsets=M),
                            det_offsets=[float(v) for v in (r - N / 2)])
    f_raw, mu = phantom_inputs(N, N, SEED)
    og, y, s = _data(spect_lib, oracle_mod, g, f_raw, mu)
    plan = spect_lib.Plan(g, _t(mu, cuda))
    x = torch.ones((N, N, N), device=cuda)
    plan.osem(_t(y, cuda), s, x, 0, ITERS * M)
    plan.check()
    ref, _ = oracle_mod.osem(y, s, og, M, 0, ITERS * M)
    err = rel_l2(x.cpu().numpy(), ref)
    print("elliptical-orbit OSEM 4x8 at 128^3: image rel L2 vs FP64 %.2e" % err)
    assert err <= 2e-5
    plan.close()
