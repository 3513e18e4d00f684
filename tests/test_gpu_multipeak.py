"""OSEM over several SPECT photopeaks (the extended system matrix of
Sec. 2.1.1) on the GPU against the FP64 oracle, through the C ABI.

Two peaks with different attenuation (mu at each energy) and PSF models and
relative scales 1 and 0.6: the image after 2 x 4 subiterations matches the
oracle's multi-peak OSEM to relative L2 2e-5; one peak with scale 1 is
bitwise plain OSEM; a plan listed twice is rejected.
"""
import numpy as np
import pytest

from helpers import f32, oracle_geom, phantom_inputs, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(dev)


def _peaks(spect, oracle, dev):
    n, na, M = 48, 24, 4
    f, mu = phantom_inputs(n, n, 41)
    mu2 = f32(0.8 * mu)
    g1 = spect.Geometry(n=n, nz=n, n_angles=na, n_subsets=M, psf_sigma0=0.5, psf_slope=0.03)
    g2 = spect.Geometry(n=n, nz=n, n_angles=na, n_subsets=M, psf_sigma0=0.7, psf_slope=0.05)
    o1, o2 = oracle_geom(oracle, g1, mu), oracle_geom(oracle, g2, mu2)
    rng = np.random.Generator(np.random.PCG64(42))
    scales = [1.0, 0.6]
    y1 = f32(rng.poisson(oracle.forward(f, o1) * 20.0 + 0.5))
    y2 = f32(rng.poisson(scales[1] * oracle.forward(f, o2) * 20.0 + 0.5))
    s = [0.5, 0.5]
    p1 = spect.Plan(g1, _t(mu, dev))
    p2 = spect.Plan(g2, _t(mu2, dev))
    return (p1, p2), (o1, o2), (y1, y2), s, scales


def test_two_peaks_match_oracle(spect_lib, oracle_mod, cuda):
    plans, ogs, ys, s, scales = _peaks(spect_lib, oracle_mod, cuda)
    ref = oracle_mod.osem_multi(list(ys), s, list(ogs), scales, 4, 0, 8)
    x = torch.ones((48, 48, 48), device=cuda)
    spect_lib.spect_multi_osem_run(list(plans), scales, [_t(y, cuda) for y in ys], s, x, 0, 8)
    for p in plans:
        p.check()
    err = rel_l2(x.cpu().numpy(), ref)
    print("two-peak OSEM 2x4 at 48^3: image rel L2 vs FP64 %.2e" % err)
    assert err <= 2e-5


def test_one_peak_is_plain_osem_bitwise(spect_lib, oracle_mod, cuda):
    plans, ogs, ys, s, scales = _peaks(spect_lib, oracle_mod, cuda)
    yd = _t(ys[0], cuda)
    a = torch.ones((48, 48, 48), device=cuda)
    plans[0].osem(yd, s[0], a, 0, 6)
    b = torch.ones((48, 48, 48), device=cuda)
    spect_lib.spect_multi_osem_run([plans[0]], [1.0], [yd], [s[0]], b, 0, 6)
    assert torch.equal(a, b)


def test_repeated_plan_is_rejected(spect_lib, oracle_mod, cuda):
    plans, ogs, ys, s, scales = _peaks(spect_lib, oracle_mod, cuda)
    x = torch.ones((48, 48, 48), device=cuda)
    yd = _t(ys[0], cuda)
    with pytest.raises(spect_lib.SpectError) as e:
        spect_lib.spect_multi_osem_run([plans[0], plans[0]], [1.0, 1.0], [yd, yd], [0.5, 0.5], x, 0, 1)
    assert e.value.status == spect_lib.SPECT_EINVAL
