"""MAP reconstruction on the GPU (OSMAPOSL and BSREM with nearest-neighbour
priors, Eq. PGA and Table 1) against the FP64 oracle, through the C ABI.

  - the prior gradient (quadratic, relative difference) matches the oracle's
    to relative L2 1e-5 (FP32 stencil, ragged sizes);
  - OSMAPOSL with beta = 0 is bitwise the OSEM run (same update arithmetic);
  - OSMAPOSL-RDP and BSREM-RDP (beta = 0.3, gamma = 2, the paper's values)
    and OSMAPOSL-quadratic on the 64^3 workload for 2 x 8 subiterations match
    the oracle's images (relative L2 bounds in the tests, with the measured
    errors printed);
  - a resumed BSREM run equals one call bitwise.
"""
import numpy as np
import pytest

from helpers import f32, oracle_geom, phantom_inputs, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(dev)


@pytest.mark.parametrize("prior", ["quadratic", "rdp"])
def test_prior_gradient_parity(spect_lib, oracle_mod, cuda, prior):
    f, _ = phantom_inputs(40, 36, 31)
    x = f32(f + np.random.Generator(np.random.PCG64(32)).uniform(0.0, 0.5, size=f.shape))
    g = torch.empty((40, 40, 36), device=cuda)
    spect_lib.spect_prior_grad(_t(x, cuda), prior, g, delta=0.7, gamma=2.0)
    ref = oracle_mod.prior_grad(x, prior, 0.7, 2.0)
    err = rel_l2(g.cpu().numpy(), ref)
    print("prior gradient %s: rel L2 %.2e" % (prior, err))
    assert err <= 1e-5


def _case(spect, oracle, dev, seed=1):
    from paper_2309_01977_gb300 import phantom
    n, na, M = 64, 64, 8
    g = spect.Geometry(n=n, nz=n, n_angles=na, n_subsets=M)
    f_raw, mu = phantom_inputs(n, n, seed)
    og = oracle_geom(oracle, g, mu)
    _, y, s, _ = phantom.make_counts(f_raw, oracle.forward(f_raw, og), 2e6, 0.05, seed)
    s = float(np.float32(s))
    return g, spect.Plan(g, _t(mu, dev)), og, y, s


def test_osmaposl_without_prior_weight_is_osem_bitwise(spect_lib, oracle_mod, cuda):
    g, plan, og, y, s = _case(spect_lib, oracle_mod, cuda)
    yd = _t(y, cuda)
    a = torch.ones((64, 64, 64), device=cuda)
    plan.osem(yd, s, a, 0, 6)
    b = torch.ones((64, 64, 64), device=cuda)
    plan.map(yd, s, b, 0, 6, "osmaposl", "rdp", beta=0.0)
    assert torch.equal(a, b)


@pytest.mark.parametrize("algorithm, prior, beta, tol", [
    ("osmaposl", "rdp", 0.3, 2e-5),
    ("bsrem", "rdp", 0.3, 2e-5),
    ("osmaposl", "quadratic", 0.05, 2e-5),
])
def test_map_parity_64(spect_lib, oracle_mod, cuda, algorithm, prior, beta, tol):
    g, plan, og, y, s = _case(spect_lib, oracle_mod, cuda)
    ref = oracle_mod.map_recon(y, s, og, 8, 0, 16, algorithm, prior, beta, delta=1.0, gamma=2.0, alpha0=1.0)
    x = torch.ones((64, 64, 64), device=cuda)
    plan.map(_t(y, cuda), s, x, 0, 16, algorithm, prior, beta, delta=1.0, gamma=2.0, alpha0=1.0)
    plan.check()
    err = rel_l2(x.cpu().numpy(), ref)
    print("%s-%s beta %.2f, 2x8 at 64^3: image rel L2 vs FP64 %.2e" % (algorithm, prior, beta, err))
    assert err <= tol
    assert float(x.min()) >= 0.0


def test_bsrem_resume_is_bitwise(spect_lib, oracle_mod, cuda):
    g, plan, og, y, s = _case(spect_lib, oracle_mod, cuda)
    yd = _t(y, cuda)
    a = torch.ones((64, 64, 64), device=cuda)
    plan.map(yd, s, a, 0, 10, "bsrem", "rdp", 0.3)
    b = torch.ones((64, 64, 64), device=cuda)
    plan.map(yd, s, b, 0, 3, "bsrem", "rdp", 0.3)
    plan.map(yd, s, b, 3, 7, "bsrem", "rdp", 0.3)
    assert torch.equal(a, b)


def test_map_rejects_bad_parameters(spect_lib, cuda):
    g = spect_lib.Geometry(n=32, nz=32, n_angles=8, n_subsets=2, attenuation=False)
    plan = spect_lib.Plan(g, None)
    y = torch.ones((8, 32, 32), device=cuda)
    x = torch.ones((32, 32, 32), device=cuda)
    for kw in [dict(algorithm="bsrem", prior="rdp", beta=-1.0), dict(algorithm="bsrem", prior="rdp", beta=0.3, alpha0=0.0),
               dict(algorithm="osmaposl", prior="quadratic", beta=0.3, delta=0.0)]:
        with pytest.raises(spect_lib.SpectError) as e:
            plan.map(y, 0.1, x, 0, 1, **kw)
        assert e.value.status == spect_lib.SPECT_EINVAL
