"""Autograd projector (the batch-of-4, 192^3, 128-angle differentiation
workload and a small case the oracle can finite-difference).

  - small case (2 x 32^3, 24 angles): the autograd gradient of the Poisson
    log-likelihood equals the oracle's FP64 gradient H^T(y/(Hx+s)) - H^T 1
    (relative L2 <= 1e-5) and central finite differences of the oracle's FP64
    log-likelihood on 32 seeded voxels (relative 1e-4);
  - full size (4 x 192^3, 128 angles): one batch entry's gradient against
    the oracle's FP64 gradient (relative L2 <= 1e-5, every voxel within 1e-4
    of the largest) and central finite differences of the oracle's FP64
    log-likelihood on 32 seeded voxels; the dot-product adjoint test through
    autograd, the identity <x, grad L> = sum p (y/(p+s) - 1) for the linear H,
    and batch independence (each batch entry's gradient equals the gradient of
    that volume alone, bitwise).
"""
import numpy as np
import pytest

from helpers import assert_close, f32, one_hot_projection, oracle_geom, phantom_inputs, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).to(dev)


def test_autograd_gradient_matches_oracle_and_finite_differences(spect_lib, oracle_mod, cuda):
    from paper_2309_01977_gb300 import autograd, phantom
    n, na, batch = 32, 24, 2
    g = spect_lib.Geometry(n=n, nz=n, n_angles=na, psf_slope=0.05)
    f0, mu = phantom_inputs(n, n, 21)
    og = oracle_geom(oracle_mod, g, mu)
    plan = spect_lib.Plan(g, _t(mu, cuda))
    hf = oracle_mod.forward(f0, og)
    _, y, s, _ = phantom.make_counts(f0, hf, 2e5, 0.05, 21)
    s = float(np.float32(s))
    rng = np.random.Generator(np.random.PCG64(22))
    xs = f32(rng.uniform(0.5, 1.5, size=(batch, n, n, n)) * (f0.max() / 2 + 0.1))
    x = _t(xs, cuda).requires_grad_(True)
    yb = _t(np.stack([y] * batch), cuda)
    loss = autograd.poisson_loss(x, yb, s, plan)
    loss.backward()
    grad = x.grad.cpu().numpy()
    for b in range(batch):
        p = oracle_mod.forward(xs[b], og)
        ref = oracle_mod.back(y / (p + s), og) - oracle_mod.back(np.ones_like(p), og)
        assert rel_l2(grad[b], ref) <= 1e-5
        # finite differences of the FP64 oracle likelihood on 32 voxels
        vox = rng.integers(0, n, size=(32, 3))
        for q in vox[:32 if b == 0 else 8]:
            q = tuple(q)
            h = 1e-2 * max(xs[b][q], 1e-2)
            xp = xs[b].copy(); xp[q] += h
            xm = xs[b].copy(); xm[q] -= h
            fd = (oracle_mod.poisson_ll(y, oracle_mod.forward(xp, og), s)
                  - oracle_mod.poisson_ll(y, oracle_mod.forward(xm, og), s)) / (2 * h)
            assert grad[b][q] == pytest.approx(fd, rel=1e-4, abs=1e-4 * np.abs(ref).max())
    # the likelihood value itself
    ll_ref = sum(oracle_mod.poisson_ll(y, oracle_mod.forward(xs[b], og), s) for b in range(batch))
    assert loss.item() == pytest.approx(ll_ref, rel=1e-6)


def test_autograd_full_size_properties(spect_lib, cuda):
    """4 x 192^3 volumes, 128 angles, 192 x 192 bins."""
    from paper_2309_01977_gb300 import autograd
    n, na, batch = 192, 128, 4
    g = spect_lib.Geometry(n=n, nz=n, n_angles=na)
    f0, mu = phantom_inputs(n, n, 5)
    plan = spect_lib.Plan(g, _t(mu, cuda))
    rng = np.random.Generator(np.random.PCG64(5))
    x = (_t(f0, cuda)[None] * _t(rng.uniform(0.5, 1.5, size=(batch, 1, 1, 1)), cuda)).contiguous()
    x.requires_grad_(True)
    # dot-product adjoint test through autograd
    yv = _t(rng.uniform(0.0, 1.0, size=(batch, na, n, n)), cuda)
    proj = autograd.SpectProjector.apply(x, plan, -1)
    (hty,) = torch.autograd.grad((proj * yv).sum(), x)
    lhs = (proj.double() * yv.double()).sum().item()
    rhs = (x.detach().double() * hty.double()).sum().item()
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
    # Poisson gradient: <x, grad L> = sum p (y/(p+s) - 1) because H is linear
    with torch.no_grad():
        p = proj.detach()
        counts = torch.poisson(p + 1.0)
    s = 1.0
    x.grad = None
    loss = autograd.poisson_loss(x, counts, s, plan)
    loss.backward()
    gl = x.grad.detach()
    ident = (p.double() * (counts.double() / (p.double() + s) - 1.0)).sum().item()
    assert (x.detach().double() * gl.double()).sum().item() == pytest.approx(ident, rel=1e-5)
    # batch independence, bitwise
    x1 = x.detach()[2:3].clone().requires_grad_(True)
    autograd.poisson_loss(x1, counts[2:3].contiguous(), s, plan).backward()
    assert torch.equal(x1.grad[0], gl[2])


def test_autograd_full_size_gradient_matches_oracle(spect_lib, oracle_mod, cuda):
    """The 4 x 192^3, 128-angle batch: entry 2's gradient of the Poisson
    log-likelihood against the FP64 oracle.  The batch holds f0 times 1/2, 1,
    2 and 4 (powers of two, so that H x = scale H f0 holds exactly in the
    oracle and the counts come from the oracle's projection alone).  Central
    differences of the oracle's log-likelihood use H(x +- h e_v) = Hx +- h H e_v
    (H is linear), with H e_v from the oracle on the z slab the voxel's blur
    reaches."""
    from paper_2309_01977_gb300 import autograd
    n, na, batch, b = 192, 128, 4, 2
    g = spect_lib.Geometry(n=n, nz=n, n_angles=na)
    f0, mu = phantom_inputs(n, n, 5)
    og = oracle_geom(oracle_mod, g, mu)
    scales = np.array([0.5, 1.0, 2.0, 4.0])
    hf0 = oracle_mod.forward(f0, og)
    s = 0.5
    rng = np.random.Generator(np.random.PCG64(55))
    y = rng.poisson(hf0 + s).astype(np.float64)
    plan = spect_lib.Plan(g, _t(mu, cuda))
    x = _t(f0[None] * scales[:, None, None, None], cuda).requires_grad_(True)
    yb = _t(np.stack([y] * batch), cuda)
    loss = autograd.poisson_loss(x, yb, s, plan)
    loss.backward()
    grad = x.grad[b].cpu().numpy()
    plan.close()
    p = scales[b] * hf0
    ref = oracle_mod.back(y / (p + s), og) - oracle_mod.back(np.ones_like(p), og)
    print("grad192 entry %d: gradient rel L2 vs FP64 oracle %.2e" % (b, rel_l2(grad, ref)))
    assert_close(grad, ref, 1e-5, "grad192 gradient")
    # central finite differences of the oracle's FP64 log-likelihood
    rmax = oracle_mod.psf_rmax(n, og.sigma0, og.slope, og.nsigma)
    xb = f0 * scales[b]
    inside = np.argwhere(xb > 0)
    pick = inside[rng.choice(len(inside), 32, replace=False)]
    scale = np.abs(ref).max()
    for v in map(tuple, pick):
        c = one_hot_projection(oracle_mod, og, v, rmax)
        h = 1e-2 * xb[v]
        fd = (oracle_mod.poisson_ll(y, p + h * c, s) - oracle_mod.poisson_ll(y, p - h * c, s)) / (2 * h)
        assert grad[v] == pytest.approx(fd, rel=1e-4, abs=1e-5 * scale), v
