"""Guard bands around every device buffer a call reads or writes.

A stand-in for a memory sanitizer: each input and output of the projector
calls sits inside a larger allocation whose margins (64 KiB before and after)
hold a fixed NaN bit pattern.  After each call the margins must still hold
it bit for bit, and the inputs must be unchanged, so a kernel that writes
past the end (or before the start) of a buffer, or into a buffer it only
reads, is caught on the small and ragged shapes where tails occur: a ragged
FP32 plane, a plane tiled along z, non-central projections with a
field-of-view mask, and the BF16 tensor-core path with an axial size below
128.
"""
import numpy as np
import pytest

from helpers import phantom_inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GUARD = 16384  # floats of margin on each side (64 KiB, a multiple of 4: buffers stay 16-byte aligned)
SENTINEL = 0x7FBADBAD  # a NaN bit pattern no kernel writes


class Guarded:
    """A float32 device tensor of `shape` inside sentinel margins."""

    def __init__(self, shape, dev, values=None):
        self.count = int(np.prod(shape))
        self.raw = torch.empty(self.count + 2 * GUARD, dtype=torch.float32, device=dev)
        self.raw.view(torch.int32).fill_(SENTINEL)
        self.t = self.raw[GUARD:GUARD + self.count].view(shape)
        if values is not None:
            self.t.copy_(torch.as_tensor(np.ascontiguousarray(values, dtype=np.float32)))

    def margins_intact(self) -> bool:
        bits = self.raw.view(torch.int32)
        lo, hi = bits[:GUARD], bits[GUARD + self.count:]
        return bool(torch.all(lo == SENTINEL).item()) and bool(torch.all(hi == SENTINEL).item())


CASES = {
    "ragged40x36": dict(n=40, nz=36, n_angles=12, n_subsets=3, psf_slope=0.1),
    "tiled132x44": dict(n=132, nz=44, n_angles=9, n_subsets=3),
    "trans_fov40x36": dict(n=40, nz=36, n_angles=8, n_subsets=2),
    "bf16_64x40": dict(n=64, nz=40, n_angles=12, n_subsets=3, psf_bf16=True, atten_f64=True),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_calls_stay_inside_their_buffers(spect_lib, cuda, name):
    kw = dict(CASES[name])
    n, nz, na = kw["n"], kw["nz"], kw["n_angles"]
    if name == "trans_fov40x36":
        rng = np.random.Generator(np.random.PCG64(21))
        kw["det_shifts"] = [float(v) for v in rng.uniform(-3.0, 3.0, size=na)]
        mask = np.zeros((na, n, nz), dtype=np.float32)
        mask[:, 3:37, 2:34] = 1.0
        kw["fov_mask"] = mask
    g = spect_lib.Geometry(**kw)
    f, mu = phantom_inputs(n, nz, 31)
    mu_g = Guarded((n, n, nz), cuda, mu)
    plan = spect_lib.Plan(g, mu_g.t)
    x_g = Guarded((n, n, nz), cuda, f)
    bufs = [mu_g, x_g]
    # forward and back projections, all angles and one subset
    for subset in (-1, 1):
        ns = len(plan.subset_angles(subset))
        p_g = Guarded((ns, n, nz), cuda)
        plan.forward(x_g.t, subset, out=p_g.t)
        b_g = Guarded((n, n, nz), cuda)
        plan.back(p_g.t, subset, out=b_g.t)
        bufs += [p_g, b_g]
    # OSEM: counts and the image in place
    y = np.random.Generator(np.random.PCG64(5)).poisson(20.0, size=(na, n, nz)).astype(np.float32)
    y_g = Guarded((na, n, nz), cuda, y)
    img_g = Guarded((n, n, nz), cuda, np.ones((n, n, nz), dtype=np.float32))
    plan.osem(y_g.t, 0.5, img_g.t, 0, 2 * kw["n_subsets"])
    bufs += [y_g, img_g]
    torch.cuda.synchronize()
    plan.check()
    assert all(b.margins_intact() for b in bufs), "a call wrote outside its buffer"
    # inputs that the calls only read are unchanged
    assert np.array_equal(x_g.t.cpu().numpy(), f)
    assert np.array_equal(y_g.t.cpu().numpy(), y)
    assert np.array_equal(mu_g.t.cpu().numpy(), mu)
    assert bool(torch.isfinite(img_g.t).all().item())
    plan.close()
