"""spect_poisson_ll_noalloc: the Poisson log-likelihood for callers that
cannot allocate device memory (their framework owns the device memory, or a
real-time loop cannot afford an allocation).  It keeps its partial sums in
scratch built into the library instead of a plan's memory.  Checked against
spect_poisson_ll, which uses a plan, on two calls in a row: the second call
must not see anything the first left in the shared scratch.

This file runs last (collection order), so a failure here leaves every other
test already run; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _inputs(count, seed, dev):
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.uniform(0.0, 8.0, size=count).astype(np.float32)
    y = rng.poisson(p + 0.2).astype(np.float32)
    p[:7] = 0.0  # a few empty bins: the ratio and log terms still follow the definition
    y[3] = 0.0
    return torch.from_numpy(y).to(dev), torch.from_numpy(p).to(dev)


def test_noalloc_matches_plan_entry_point_twice(spect_lib, cuda):
    g = spect_lib.Geometry(n=16, nz=16, n_angles=4, attenuation=False)
    plan = spect_lib.Plan(g)
    # calls in a row with different sizes and data: fewer blocks than the
    # call before (stale partials beyond the count must be ignored), then
    # more blocks again
    for count, seed, s in [(1_000_003, 1, 0.25), (262_144, 2, 0.1), (3_000_001, 3, 0.5)]:
        y, p = _inputs(count, seed, cuda)
        ll_ref = torch.zeros(1, device=cuda, dtype=torch.float64)
        gr_ref = torch.empty_like(p)
        spect_lib.spect_poisson_ll(plan.handle, y, p, s, ll_ref, gr_ref)
        ll = torch.full((1,), float("nan"), device=cuda, dtype=torch.float64)
        gr = torch.full_like(p, float("nan"))
        spect_lib.spect_poisson_ll_noalloc(y, p, s, ll, gr)
        torch.cuda.synchronize()
        assert ll.item() == pytest.approx(ll_ref.item(), rel=1e-12)
        assert torch.allclose(gr, gr_ref, rtol=1e-6, atol=1e-6)
        # without a gradient buffer the sum is the same
        ll2 = torch.zeros(1, device=cuda, dtype=torch.float64)
        spect_lib.spect_poisson_ll_noalloc(y, p, s, ll2, None)
        torch.cuda.synchronize()
        assert ll2.item() == ll.item()
    plan.close()


def test_noalloc_rejects_counts_beyond_its_scratch(spect_lib, cuda):
    lib = spect_lib.load()
    ll = torch.zeros(1, device=cuda, dtype=torch.float64)
    y = torch.zeros(4, device=cuda)
    too_many = 4096 * 16384 + 1
    rc = lib.spect_poisson_ll_noalloc(y.data_ptr(), y.data_ptr(), 0.0, too_many, ll.data_ptr(), None, None)
    assert rc == spect_lib.SPECT_EINVAL
    assert b"exceeds" in lib.spect_last_error()


def test_noalloc_empty_count_gives_zero(spect_lib, cuda):
    """count 0: no partial block runs, the total of nothing is 0 (whatever an
    earlier call left in the scratch)."""
    y, p = _inputs(100_000, 4, cuda)
    ll = torch.zeros(1, device=cuda, dtype=torch.float64)
    spect_lib.spect_poisson_ll_noalloc(y, p, 0.25, ll, None)
    ll0 = torch.full((1,), float("nan"), device=cuda, dtype=torch.float64)
    lib = spect_lib.load()
    rc = lib.spect_poisson_ll_noalloc(y.data_ptr(), p.data_ptr(), 0.25, 0, ll0.data_ptr(), None,
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == spect_lib.SPECT_OK
    torch.cuda.synchronize()
    assert ll0.item() == 0.0


def test_noalloc_rejects_misaligned_buffers(spect_lib, cuda):
    lib = spect_lib.load()
    y, p = _inputs(1000, 5, cuda)
    ll = torch.zeros(1, device=cuda, dtype=torch.float64)
    rc = lib.spect_poisson_ll_noalloc(y.data_ptr() + 4, p.data_ptr(), 0.25, 100, ll.data_ptr(), None, None)
    assert rc == spect_lib.SPECT_EINVAL
    assert b"aligned" in lib.spect_last_error()
