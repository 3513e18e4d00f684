"""One plan on several streams at once (the boundary's concurrency
contract): each stream has its own scratch, so forward projections, back
projections and OSEM runs queued on two streams without any ordering between
them give bitwise the results of the same calls run one after another.
The 128^3 x 120-angle geometry keeps every launch long enough for the two
streams' kernels to overlap on the device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _plan(spect, dev, n=128, na=120, M=8):
    from paper_2309_01977_gb300 import phantom
    f, mu = phantom.make_phantom(n, n, 2)
    g = spect.Geometry(n=n, nz=n, n_angles=na, n_subsets=M)
    return spect.Plan(g, torch.from_numpy(mu.astype(np.float32)).to(dev)), torch.from_numpy(f.astype(np.float32)).to(dev)


def test_two_streams_equal_serial_bitwise(spect_lib, cuda):
    plan, f = _plan(spect_lib, cuda)
    rng = np.random.Generator(np.random.PCG64(3))
    xs = [f * float(1 + k) + torch.from_numpy(rng.uniform(0, 0.1, size=f.shape).astype(np.float32)).to(cuda)
          for k in range(2)]
    qs = [torch.from_numpy(rng.uniform(0.5, 1.5, size=(120, 128, 128)).astype(np.float32)).to(cuda) for _ in range(2)]
    # serial references on the current stream
    ref_p = [plan.forward(x) for x in xs]
    ref_b = [plan.back(q) for q in qs]
    ref_s = [plan.forward(x, 3) for x in xs]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for rep in range(3):
        outs_p = [torch.empty_like(r) for r in ref_p]
        outs_b = [torch.empty_like(r) for r in ref_b]
        outs_s = [torch.empty_like(r) for r in ref_s]
        torch.cuda.synchronize()
        # interleaved issue on two unordered streams
        for k in (0, 1):
            plan.forward(xs[k], -1, outs_p[k], stream=streams[k])
        for k in (0, 1):
            plan.back(qs[k], -1, outs_b[k], stream=streams[k])
        for k in (0, 1):
            plan.forward(xs[k], 3, outs_s[k], stream=streams[k])
        torch.cuda.synchronize()
        for k in (0, 1):
            assert torch.equal(outs_p[k], ref_p[k]), ("forward", rep, k)
            assert torch.equal(outs_b[k], ref_b[k]), ("back", rep, k)
            assert torch.equal(outs_s[k], ref_s[k]), ("forward subset", rep, k)
    plan.check()
    plan.close()


def test_two_streams_osem_equal_serial_bitwise(spect_lib, cuda):
    plan, f = _plan(spect_lib, cuda)
    y = [plan.forward(f) + 0.5, plan.forward(f * 0.5) + 0.25]
    torch.cuda.synchronize()
    ref = []
    for k in (0, 1):
        x = torch.ones_like(f)
        plan.osem(y[k], 0.5, x, 0, 8)
        ref.append(x)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    xs = [torch.ones_like(f), torch.ones_like(f)]
    torch.cuda.synchronize()
    for t in range(8):  # alternate the subiterations of the two runs
        for k in (0, 1):
            plan.osem(y[k], 0.5, xs[k], t, 1, stream=streams[k])
    torch.cuda.synchronize()
    for k in (0, 1):
        assert torch.equal(xs[k], ref[k]), k
    plan.close()


def test_reserve_and_release_stream(spect_lib, cuda):
    plan, f = _plan(spect_lib, cuda, n=64, na=32, M=4)
    base = plan.info()["device_bytes"]
    s = torch.cuda.Stream()
    spect_lib.spect_plan_reserve_stream(plan.handle, s)
    grown = plan.info()["device_bytes"]
    assert grown > base
    spect_lib.spect_plan_reserve_stream(plan.handle, s)  # exists already: nothing more
    assert plan.info()["device_bytes"] == grown
    ref = plan.forward(f)
    out = torch.empty_like(ref)
    torch.cuda.synchronize()
    plan.forward(f, -1, out, stream=s)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    spect_lib.spect_plan_release_stream(plan.handle, s)
    assert plan.info()["device_bytes"] == base
    plan.forward(f, -1, out, stream=s)  # recreated on demand
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    plan.close()
