"""Continuous-batching server (include/spect_serve.h), on the GPU.

  - every request's image is bitwise the same alone, in a mix of requests of
    other sizes admitted together, and through the direct spect_osem_run path;
  - a 64^3 x 60-angle request served in a mix agrees with the FP64 oracle;
  - admission respects the HBM budget (peak bytes <= budget) and a request
    larger than the whole budget is refused; queued requests can be
    cancelled; a bounded wait reports SPECT_ETIMEDOUT;
  - BF16-PSF requests mix with FP32 ones and stay within 1e-4 of FP32 (the
    three-product BF16 form measures about 5e-6).
"""
import numpy as np
import pytest

from helpers import oracle_geom, phantom_inputs, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _request(spect, dev, n, na, seed, counts, bf16=False):
    from paper_2309_01977_gb300 import phantom
    geom = spect.Geometry(n=n, nz=n, n_angles=na, n_subsets=8, psf_bf16=bf16, atten_f64=bf16)
    f, mu = phantom_inputs(n, n, seed)
    plan = spect.Plan(spect.Geometry(n=n, nz=n, n_angles=na, n_subsets=8), torch.from_numpy(mu.astype(np.float32)).to(dev))
    hf = plan.forward(torch.from_numpy(f.astype(np.float32)).to(dev)).double().cpu().numpy()
    plan.close()
    _, y, s, _ = phantom.make_counts(f, hf, counts, 0.05, seed)
    return geom, mu.astype(np.float32), y.astype(np.float32), float(np.float32(s))


REQS = [(64, 60, 1001, 1e6, 2), (96, 96, 1002, 3e6, 3), (128, 120, 1003, 1e7, 2), (64, 60, 1004, 2e6, 4),
        (96, 96, 1005, 1e6, 2), (128, 120, 1006, 5e6, 3)]


def test_serve_alone_equals_mix_and_direct(spect_lib, cuda):
    data = [(_request(spect_lib, cuda, n, na, seed, c), it) for n, na, seed, c, it in REQS]
    budget = 6 << 30
    sv = spect_lib.Server(budget, max_slots=4, n_streams=4)
    alone = []
    for (geom, mu, y, s), it in data:
        x, _ = sv.wait(sv.submit(geom, mu, y, s, it))
        alone.append(x)
    ids = [sv.submit(geom, mu, y, s, it) for (geom, mu, y, s), it in data]
    mix = [sv.wait(i)[0] for i in ids]
    st = sv.stats()
    sv.close()
    for a, m in zip(alone, mix):
        assert np.array_equal(a, m)
        assert np.isfinite(a).all() and a.max() > 0
    assert st["completed"] == 2 * len(data)
    assert st["peak_active"] >= 2          # requests overlapped on the device
    assert st["peak_bytes"] <= budget
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # the server's graph-launched run equals the direct call bitwise
    (geom, mu, y, s), it = data[1]
    plan = spect_lib.Plan(geom, torch.from_numpy(mu).to(cuda))
    x = torch.ones((geom.n, geom.n, geom.nz), device=cuda)
    plan.osem(torch.from_numpy(y).to(cuda), s, x, 0, it * 8)
    assert np.array_equal(x.cpu().numpy(), alone[1])


def test_serve_oracle_parity_in_mix(spect_lib, oracle_mod, cuda):
    from paper_2309_01977_gb300 import phantom
    n, na = 64, 60
    f, mu = phantom_inputs(n, n, 2024)
    geom = spect_lib.Geometry(n=n, nz=n, n_angles=na, n_subsets=8)
    og = oracle_geom(oracle_mod, geom, mu)
    _, y, s, _ = phantom.make_counts(f, oracle_mod.forward(f, og), 1e6, 0.05, 2024)
    s = float(np.float32(s))
    ref, _ = oracle_mod.osem(y, s, og, 8, 0, 16)
    others = [_request(spect_lib, cuda, 96, 96, 77, 2e6), _request(spect_lib, cuda, 64, 60, 78, 1e6)]
    sv = spect_lib.Server(4 << 30, max_slots=3, n_streams=3)
    i0 = sv.submit(*others[0], 3)
    i1 = sv.submit(geom, mu.astype(np.float32), y.astype(np.float32), s, 2)
    i2 = sv.submit(*others[1], 4)
    x, lat = sv.wait(i1)
    sv.wait(i0)
    sv.wait(i2)
    sv.close()
    assert rel_l2(x, ref) <= 2e-5
    assert lat > 0


def test_serve_budget_cancel_timeout(spect_lib, cuda):
    big = _request(spect_lib, cuda, 128, 120, 31, 1e7)
    small = _request(spect_lib, cuda, 64, 60, 32, 1e6)
    budget = int(1.6 * (1 << 30))            # one 128^3 x 120-angle request at a time
    sv = spect_lib.Server(budget, max_slots=4, n_streams=4)
    with pytest.raises(spect_lib.SpectError) as e:
        g = spect_lib.Geometry(n=128, nz=128, n_angles=360, n_subsets=8)
        sv.submit(g, np.zeros((128, 128, 128), np.float32), np.zeros((360, 128, 128), np.float32), 0.1, 1)
    assert e.value.status == spect_lib.SPECT_EBUDGET
    a = sv.submit(*big, 6)
    b = sv.submit(*big, 2)
    c = sv.submit(*big, 2)
    try:
        sv.cancel(c)
        cancelled = True
    except spect_lib.SpectError as err:
        assert err.status == spect_lib.SPECT_ESTATE    # already admitted: the race is allowed
        cancelled = False
    try:
        sv.wait(a, timeout_ms=1)
    except spect_lib.SpectError as err:
        assert err.status == spect_lib.SPECT_ETIMEDOUT
    sv.wait(a)
    sv.wait(b)
    if cancelled:
        with pytest.raises(spect_lib.SpectError) as e:
            sv.wait(c)
        assert e.value.status == spect_lib.SPECT_ECANCELLED
    else:
        sv.wait(c)
    d = sv.submit(*small, 2)
    sv.wait(d)
    st = sv.stats()
    sv.close()
    assert st["peak_bytes"] <= budget
    assert st["rejected"] == 1


def test_serve_bf16_requests(spect_lib, cuda):
    r32 = _request(spect_lib, cuda, 64, 60, 41, 2e6)
    r16 = _request(spect_lib, cuda, 64, 60, 41, 2e6, bf16=True)
    other = _request(spect_lib, cuda, 128, 120, 42, 1e7, bf16=True)
    sv = spect_lib.Server(8 << 30, max_slots=4, n_streams=4)
    x16_alone, _ = sv.wait(sv.submit(*r16, 3))
    ids = [sv.submit(*other, 2), sv.submit(*r16, 3), sv.submit(*r32, 3)]
    xs = [sv.wait(i)[0] for i in ids]
    sv.close()
    assert np.array_equal(xs[1], x16_alone)
    assert rel_l2(xs[1], xs[2]) <= 1e-4
