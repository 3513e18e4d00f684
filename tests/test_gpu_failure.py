"""Failure detection on the GPU without a fault: every wait of the projector kernels on an asynchronous copy
is bounded and, when it runs out, the kernel records SPECT_ETIMEDOUT in the
plan's status word and returns.  spect_plan_selftest_timeout runs that path
with a short limit on a barrier that nothing arrives on; the host reads the
status with spect_plan_check, and the context stays usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(spect_lib, cuda):
    g = spect_lib.Geometry(n=32, nz=32, n_angles=8, n_subsets=2, attenuation=False)
    plan = spect_lib.Plan(g)
    x = torch.rand((32, 32, 32), device=cuda)
    p0 = plan.forward(x)
    spect_lib.spect_plan_check(plan.handle)  # nothing timed out yet
    # about 1 ms at the SM clock: the wait runs out and is reported
    spect_lib.spect_plan_selftest_timeout(plan.handle, 2_000_000)
    with pytest.raises(spect_lib.SpectError) as e:
        spect_lib.spect_plan_check(plan.handle)
    assert e.value.status == spect_lib.SPECT_ETIMEDOUT
    # the check cleared the status word; the plan and context still work
    spect_lib.spect_plan_check(plan.handle)
    assert torch.equal(plan.forward(x), p0)
    spect_lib.spect_plan_check(plan.handle)
    # out-of-range limits are rejected without a launch
    for bad in (0, -5, 4_000_000_001):
        with pytest.raises(spect_lib.SpectError) as e:
            spect_lib.spect_plan_selftest_timeout(plan.handle, bad)
        assert e.value.status == spect_lib.SPECT_EINVAL
    plan.close()
