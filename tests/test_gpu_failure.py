"""Failure detection of the bounded device waits, exercised without a fault.

The x pass stages its rows with TMA copies that complete on an mbarrier, and
every wait on that barrier gives up after a limit of polls instead of
hanging.  The plan's test hook (ps_plan_set_wait_test) makes every CTA wait
for a copy that is never issued, with a short limit, so the give-up path
runs for real: the pass records the timeout in the device error word, the
right-hand side comes out as NaN instead of a wrong value, the next
synchronising call returns PS_ERR_TIMEOUT once, and the same plan then
computes correct results again (checked against the oracle)."""

import math

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs

from .parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_wait_that_gives_up_is_reported_and_the_plan_recovers(ps, prec):
    n, nu = 32, 2e-3
    P, dtype, tol = ((ps.Precision.FP32, torch.complex64, 2e-6) if prec == "fp32"
                     else (ps.Precision.FP64, torch.complex128, 1e-12))
    uh = inputs.random_solenoidal_field(n, n, n, seed=3)
    u = torch.from_numpy(uh).to("cuda", dtype)
    plan = ps.Plan(n, prec=P, nu=nu)
    ps.ps_plan_set_wait_test(plan.handle, 4096)
    out = plan.rhs(u)
    torch.cuda.synchronize()
    mask = oracle.dealias_mask(oracle.Config(n, n, n))
    got = out.cpu().numpy()
    assert np.all(np.isnan(got[:, mask]))          # no wrong value escapes
    with pytest.raises(ps.PsError) as e:
        ps.ps_step_stats(plan.handle)              # the next synchronising call
    assert e.value.status == ps.PS_ERR_TIMEOUT
    ps.ps_step_stats(plan.handle)                  # reported once: the word is clear

    # an RK step under the hook: the state turns NaN and the timeout is reported
    ps.ps_plan_set_wait_test(plan.handle, 4096)
    v = u.clone()
    plan.rk_step(v, 1e-3)
    with pytest.raises(ps.PsError) as e:
        plan.diagnostics(u)
    assert e.value.status == ps.PS_ERR_TIMEOUT
    assert torch.isnan(torch.view_as_real(v)).any()

    # hook off: the same plan is correct again
    ps.ps_plan_set_wait_test(plan.handle, 0)
    good = plan.rhs(u).cpu().numpy().astype(np.complex128)
    assert_parity(good, oracle.rhs(uh, oracle.Config(n, n, n, nu=nu)), tol, "rhs after recovery")
    ps.ps_step_stats(plan.handle)
    plan.close()


def test_wait_test_hook_rejects_bad_limits(ps):
    plan = ps.Plan(16, prec=ps.Precision.FP32)
    for bad in (-1, 1 << 21):
        with pytest.raises(ps.PsError) as e:
            ps.ps_plan_set_wait_test(plan.handle, bad)
        assert e.value.status == ps.PS_ERR_INVALID_ARG
    plan.close()
    assert math.isfinite(1.0)
