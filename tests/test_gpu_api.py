"""The rest of the C ABI on the GPU: host-buffer stepping, step statistics,
per-kernel timing, launch counting, error reporting and plan reuse."""

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


def test_host_buffer_steps_equal_device_steps(ps):
    n, dt = 32, 2e-3
    u = inputs.random_solenoidal_field(n, n, n, seed=4)
    f = torch.from_numpy(inputs.forcing_field(n, n, n, seed=2)).to("cuda", torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=5e-3, forcing=f)
    dev = torch.from_numpy(u).to("cuda", torch.complex64)
    for i in range(3):
        plan.rk_step(dev, dt, t=i * dt)
    host = torch.from_numpy(u.astype(np.complex64)).pin_memory()
    ps.ps_rk_step_host(plan.handle, host, dt, 0.0, 3)
    assert torch.equal(host, dev.cpu())
    # pageable memory under the default mode takes the copy-engine path
    pageable = torch.from_numpy(u.astype(np.complex64))
    ps.ps_rk_step_host(plan.handle, pageable, dt, 0.0, 3)
    assert torch.equal(pageable, host)
    plan.close()


@pytest.mark.parametrize("mode", ["auto", "copy", "mapped", "smcopy", "cube_ce"])
def test_host_state_modes_match_device_steps(ps, mode):
    """Host-buffer stepping copies the state or lets the kernels access the
    page-locked buffer in place; both give the device result bit for bit."""
    n, dt = 32, 2e-3
    # content outside the retained modes: every mode must write its zeros
    u = 2.0 * inputs.random_solenoidal_field(n, n, n, seed=6, kmax=(n, n, n))
    f = torch.from_numpy(inputs.forcing_field(n, n, n, seed=2)).to("cuda", torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=3e-3, forcing=f)
    dev = torch.from_numpy(u.astype(np.complex64)).cuda()
    for i in range(2):
        plan.rk_step(dev, dt, t=i * dt)
    mask = oracle.dealias_mask(oracle.Config(n, n, n))
    assert np.all(dev.cpu().numpy()[:, ~mask] == 0)
    ps.ps_plan_set_host_mode(plan.handle, {"auto": ps.HOST_AUTO, "copy": ps.HOST_COPY,
                                           "mapped": ps.HOST_MAPPED, "smcopy": ps.HOST_SMCOPY,
                                           "cube_ce": ps.HOST_CUBE_CE}[mode])
    host = torch.from_numpy(u.astype(np.complex64)).pin_memory()
    for i in range(2):
        ps.ps_rk_step_host(plan.handle, host, dt, i * dt, 1)
    assert torch.equal(host, dev.cpu())
    # several steps per call, and an MHD/FP64 plan (6 components, 16-byte modes)
    host2 = torch.from_numpy(u.astype(np.complex64)).pin_memory()
    ps.ps_rk_step_host(plan.handle, host2, dt, 0.0, 2)
    assert torch.equal(host2, dev.cpu())
    ub = np.concatenate([u, 0.5 * inputs.random_solenoidal_field(n, n, n, seed=7, kmax=(n, n, n))])
    pm = ps.Plan(n, prec=ps.Precision.FP64, eq=ps.Equations.MHD, nu=3e-3, eta=2e-3)
    dm = torch.from_numpy(ub).cuda()
    pm.rk_step(dm, dt)
    ps.ps_plan_set_host_mode(pm.handle, {"auto": ps.HOST_AUTO, "copy": ps.HOST_COPY,
                                         "mapped": ps.HOST_MAPPED, "smcopy": ps.HOST_SMCOPY,
                                           "cube_ce": ps.HOST_CUBE_CE}[mode])
    hm = torch.from_numpy(ub).pin_memory()
    ps.ps_rk_step_host(pm.handle, hm, dt, 0.0, 1)
    assert torch.equal(hm, dm.cpu())
    pm.close()
    if mode in ("mapped", "smcopy"):
        pageable = torch.from_numpy(u.astype(np.complex64))
        with pytest.raises(ps.PsError):
            ps.ps_rk_step_host(plan.handle, pageable, dt, 0.0, 1)
    with pytest.raises(ps.PsError):
        ps.ps_plan_set_host_mode(plan.handle, 9)
    plan.close()


def test_graph_replayed_steps_equal_single_steps(ps):
    """ps_rk_steps captures the steps once per (state, dt, nsteps) and replays
    them; results equal ps_rk_step calls bit for bit (HD with forcing, MHD)."""
    n, dt = 32, 2e-3
    u = inputs.random_solenoidal_field(n, n, n, seed=8)
    f = torch.from_numpy(inputs.forcing_field(n, n, n, seed=2)).to("cuda", torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=4e-3, forcing=f)
    a = torch.from_numpy(u.astype(np.complex64)).cuda()
    b = a.clone()
    for i in range(6):
        plan.rk_step(a, dt, t=i * dt)
    l0 = ps.ps_plan_launch_count(plan.handle)
    plan.rk_steps(b, dt, 3, t=0.0)
    plan.rk_steps(b, dt, 3, t=3 * dt)  # replay of the same graph
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert ps.ps_plan_launch_count(plan.handle) - l0 >= 2 * 3 * 25
    # a different step size re-captures
    plan.rk_step(a, 1e-3)
    plan.rk_steps(b, 1e-3, 1)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    plan.close()
    ub = np.concatenate([u, 0.3 * inputs.random_solenoidal_field(n, n, n, seed=9)])
    pm = ps.Plan(n, prec=ps.Precision.FP64, eq=ps.Equations.MHD, nu=3e-3, eta=2e-3)
    a = torch.from_numpy(ub).cuda()
    b = a.clone()
    for i in range(2):
        pm.rk_step(a, dt)
    pm.rk_steps(b, dt, 2)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    pm.close()


def test_timing_and_launch_counts(ps):
    n = 32
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=1e-3)
    u = torch.from_numpy(inputs.random_solenoidal_field(n, n, n, seed=5)).to("cuda", torch.complex64)
    plan.rk_step(u, 1e-3)
    l0 = ps.ps_plan_launch_count(plan.handle)
    ps.ps_plan_set_timing(plan.handle, True)
    for _ in range(2):
        plan.rk_step(u, 1e-3)
    t = ps.ps_plan_get_timing(plan.handle)
    ps.ps_plan_set_timing(plan.handle, False)
    launched = ps.ps_plan_launch_count(plan.handle) - l0
    # per RK4 step: 4 x (5 passes + update) + energy reduction; dt unchanged -> no table launch
    assert launched == 2 * 25
    for kind in ("z_inverse", "y_inverse", "x_fused", "y_forward", "z_forward", "update"):
        ms, count = t[kind]
        assert count == 8 and ms > 0
    assert sum(c for _, c in t.values()) == launched
    plan.close()


def test_rhs_rejects_aliasing_and_reports_message(ps):
    n = 16
    plan = ps.Plan(n, prec=ps.Precision.FP64)
    u = torch.zeros(plan.shape, dtype=torch.complex128, device="cuda")
    with pytest.raises(ps.PsError) as e:
        ps.ps_rhs(plan.handle, u, u)
    assert e.value.status == ps.PS_ERR_INVALID_ARG and "overlaps" in str(e.value)
    # the plan stays usable after an invalid-argument error
    out = plan.rhs(u)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
    with pytest.raises(ps.PsError):
        ps.ps_rk_step(plan.handle, u, float("nan"))
    plan.close()


def test_plans_are_independent_and_reusable(ps):
    n = 16
    u = inputs.random_solenoidal_field(n, n, n, seed=6)
    cfg = oracle.Config(n, n, n, nu=1e-2)
    ref = oracle.rhs(u, cfg)
    plans = [ps.Plan(n, prec=ps.Precision.FP64, nu=1e-2) for _ in range(3)]
    ud = torch.from_numpy(u).to("cuda")
    for p in plans:
        for _ in range(2):
            got = p.rhs(ud).cpu().numpy()
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    for p in plans:
        p.close()


def test_diagnostics_of_zero_field(ps):
    plan = ps.Plan(16, prec=ps.Precision.FP32)
    d = plan.diagnostics(torch.zeros(plan.shape, dtype=torch.complex64, device="cuda"))
    assert d["energy"] == 0 and d["max_u"] == 0 and d["cfl_dt"] == float("inf")
    plan.close()


def test_nonfinite_state_is_reported(ps):
    plan = ps.Plan(16, prec=ps.Precision.FP32)
    u = torch.zeros(plan.shape, dtype=torch.complex64, device="cuda")
    u[0, 1, 1, 1] = complex(float("nan"), 0.0)
    d = plan.diagnostics(u)
    assert d["status"] == ps.PS_ERR_NONFINITE
    plan.close()
