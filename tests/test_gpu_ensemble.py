"""Ensembles of independent solves of uneven sizes (one CUDA graph vs
member-by-member launches), and the radix-3 grid lengths they need."""

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


SIZES = [32, 48, 64, 32, 48, 64, 96]


def _members(ps, prec="fp32"):
    P, dt = (ps.Precision.FP32, torch.complex64) if prec == "fp32" else (ps.Precision.FP64, torch.complex128)
    cfgs, states, host = [], [], []
    for i, n in enumerate(SIZES):
        nu = inputs.ensemble_viscosity(i)
        cfgs.append(ps.make_config(n, prec=P, nu=nu, rk_order=4))
        u = inputs.random_solenoidal_field(n, n, n, seed=1000 + i) * 2.0
        host.append(u)
        states.append(torch.from_numpy(u).to("cuda", dt))
    return cfgs, states, host


def test_graph_and_sequential_are_identical_and_match_single_plans(ps):
    cfgs, s_graph, host = _members(ps)
    s_seq = [s.clone() for s in s_graph]
    s_one = [s.clone() for s in s_graph]
    ens = ps.ps_ensemble_create(cfgs)
    ps.ps_ensemble_rk_steps(ens, s_graph, 2e-3, 0.0, 3, ps.ENS_GRAPH)
    ps.ps_ensemble_rk_steps(ens, s_seq, 2e-3, 0.0, 3, ps.ENS_SEQUENTIAL)
    torch.cuda.synchronize()
    for i, c in enumerate(cfgs):
        plan = ps.Plan(c.nx, prec=ps.Precision.FP32, nu=c.nu, rk_order=4)
        for k in range(3):
            plan.rk_step(s_one[i], 2e-3, t=k * 2e-3)
        torch.cuda.synchronize()
        assert torch.equal(s_graph[i], s_seq[i])
        assert torch.equal(s_graph[i], s_one[i])
        plan.close()
    # replaying the captured graph continues the same trajectory
    ps.ps_ensemble_rk_steps(ens, s_graph, 2e-3, 0.0, 3, ps.ENS_GRAPH)
    ps.ps_ensemble_rk_steps(ens, s_seq, 2e-3, 0.0, 3, ps.ENS_SEQUENTIAL)
    torch.cuda.synchronize()
    for a, b in zip(s_graph, s_seq):
        assert torch.equal(a, b)
    ps.ps_ensemble_destroy(ens)


@pytest.mark.parametrize("member", [1, 6])
def test_ensemble_member_matches_oracle(ps, member):
    cfgs, states, host = _members(ps, "fp64")
    ens = ps.ps_ensemble_create(cfgs)
    ps.ps_ensemble_rk_steps(ens, states, 2e-3, 0.0, 2, ps.ENS_GRAPH)
    torch.cuda.synchronize()
    n = SIZES[member]
    ref = host[member]
    cfg = oracle.Config(n, n, n, nu=cfgs[member].nu, rk_order=4)
    for _ in range(2):
        ref = oracle.rk_step(ref, 2e-3, cfg)
    got = states[member].cpu().numpy()
    assert_parity(got, ref, 1e-12, "ensemble member")
    ps.ps_ensemble_destroy(ens)


def test_tuner_keeps_states_and_results(ps):
    cfgs, states, _ = _members(ps)
    before = [s.clone() for s in states]
    ens = ps.ps_ensemble_create(cfgs)
    tuning = ps.ps_ensemble_tune(ens, states, 2e-3)
    torch.cuda.synchronize()
    for a, b in zip(states, before):
        assert torch.equal(a, b)
    assert 1 <= tuning["branches"] <= len(SIZES) and tuning["step_ms"] > 0
    assert set(tuning["xrpc"]) == {32, 48, 64, 96}
    assert set(tuning["pass_shapes"]) == {32, 48, 64, 96}
    for n, passes in tuning["pass_shapes"].items():
        for cols, pts in passes.values():
            assert cols in (4, 8) and pts in (8, 12, 16)
    ref = [s.clone() for s in states]
    ps.ps_ensemble_rk_steps(ens, states, 2e-3, 0.0, 2, ps.ENS_GRAPH)
    ps.ps_ensemble_rk_steps(ens, ref, 2e-3, 0.0, 2, ps.ENS_SEQUENTIAL)
    torch.cuda.synchronize()
    for a, b in zip(states, ref):
        assert torch.equal(a, b)
    ps.ps_ensemble_destroy(ens)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(96, 96, 96), (48, 192, 96), (192, 48, 64)])
def test_radix3_lengths_rhs_matches_oracle(ps, prec, shape):
    nx, ny, nz = shape
    u = inputs.random_solenoidal_field(nx, ny, nz, seed=3, kmax=(nx, ny, nz), ly=4.0)
    f = inputs.forcing_field(nx, ny, nz, seed=2, ly=4.0)
    cfg = oracle.Config(nx, ny, nz, ly=4.0, nu=2e-3)
    ref = oracle.rhs(u, cfg, forcing=f)
    P, dt = (ps.Precision.FP32, torch.complex64) if prec == "fp32" else (ps.Precision.FP64, torch.complex128)
    plan = ps.Plan(nx, ny, nz, ly=4.0, prec=P, nu=2e-3, forcing=torch.from_numpy(f).to("cuda", dt))
    got = plan.rhs(torch.from_numpy(u).to("cuda", dt)).cpu().numpy().astype(np.complex128)
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert_parity(got, ref, tol, "ensemble member")
    plan.close()


# ---- persistent launch: one kernel over a device queue of (member, pass, tile)

def test_persistent_matches_graph_bitwise_and_replays(ps):
    cfgs, s_per, _ = _members(ps)
    s_graph = [s.clone() for s in s_per]
    ens = ps.ps_ensemble_create(cfgs)
    ps.ps_ensemble_rk_steps(ens, s_per, 2e-3, 0.0, 3, ps.ENS_PERSISTENT)
    ps.ps_ensemble_rk_steps(ens, s_graph, 2e-3, 0.0, 3, ps.ENS_GRAPH)
    ps.ps_ensemble_check(ens)
    torch.cuda.synchronize()
    for a, b in zip(s_per, s_graph):
        assert torch.equal(a, b)
    # the captured persistent graph replays the next steps of the same trajectory
    ps.ps_ensemble_rk_steps(ens, s_per, 2e-3, 0.0, 3, ps.ENS_PERSISTENT)
    ps.ps_ensemble_rk_steps(ens, s_graph, 2e-3, 0.0, 3, ps.ENS_GRAPH)
    ps.ps_ensemble_check(ens)
    torch.cuda.synchronize()
    for a, b in zip(s_per, s_graph):
        assert torch.equal(a, b)
    ps.ps_ensemble_destroy(ens)


@pytest.mark.parametrize("member", [0, 6])
def test_persistent_member_matches_oracle_fp64(ps, member):
    cfgs, states, host = _members(ps, "fp64")
    ens = ps.ps_ensemble_create(cfgs)
    ps.ps_ensemble_rk_steps(ens, states, 2e-3, 0.0, 2, ps.ENS_PERSISTENT)
    ps.ps_ensemble_check(ens)
    torch.cuda.synchronize()
    n = SIZES[member]
    ref = host[member]
    cfg = oracle.Config(n, n, n, nu=cfgs[member].nu, rk_order=4)
    for _ in range(2):
        ref = oracle.rk_step(ref, 2e-3, cfg)
    assert_parity(states[member].cpu().numpy(), ref, 1e-12, "persistent ensemble member")
    ps.ps_ensemble_destroy(ens)


def test_persistent_fp32_rk2_forced_anisotropic_matches_oracle(ps):
    shapes = [(64, 32, 48), (32, 96, 64), (128, 64, 32)]
    cfgs, states, refs, keep = [], [], [], []
    for i, (nx, ny, nz) in enumerate(shapes):
        u = inputs.random_solenoidal_field(nx, ny, nz, seed=70 + i, kmax=(nx, ny, nz))
        f = inputs.forcing_field(nx, ny, nz, seed=2)
        fd = torch.from_numpy(f).to("cuda", torch.complex64)
        cfgs.append(ps.make_config(nx, ny, nz, prec=ps.Precision.FP32, nu=3e-3, rk_order=2, forcing=fd))
        states.append(torch.from_numpy(u).to("cuda", torch.complex64))
        cfg = oracle.Config(nx, ny, nz, nu=3e-3, rk_order=2)
        ref = u
        for _ in range(2):
            ref = oracle.rk_step(ref, 2e-3, cfg, forcing=f)
        refs.append(ref)
        keep.append(fd)
    ens = ps.ps_ensemble_create(cfgs)
    ps.ps_ensemble_rk_steps(ens, states, 2e-3, 0.0, 2, ps.ENS_PERSISTENT)
    ps.ps_ensemble_check(ens)
    torch.cuda.synchronize()
    for s, ref in zip(states, refs):
        assert_parity(s.cpu().numpy().astype(np.complex128), ref, 2e-6, "persistent ensemble member")
    ps.ps_ensemble_destroy(ens)


def test_persistent_bounded_wait_reports_timeout_then_recovers(ps):
    cfgs, states, _ = _members(ps)
    start = [s.clone() for s in states]
    ref = [s.clone() for s in states]
    ens = ps.ps_ensemble_create(cfgs)
    ps.ps_ensemble_set_wait_test(ens, 1 << 12)
    ps.ps_ensemble_rk_steps(ens, states, 2e-3, 0.0, 1, ps.ENS_PERSISTENT)
    with pytest.raises(ps.PsError) as ei:
        ps.ps_ensemble_check(ens)
    assert ei.value.status == ps.PS_ERR_TIMEOUT
    ps.ps_ensemble_check(ens)  # reported once
    ps.ps_ensemble_set_wait_test(ens, 0)
    for s, s0 in zip(states, start):
        s.copy_(s0)
    ps.ps_ensemble_rk_steps(ens, states, 2e-3, 0.0, 1, ps.ENS_PERSISTENT)
    ps.ps_ensemble_rk_steps(ens, ref, 2e-3, 0.0, 1, ps.ENS_SEQUENTIAL)
    ps.ps_ensemble_check(ens)
    torch.cuda.synchronize()
    for a, b in zip(states, ref):
        assert torch.equal(a, b)
    ps.ps_ensemble_destroy(ens)


def test_persistent_rejects_unsupported_members(ps):
    cfgs = [ps.make_config(32, prec=ps.Precision.FP32, nu=1e-3),
            ps.make_config(256, 32, 32, prec=ps.Precision.FP32, nu=1e-3)]
    states = [torch.zeros(3, 32, 32, 17, dtype=torch.complex64, device="cuda"),
              torch.zeros(3, 32, 32, 129, dtype=torch.complex64, device="cuda")]
    ens = ps.ps_ensemble_create(cfgs)
    for mode in (ps.ENS_PERSISTENT, ps.ENS_BATCHED):
        with pytest.raises(ps.PsError) as ei:
            ps.ps_ensemble_rk_steps(ens, states, 1e-3, 0.0, 1, mode)
        assert ei.value.status == ps.PS_ERR_UNSUPPORTED
    ps.ps_ensemble_rk_steps(ens, states, 1e-3, 0.0, 1, ps.ENS_GRAPH)  # the other modes still run
    ps.ps_ensemble_destroy(ens)


def test_tuner_times_persistent_knobs_and_auto_mode_runs_the_faster(ps):
    cfgs, states, _ = _members(ps)
    ens = ps.ps_ensemble_create(cfgs)
    tuning = ps.ps_ensemble_tune(ens, states, 2e-3)
    assert tuning["persistent_step_ms"] > 0 and tuning["batched_step_ms"] > 0
    assert tuning["batched_members_per_launch"] in (2, 4, 8, 16, 32)
    assert tuning["best_mode"] in ("graph", "persistent", "batched")
    assert tuning["persistent_ctas_per_sm"] in (0, 1) and tuning["persistent_order"] in (0, 1)
    assert all(v >= 1 for v in tuning["persistent_tiles_per_item"].values())
    ref = [s.clone() for s in states]
    ps.ps_ensemble_rk_steps(ens, states, 2e-3, 0.0, 2, ps.ENS_AUTO)
    ps.ps_ensemble_rk_steps(ens, ref, 2e-3, 0.0, 2, ps.ENS_SEQUENTIAL)
    ps.ps_ensemble_check(ens)
    torch.cuda.synchronize()
    for a, b in zip(states, ref):
        assert torch.equal(a, b)
    ps.ps_ensemble_destroy(ens)


# ---- batched launches: one launch per pass for all members of a grid class

def test_batched_matches_graph_bitwise_and_replays(ps):
    cfgs, s_bat, _ = _members(ps)
    s_graph = [s.clone() for s in s_bat]
    ens = ps.ps_ensemble_create(cfgs)
    for _ in range(2):  # capture, then replay of the same graph
        ps.ps_ensemble_rk_steps(ens, s_bat, 2e-3, 0.0, 3, ps.ENS_BATCHED)
        ps.ps_ensemble_rk_steps(ens, s_graph, 2e-3, 0.0, 3, ps.ENS_GRAPH)
        torch.cuda.synchronize()
        for a, b in zip(s_bat, s_graph):
            assert torch.equal(a, b)
    ps.ps_ensemble_destroy(ens)


@pytest.mark.parametrize("member", [2, 6])
def test_batched_member_matches_oracle_fp64(ps, member):
    cfgs, states, host = _members(ps, "fp64")
    ens = ps.ps_ensemble_create(cfgs)
    ps.ps_ensemble_rk_steps(ens, states, 2e-3, 0.0, 2, ps.ENS_BATCHED)
    torch.cuda.synchronize()
    n = SIZES[member]
    ref = host[member]
    cfg = oracle.Config(n, n, n, nu=cfgs[member].nu, rk_order=4)
    for _ in range(2):
        ref = oracle.rk_step(ref, 2e-3, cfg)
    assert_parity(states[member].cpu().numpy(), ref, 1e-12, "batched ensemble member")
    ps.ps_ensemble_destroy(ens)


def test_batched_forced_rk2_classes_match_single_plans(ps):
    shapes = [(64, 32, 48), (64, 32, 48), (32, 96, 64), (64, 32, 48)]
    cfgs, states, keep = [], [], []
    for i, (nx, ny, nz) in enumerate(shapes):
        u = inputs.random_solenoidal_field(nx, ny, nz, seed=80 + i, kmax=(nx, ny, nz))
        f = inputs.forcing_field(nx, ny, nz, seed=3 + i)
        fd = torch.from_numpy(f).to("cuda", torch.complex64)
        keep.append(fd)
        cfgs.append(ps.make_config(nx, ny, nz, prec=ps.Precision.FP32, nu=1e-3 * (i + 1), rk_order=2, forcing=fd))
        states.append(torch.from_numpy(u).to("cuda", torch.complex64))
    single = [s.clone() for s in states]
    ens = ps.ps_ensemble_create(cfgs)
    ps.ps_ensemble_rk_steps(ens, states, 2e-3, 0.0, 2, ps.ENS_BATCHED)
    for i, c in enumerate(cfgs):
        plan = ps.Plan(c.nx, c.ny, c.nz, prec=ps.Precision.FP32, nu=c.nu, rk_order=2, forcing=keep[i])
        for k in range(2):
            plan.rk_step(single[i], 2e-3, t=k * 2e-3)
        torch.cuda.synchronize()
        assert torch.equal(states[i], single[i])
        plan.close()
    ps.ps_ensemble_destroy(ens)
