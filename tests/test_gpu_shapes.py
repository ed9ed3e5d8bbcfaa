"""Tile-shape variants of the column passes (ps_plan_set_pass_shape): fewer
kx columns per CTA, or the other radix schedule (8 <-> 16 points per thread),
compute the same right-hand side; each is checked against the FP64 oracle at
the FP32 tolerance, alone and mixed, on cubic and anisotropic grids."""

import functools

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


@functools.lru_cache(maxsize=None)
def _case(nx, ny, nz):
    u = inputs.random_solenoidal_field(nx, ny, nz, seed=11, kmax=(nx, ny, nz))
    f = inputs.forcing_field(nx, ny, nz, seed=2)
    ref = oracle.rhs(u, oracle.Config(nx, ny, nz, nu=2e-3), forcing=f)
    return u, f, ref


def _plan(ps, shape, f):
    nx, ny, nz = shape
    fd = torch.from_numpy(f).to("cuda", torch.complex64)
    return ps.Plan(nx, ny, nz, prec=ps.Precision.FP32, nu=2e-3, forcing=fd), fd


@pytest.mark.parametrize("n", [64, 96, 128])
@pytest.mark.parametrize("variant", [1, 2])
def test_variant_rhs_matches_oracle(ps, n, variant):
    u, f, ref = _case(n, n, n)
    plan, _fd = _plan(ps, (n, n, n), f)
    if variant == 2 and n == 96:
        for k in range(3):
            with pytest.raises(ps.PsError) as ei:
                plan.set_pass_shape(k, 2)
            assert ei.value.status == ps.PS_ERR_UNSUPPORTED
        plan.close()
        return
    base = [plan.set_pass_shape(k, 0) for k in range(3)]
    shapes = [plan.set_pass_shape(k, variant) for k in range(3)]
    for (c0, e0), (c1, e1) in zip(base, shapes):
        assert (c1, e1) == ((c0 // 2, e0) if variant == 1 else (c0, 8 if e0 == 16 else 16))
    got = plan.rhs(torch.from_numpy(u).to("cuda", torch.complex64)).cpu().numpy().astype(np.complex128)
    assert_parity(got, ref, 2e-6, f"shape variant {variant}")
    plan.close()


@pytest.mark.parametrize("shape", [(64, 128, 96), (128, 96, 64)])
def test_mixed_variants_anisotropic_rhs_and_step(ps, shape):
    u, f, ref = _case(*shape)
    plan, _fd = _plan(ps, shape, f)
    ud = torch.from_numpy(u).to("cuda", torch.complex64)
    step0 = ud.clone()
    plan.rk_step(step0, 1e-3)
    nx, ny, nz = shape
    plan.set_pass_shape(0, 2 if nz != 96 else 1)
    plan.set_pass_shape(1, 1)
    plan.set_pass_shape(2, 2 if nz != 96 else 1)
    got = plan.rhs(ud).cpu().numpy().astype(np.complex128)
    assert_parity(got, ref, 2e-6, "mixed shape variants")
    step1 = ud.clone()
    plan.rk_step(step1, 1e-3)
    torch.cuda.synchronize()
    d = (step1 - step0).abs().max().item() / step0.abs().max().item()
    assert d < 1e-6
    plan.close()


def test_variants_rejected_where_absent(ps):
    plan = ps.Plan(32, prec=ps.Precision.FP32, nu=1e-3)
    with pytest.raises(ps.PsError) as ei:
        plan.set_pass_shape(1, 1)
    assert ei.value.status == ps.PS_ERR_UNSUPPORTED
    assert plan.set_pass_shape(1, 0) == (8, 8)
    with pytest.raises(ps.PsError) as ei:
        plan.set_pass_shape(3, 0)
    assert ei.value.status == ps.PS_ERR_INVALID_ARG
    plan.close()
    plan = ps.Plan(64, prec=ps.Precision.FP64, nu=1e-3)
    with pytest.raises(ps.PsError):
        plan.set_pass_shape(0, 1)
    plan.close()
