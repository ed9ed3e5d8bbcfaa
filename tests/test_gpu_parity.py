"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over the whole field): FP64 1e-12 per RHS / step,
FP32 2e-6 per RHS / step."""

import math

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs

from .parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6}


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


def _prec(ps, name):
    return (ps.Precision.FP64, torch.complex128) if name == "fp64" else (ps.Precision.FP32, torch.complex64)


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def to_np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


DEALIAS = {"cubic": oracle.spectral.CUBIC, "spherical": oracle.spectral.SPHERICAL, "none": oracle.spectral.NONE}

RHS_CASES = [
    # (nx, ny, nz, lx, ly, lz, dealias, forcing)
    (16, 16, 16, 2 * math.pi, 2 * math.pi, 2 * math.pi, "cubic", True),
    (32, 32, 32, 2 * math.pi, 2 * math.pi, 2 * math.pi, "cubic", True),
    (64, 64, 64, 2 * math.pi, 2 * math.pi, 2 * math.pi, "cubic", False),
    (128, 128, 128, 2 * math.pi, 2 * math.pi, 2 * math.pi, "cubic", True),
    (32, 64, 16, 3.0, 7.0, 2 * math.pi, "cubic", True),
    (8, 32, 128, 2 * math.pi, 1.5, 4.0, "cubic", False),
    (64, 16, 32, 2 * math.pi, 2 * math.pi, 9.0, "spherical", True),
    (32, 32, 32, 2 * math.pi, 2 * math.pi, 2 * math.pi, "none", True),
    (256, 32, 16, 2 * math.pi, 2 * math.pi, 2 * math.pi, "cubic", False),
    (16, 256, 512, 2 * math.pi, 2 * math.pi, 2 * math.pi, "cubic", False),
    (1024, 8, 16, 2 * math.pi, 2 * math.pi, 2 * math.pi, "cubic", False),
    (16, 1024, 8, 2 * math.pi, 2 * math.pi, 2 * math.pi, "cubic", False),
    (8, 16, 1024, 2 * math.pi, 2 * math.pi, 2 * math.pi, "cubic", False),
]


def _fields(nx, ny, nz, lx, ly, lz, forcing, seed=1):
    # kmax beyond the mask: modes outside the retained set must be ignored
    u = inputs.random_solenoidal_field(nx, ny, nz, seed=seed, kmax=(nx, ny, nz), lx=lx, ly=ly, lz=lz)
    f = inputs.forcing_field(nx, ny, nz, seed=2, kmax=(nx, ny, nz), lx=lx, ly=ly, lz=lz) if forcing else None
    return u, f


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", RHS_CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}-{c[6]}{'-f' if c[7] else ''}")
def test_rhs_matches_oracle(ps, prec, case):
    nx, ny, nz, lx, ly, lz, dealias, forcing = case
    nu = 3e-3
    u, f = _fields(nx, ny, nz, lx, ly, lz, forcing)
    cfg = oracle.Config(nx, ny, nz, lx=lx, ly=ly, lz=lz, nu=nu, dealias=DEALIAS[dealias])
    ref = oracle.rhs(u, cfg, forcing=f)
    P, dt = _prec(ps, prec)
    fd = to_dev(f, dt) if forcing else None
    plan = ps.Plan(nx, ny, nz, lx=lx, ly=ly, lz=lz, prec=P, nu=nu,
                   dealias=getattr(ps.Dealias, dealias.upper()), forcing=fd)
    ud = to_dev(u, dt)
    before = ud.clone()
    out = plan.rhs(ud)
    got = to_np(out)
    assert_parity(got, ref, TOL[prec], "rhs")
    # masked modes are exactly zero, the input is untouched
    mask = oracle.dealias_mask(cfg)
    assert np.all(got[:, ~mask] == 0)
    assert torch.equal(ud, before)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("n3", [(32, 32, 32), (16, 64, 32)])
def test_rk_step_matches_oracle(ps, prec, order, n3):
    nx, ny, nz = n3
    nu, dt = 5e-3, 2e-3
    u, f = _fields(nx, ny, nz, 2 * math.pi, 2 * math.pi, 2 * math.pi, True, seed=3)
    u = u * 3.0
    cfg = oracle.Config(nx, ny, nz, nu=nu, rk_order=order)
    ref = u
    for i in range(3):
        ref = oracle.rk_step(ref, dt, cfg, forcing=f)
    P, dtype = _prec(ps, prec)
    plan = ps.Plan(nx, ny, nz, prec=P, nu=nu, rk_order=order, forcing=to_dev(f, dtype))
    ud = to_dev(u, dtype)
    for i in range(3):
        plan.rk_step(ud, dt, t=i * dt)
    got = to_np(ud)
    assert_parity(got, ref, TOL[prec], "rk step")
    # stats of the state at the start of the last step
    prev = u
    for i in range(2):
        prev = oracle.rk_step(prev, dt, cfg, forcing=f)
    e, umax = plan.step_stats()
    d = oracle.diagnostics(prev, cfg)
    assert abs(e - d["energy"]) < 10 * TOL[prec] * d["energy"]
    assert abs(umax - d["max_u"]) < 10 * TOL[prec] * d["max_u"]
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", [(32, 32, 32, "cubic"), (64, 32, 16, "spherical"), (16, 16, 16, "none")])
def test_diagnostics_match_oracle(ps, prec, case):
    nx, ny, nz, dealias = case
    lx, ly, lz = 2 * math.pi, 5.0, 2 * math.pi
    u, _ = _fields(nx, ny, nz, lx, ly, lz, False, seed=5)
    cfg = oracle.Config(nx, ny, nz, lx=lx, ly=ly, lz=lz, dealias=DEALIAS[dealias])
    ref = oracle.diagnostics(u, cfg, cfl=0.4)
    P, dtype = _prec(ps, prec)
    plan = ps.Plan(nx, ny, nz, lx=lx, ly=ly, lz=lz, prec=P, dealias=getattr(ps.Dealias, dealias.upper()))
    d = plan.diagnostics(to_dev(u, dtype), cfl=0.4)
    tol = 1e-12 if prec == "fp64" else 2e-6
    for key in ("energy", "enstrophy", "max_u", "cfl_dt"):
        assert abs(d[key] - ref[key]) <= tol * abs(ref[key]), key
    assert abs(d["helicity"] - ref["helicity"]) <= tol * ref["enstrophy"]
    # the input rounded to FP32 is only divergence-free to FP32 rounding
    div_tol = 1e-10 if prec == "fp64" else 1e-5
    assert d["max_div"] <= div_tol * math.sqrt(ref["enstrophy"])
    spec = np.array(d["spectrum"])
    n = len(ref["spectrum"])
    assert np.allclose(spec[:n], ref["spectrum"], rtol=tol, atol=tol * ref["energy"])
    assert np.all(spec[n:] == 0)
    plan.close()


def test_taylor_green_config(ps):
    """32^3 FP64, nu = 1e-2, dt = 1e-3, RK2, 10 steps (the Taylor-Green case)."""
    n, nu, dt = 32, 1e-2, 1e-3
    u = inputs.taylor_green(n, n, n)
    cfg = oracle.Config(n, n, n, nu=nu, rk_order=2)
    ref = u
    for _ in range(10):
        ref = oracle.rk_step(ref, dt, cfg)
    plan = ps.Plan(n, prec=ps.Precision.FP64, nu=nu, rk_order=2)
    ud = to_dev(u, torch.complex128)
    for i in range(10):
        plan.rk_step(ud, dt, t=i * dt)
    got = to_np(ud)
    assert_parity(got, ref, 1e-12, "taylor-green steps")
    d = plan.diagnostics(ud)
    assert abs(d["energy"] - oracle.diagnostics(ref, cfg)["energy"]) < 1e-14
    plan.close()
