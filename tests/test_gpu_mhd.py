"""MHD (Eqs. uMHD, bMHD) on the CUDA path against the FP64 oracle: the
right-hand side, IF-RK steps and the magnetic diagnostics."""

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


def _state(nx, ny, nz, seed, **box):
    u = inputs.random_solenoidal_field(nx, ny, nz, seed=seed, kmax=(nx, ny, nz), **box)
    b = inputs.random_solenoidal_field(nx, ny, nz, seed=seed + 50, kmax=(nx, ny, nz), **box) * 0.7
    return np.concatenate([u, b])


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 16, 32), (16, 64, 128), (96, 48, 32)])
def test_mhd_rhs_matches_oracle(ps, prec, shape):
    nx, ny, nz = shape
    box = dict(lx=2 * math.pi, ly=3.0, lz=5.0)
    ub = _state(nx, ny, nz, 7, **box)
    f = inputs.forcing_field(nx, ny, nz, seed=2, **box)
    cfg = oracle.Config(nx, ny, nz, nu=3e-3, eta=5e-3, **box)
    ref = oracle.mhd_rhs(ub, cfg, forcing=f)
    P, dt = _prec(ps, prec)
    plan = ps.Plan(nx, ny, nz, prec=P, eq=ps.Equations.MHD, nu=3e-3, eta=5e-3,
                   forcing=torch.from_numpy(f).to("cuda", dt), **box)
    assert plan.shape == (6, nz, ny, nx // 2 + 1)
    got = plan.rhs(torch.from_numpy(ub).to("cuda", dt)).cpu().numpy().astype(np.complex128)
    assert_parity(got, ref, TOL[prec], "mhd rhs")
    assert np.all(got[:, ~oracle.dealias_mask(cfg)] == 0)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [2, 4])
def test_mhd_rk_steps_match_oracle(ps, prec, order):
    n, dt = 32, 2e-3
    ub = _state(n, n, n, 9) * 2.0
    cfg = oracle.Config(n, n, n, nu=4e-3, eta=8e-3, rk_order=order)
    ref = ub
    for _ in range(3):
        ref = oracle.mhd_rk_step(ref, dt, cfg)
    P, dtype = _prec(ps, prec)
    plan = ps.Plan(n, prec=P, eq=ps.Equations.MHD, nu=4e-3, eta=8e-3, rk_order=order)
    d = torch.from_numpy(ub).to("cuda", dtype)
    for i in range(3):
        plan.rk_step(d, dt, t=i * dt)
    assert_parity(d.cpu().numpy().astype(np.complex128), ref, TOL[prec], "mhd step")
    plan.close()


def test_mhd_diagnostics_match_oracle(ps):
    n = 32
    ub = _state(n, n, n, 13)
    cfg = oracle.Config(n, n, n)
    ref = oracle.mhd_diagnostics(ub, cfg)
    plan = ps.Plan(n, prec=ps.Precision.FP64, eq=ps.Equations.MHD)
    d = plan.diagnostics(torch.from_numpy(ub).to("cuda"))
    for key in ("energy", "enstrophy", "magnetic_energy", "max_u"):
        assert abs(d[key] - ref[key]) < 1e-12 * abs(ref[key]), key
    for key in ("helicity", "cross_helicity", "magnetic_helicity"):
        assert abs(d[key] - ref[key]) < 1e-12 * (ref["energy"] + ref["enstrophy"]), key
    plan.close()


def test_mhd_energy_stat_is_total_energy(ps):
    n = 16
    ub = _state(n, n, n, 17)
    cfg = oracle.Config(n, n, n)
    d = oracle.mhd_diagnostics(ub, cfg)
    plan = ps.Plan(n, prec=ps.Precision.FP64, eq=ps.Equations.MHD, nu=1e-3, eta=1e-3)
    plan.rk_step(torch.from_numpy(ub).to("cuda"), 1e-3)
    e, _ = plan.step_stats()
    assert abs(e - (d["energy"] + d["magnetic_energy"])) < 1e-12
    plan.close()
