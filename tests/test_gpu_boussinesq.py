"""Boussinesq system (Eqs. mom, temp, divv) on the CUDA path against the FP64
oracle: the right-hand side, IF-RK steps, diagnostics, and an internal
gravity wave against its exact solution."""

import math

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs

from .parity import BAND_M, assert_device_parity, assert_parity, embed_on_device

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


def _state(nx, ny, nz, seed, full=True, **box):
    kmax = (nx, ny, nz) if full else None  # full: content outside the mask too
    u = inputs.random_solenoidal_field(nx, ny, nz, seed=seed, kmax=kmax, **box)
    th = inputs.random_scalar_field(nx, ny, nz, seed=seed + 60, kmax=kmax, **box) * 0.8
    return np.concatenate([u, th])


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 16, 32), (16, 64, 128), (96, 48, 32), (128, 128, 128)])
def test_boussinesq_rhs_matches_oracle(ps, prec, shape):
    nx, ny, nz = shape
    box = dict(lx=2 * math.pi, ly=3.0, lz=5.0)
    st = _state(nx, ny, nz, 7, **box)
    f = inputs.forcing_field(nx, ny, nz, seed=2, **box)
    kw = dict(nu=3e-3, kappa=5e-3, n_bv=1.7)
    cfg = oracle.Config(nx, ny, nz, **kw, **box)
    ref = oracle.boussinesq_rhs(st, cfg, forcing=f)
    P, dt = _prec(ps, prec)
    plan = ps.Plan(nx, ny, nz, prec=P, eq=ps.Equations.BOUSSINESQ, forcing=torch.from_numpy(f).to("cuda", dt),
                   **kw, **box)
    assert plan.shape == (4, nz, ny, nx // 2 + 1)
    got = plan.rhs(torch.from_numpy(st).to("cuda", dt)).cpu().numpy().astype(np.complex128)
    assert_parity(got, ref, TOL[prec], "boussinesq rhs")
    assert relerr(got[3], ref[3]) < TOL[prec]  # the scalar alone
    assert np.all(got[:, ~oracle.dealias_mask(cfg)] == 0)
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [2, 4])
def test_boussinesq_rk_steps_match_oracle(ps, prec, order):
    n, dt = 32, 2e-3
    st = _state(n, n, n, 9, full=False) * 2.0
    kw = dict(nu=4e-3, kappa=8e-3, n_bv=2.5)
    f = inputs.forcing_field(n, n, n, seed=2)
    cfg = oracle.Config(n, n, n, rk_order=order, **kw)
    ref = st
    for _ in range(3):
        ref = oracle.boussinesq_rk_step(ref, dt, cfg, forcing=f)
    P, dtype = _prec(ps, prec)
    plan = ps.Plan(n, prec=P, eq=ps.Equations.BOUSSINESQ, rk_order=order,
                   forcing=torch.from_numpy(f).to("cuda", dtype), **kw)
    d = torch.from_numpy(st).to("cuda", dtype)
    for i in range(3):
        plan.rk_step(d, dt, t=i * dt)
    assert_parity(d.cpu().numpy().astype(np.complex128), ref, TOL[prec], "boussinesq step")
    plan.close()


def test_boussinesq_diagnostics_and_energy_stat(ps):
    n = 32
    st = _state(n, n, n, 13, full=False)
    cfg = oracle.Config(n, n, n)
    ref = oracle.boussinesq_diagnostics(st, cfg)
    plan = ps.Plan(n, prec=ps.Precision.FP64, eq=ps.Equations.BOUSSINESQ, nu=1e-3, kappa=1e-3, n_bv=1.0)
    d = plan.diagnostics(torch.from_numpy(st).to("cuda"))
    for key in ("energy", "enstrophy", "potential_energy", "max_u"):
        assert abs(d[key] - ref[key]) < 1e-12 * abs(ref[key]), key
    assert abs(d["helicity"] - ref["helicity"]) < 1e-12 * (ref["energy"] + ref["enstrophy"])
    plan.rk_step(torch.from_numpy(st).to("cuda"), 1e-3)
    e, _ = plan.step_stats()  # kinetic + potential energy of the step's start
    assert abs(e - (ref["energy"] + ref["potential_energy"])) < 1e-12
    plan.close()


def test_internal_gravity_wave_on_the_device(ps):
    """A single real plane wave rotates in the (velocity, theta) plane at
    Omega = N k_h/|k| and decays by exp(-nu |k|^2 t) (nu = kappa): 200 FP64
    IF-RK4 steps against the exact solution (the RK4 error at this step is
    far below the bound)."""
    n, nbv, nu = 32, 4.0, 0.01
    p, q, r = 3, 2, 1
    A, th0 = 0.6, 0.3
    k = np.array([p, q, r], dtype=float)
    e = np.array([0.0, 0.0, 1.0]) - k * k[2] / k.dot(k)
    e /= np.linalg.norm(e)
    st = np.zeros((4, n, n, n // 2 + 1), dtype=np.complex128)
    st[:3, r, q, p] = 0.5 * A * e
    st[3, r, q, p] = 0.5 * th0
    plan = ps.Plan(n, prec=ps.Precision.FP64, eq=ps.Equations.BOUSSINESQ, nu=nu, kappa=nu, n_bv=nbv)
    d = torch.from_numpy(st).to("cuda")
    dt, steps = 2e-3, 200
    for i in range(steps):
        plan.rk_step(d, dt, t=i * dt)
    out = d.cpu().numpy()
    T = dt * steps
    k2 = k.dot(k)
    om = nbv * math.sqrt(p * p + q * q) / math.sqrt(k2)
    c, s, dec = math.cos(om * T), math.sin(om * T), math.exp(-nu * k2 * T)
    a_ex, t_ex = dec * (A * c - th0 * s), dec * (th0 * c + A * s)
    assert abs(2 * np.real(np.dot(out[:3, r, q, p], e)) - a_ex) < 1e-9
    assert abs(2 * out[3, r, q, p].real - t_ex) < 1e-9
    other = out.copy()
    other[:, r, q, p] = 0
    assert np.max(np.abs(other)) < 1e-13
    plan.close()


def test_boussinesq_rhs_256_fp32_matches_oracle(ps):
    n = 256
    st = _state(n, n, n, 1, full=False)
    f = inputs.forcing_field(n, n, n, seed=2)
    kw = dict(nu=2e-3, kappa=2e-3, n_bv=1.0)
    ref = oracle.boussinesq_rhs(st, oracle.Config(n, n, n, **kw), forcing=f)
    plan = ps.Plan(n, prec=ps.Precision.FP32, eq=ps.Equations.BOUSSINESQ, rk_order=4,
                   forcing=torch.from_numpy(f).to("cuda", torch.complex64), **kw)
    got = plan.rhs(torch.from_numpy(st).to("cuda", torch.complex64)).cpu().numpy().astype(np.complex128)
    assert_parity(got, ref, 2e-6, "boussinesq rhs 256")
    plan.close()


def test_boussinesq_rhs_512_band_limited_matches_oracle(ps):
    """The benchmark's 512^3 Boussinesq launch shapes against the oracle: u and
    theta seeded on |p|, |q|, |r| <= 5 with the forcing, whose right-hand side
    the oracle gives exactly on a 32^3 grid (tests/parity.py); every mode
    compared on the device."""
    n, m = 512, BAND_M
    u = inputs.random_solenoidal_field(m, m, m, seed=1, kmax=(5, 5, 5))
    th = inputs.random_scalar_field(m, m, m, seed=61, kmax=(5, 5, 5))
    st = np.concatenate([u, th])
    f = inputs.forcing_field(m, m, m, seed=2)
    kw = dict(nu=2e-3, kappa=4e-3, n_bv=1.0)
    ref = oracle.boussinesq_rhs(st, oracle.Config(m, m, m, **kw), forcing=f)
    c64 = torch.complex64
    plan = ps.Plan(n, prec=ps.Precision.FP32, eq=ps.Equations.BOUSSINESQ, rk_order=4,
                   forcing=embed_on_device(f, n, torch, c64), **kw)
    out = plan.rhs(embed_on_device(st, n, torch, c64))
    torch.cuda.synchronize()
    plan.close()
    assert_device_parity(out, embed_on_device(ref, n, torch, c64), torch, 2e-6, "boussinesq rhs 512")
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mode", ["auto", "copy", "mapped"])
def test_boussinesq_host_steps_and_graph_replay_equal_device_steps(ps, mode):
    """The four-component state through the host-buffer path (every host mode
    writes the zeros of the masked modes) and through graph-replayed steps
    gives the device result bit for bit."""
    n, dt = 32, 2e-3
    st = _state(n, n, n, 23)  # content outside the retained modes
    kw = dict(nu=3e-3, kappa=4e-3, n_bv=2.0)
    plan = ps.Plan(n, prec=ps.Precision.FP32, eq=ps.Equations.BOUSSINESQ, **kw)
    dev = torch.from_numpy(st.astype(np.complex64)).cuda()
    for i in range(2):
        plan.rk_step(dev, dt, t=i * dt)
    mask = oracle.dealias_mask(oracle.Config(n, n, n))
    assert np.all(dev.cpu().numpy()[:, ~mask] == 0)
    ps.ps_plan_set_host_mode(plan.handle, {"auto": ps.HOST_AUTO, "copy": ps.HOST_COPY,
                                           "mapped": ps.HOST_MAPPED}[mode])
    host = torch.from_numpy(st.astype(np.complex64)).pin_memory()
    ps.ps_rk_step_host(plan.handle, host, dt, 0.0, 2)
    assert torch.equal(host, dev.cpu())
    g = torch.from_numpy(st.astype(np.complex64)).cuda()
    plan.rk_steps(g, dt, 2, t=0.0)
    torch.cuda.synchronize()
    assert torch.equal(g, dev)
    plan.close()
