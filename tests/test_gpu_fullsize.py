"""Parity at the benchmark's own sizes and launch configuration, and the
100-step energy criterion.

* 512^3 FP32 RHS of the seeded random field and forcing (the bench workload,
  same plan configuration) against the FP64 oracle, relative L2 <= 2e-6.
* 512^3 Taylor-Green: every mode of the RHS against the exact rational
  tendency -P[(u.grad)u] (no oracle run needed at that size).
* 1024^3 Taylor-Green (FP32, the largest benchmark grid): the same, built
  and compared on the device; and a band-limited seeded random field with
  forcing and viscosity at 1024^3 against the oracle's exact 32^3 result.
* 512^3 ABC flow: the nonlinear term vanishes identically.
* 100 IF-RK4 steps in FP32: total energy within 1e-4 of the FP64 oracle
  (64^3, oracle run in full) and of the FP64 CUDA path (256^3, whose every
  RHS is itself held to 1e-12 of the oracle by test_gpu_parity).
* The 256^3 workload in FP32 against the oracle itself for its right-hand
  side and its first two RK4 steps, mode by mode.
"""

import math

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs

from . import exact_fourier as xf
from .parity import BAND_K, BAND_M, assert_device_parity, assert_parity, embed_on_device

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_bench_workload_rhs_512_matches_oracle(ps):
    n, nu = 512, 2e-3
    u = inputs.random_solenoidal_field(n, n, n, seed=1)
    f = inputs.forcing_field(n, n, n, seed=2)
    ud = torch.from_numpy(u).to("cuda", torch.complex64)
    fd = torch.from_numpy(f).to("cuda", torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=nu, rk_order=4, forcing=fd)
    out = plan.rhs(ud)
    got = out.cpu().numpy()
    plan.close()
    del ud, fd, out
    torch.cuda.empty_cache()
    ref = oracle.rhs(u, oracle.Config(n, n, n, nu=nu), forcing=f)
    assert_parity(got.astype(np.complex128), ref, 2e-6, "512^3 rhs")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_taylor_green_512_matches_exact_tendency(ps, prec):
    n = 512
    P, dt = (ps.Precision.FP32, torch.complex64) if prec == "fp32" else (ps.Precision.FP64, torch.complex128)
    ud = torch.from_numpy(inputs.taylor_green(n, n, n)).to("cuda", dt)
    plan = ps.Plan(n, prec=P, nu=0.0)
    out = plan.rhs(ud).cpu().numpy().astype(np.complex128)
    plan.close()
    exact = np.zeros_like(out)
    for (p, q, r), v in xf.euler_rate(xf.trig_modes([(0, 1, ("s", 1), ("c", 1), ("c", 1)),
                                                      (1, -1, ("c", 1), ("s", 1), ("c", 1))])).items():
        if p >= 0:
            exact[:, r % n, q % n, p] = [complex(c) for c in v]
    tol = 2e-6 if prec == "fp32" else 1e-12
    assert np.max(np.abs(out - exact)) < tol * np.max(np.abs(exact))


def _device_modes(modes, n, dtype):
    """A state or tendency given as exact modes, built on the device (no host
    copy of a 1024^3 field)."""
    t = torch.zeros((3, n, n, n // 2 + 1), dtype=dtype, device="cuda")
    for (p, q, r), v in modes.items():
        if p >= 0:
            t[:, r % n, q % n, p] = torch.tensor([complex(c) for c in v], dtype=dtype)
    return t


def test_taylor_green_1024_matches_exact_tendency(ps):
    """The largest grid the bench times (1024^3 FP32: 16 points per thread in
    the x pass, half the rows per CTA): every mode of the right-hand side of
    the Taylor-Green vortex against its exact rational tendency, on the
    device."""
    n = 1024
    tg = xf.trig_modes([(0, 1, ("s", 1), ("c", 1), ("c", 1)), (1, -1, ("c", 1), ("s", 1), ("c", 1))])
    ud = _device_modes(tg, n, torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=0.0)
    out = plan.rhs(ud)
    torch.cuda.synchronize()
    plan.close()
    del ud
    exact = _device_modes(xf.euler_rate(tg), n, torch.complex64)
    scale = float(exact.abs().max())
    err = float((out - exact).abs().max())
    del out, exact
    torch.cuda.empty_cache()
    assert scale == 1.0 / 32  # the largest exact coefficient
    assert err < 2e-6 * scale, err


def test_band_limited_random_field_1024_matches_oracle(ps):
    """A seeded random solenoidal field on |p|, |q|, |r| <= 5 with the forcing
    (2 <= |k| <= 3) and viscosity: its right-hand side lies on |p|, |q|, |r|
    <= 10, which a 32^3 grid (2/3 half-width 10) and the 1024^3 grid both
    hold without truncation or aliasing, so the oracle's 32^3 right-hand
    side placed at the same signed modes is the 1024^3 one.  Every mode of
    the 1024^3 FP32 result is compared on the device."""
    n, m, nu = 1024, BAND_M, 2e-3
    u = inputs.random_solenoidal_field(m, m, m, seed=1, kmax=(5, 5, 5))
    f = inputs.forcing_field(m, m, m, seed=2)
    ref = oracle.rhs(u, oracle.Config(m, m, m, nu=nu), forcing=f)
    assert np.max(np.abs(ref[:, :, :, BAND_K + 1:])) == 0.0
    ud, fd = embed_on_device(u, n, torch, torch.complex64), embed_on_device(f, n, torch, torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=nu, forcing=fd)
    out = plan.rhs(ud)
    torch.cuda.synchronize()
    plan.close()
    del ud, fd
    assert_device_parity(out, embed_on_device(ref, n, torch, torch.complex64), torch, 2e-6, "1024^3 rhs")
    del out
    torch.cuda.empty_cache()


def test_abc_512_nonlinear_term_vanishes(ps):
    n = 512
    ud = torch.from_numpy(inputs.abc_flow(n, n, n)).to("cuda", torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=0.0)
    out = plan.rhs(ud)
    assert float(out.abs().max()) < 2e-6
    plan.close()


def _energy_after(ps, n, prec, steps, dt=1e-3, nu=2e-3):
    P, dtype = (ps.Precision.FP32, torch.complex64) if prec == "fp32" else (ps.Precision.FP64, torch.complex128)
    u = inputs.random_solenoidal_field(n, n, n, seed=1)
    f = inputs.forcing_field(n, n, n, seed=2)
    ud = torch.from_numpy(u).to("cuda", dtype)
    plan = ps.Plan(n, prec=P, nu=nu, rk_order=4, forcing=torch.from_numpy(f).to("cuda", dtype))
    for i in range(steps):
        plan.rk_step(ud, dt, t=i * dt)
    e = plan.diagnostics(ud)["energy"]
    plan.close()
    return e


def test_fp32_energy_after_100_steps_matches_oracle_64(ps):
    n, dt, nu = 64, 1e-3, 2e-3
    u = inputs.random_solenoidal_field(n, n, n, seed=1)
    f = inputs.forcing_field(n, n, n, seed=2)
    cfg = oracle.Config(n, n, n, nu=nu, rk_order=4)
    for _ in range(100):
        u = oracle.rk_step(u, dt, cfg, forcing=f)
    e_ref = oracle.diagnostics(u, cfg)["energy"]
    e32 = _energy_after(ps, n, "fp32", 100, dt, nu)
    assert abs(e32 - e_ref) <= 1e-4 * e_ref


def test_fp32_energy_after_100_steps_256(ps):
    e32 = _energy_after(ps, 256, "fp32", 100)
    e64 = _energy_after(ps, 256, "fp64", 100)
    assert abs(e32 - e64) <= 1e-4 * e64
    assert math.isfinite(e32) and 0.3 < e32 < 0.7


def test_fp32_state_error_per_step_256(ps):
    """FP32 against the FP64 CUDA path on the forced 256^3 workload, every step
    of 100: the relative L2 distance of the states stays small (its growth is
    the FP32 rounding carried by the flow) and the energies agree to 1e-4."""
    import bench
    r = bench.fp32_error_per_step(100, torch.device("cuda"), torch.cuda.current_stream())
    assert r["max_rel_l2"] < 1e-4
    assert r["energy_rel_diff"] < 1e-4



def test_fp32_rk4_steps_256_match_oracle(ps):
    """The forced 256^3 workload in FP32 against the FP64 oracle itself, mode
    by mode: the right-hand side and the states after the first two IF-RK4
    steps (relative L2 and per-mode bound 2e-6), and the diagnostics of the
    stepped state."""
    n, nu, dt = 256, 2e-3, 1e-3
    u = inputs.random_solenoidal_field(n, n, n, seed=1)
    f = inputs.forcing_field(n, n, n, seed=2)
    cfg = oracle.Config(n, n, n, nu=nu, rk_order=4)
    ud = torch.from_numpy(u).to("cuda", torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=nu, rk_order=4,
                   forcing=torch.from_numpy(f).to("cuda", torch.complex64))
    got_rhs = plan.rhs(ud).cpu().numpy().astype(np.complex128)
    got = []
    for i in range(2):
        plan.rk_step(ud, dt, t=i * dt)
        got.append(ud.cpu().numpy().astype(np.complex128))
    d_gpu = plan.diagnostics(ud)
    plan.close()
    del ud
    torch.cuda.empty_cache()
    assert_parity(got_rhs, oracle.rhs(u, cfg, forcing=f), 2e-6, "256^3 rhs")
    ref = u
    for i in range(2):
        ref = oracle.rk_step(ref, dt, cfg, forcing=f)
        assert_parity(got[i], ref, 2e-6, f"256^3 state after step {i + 1}")
    d = oracle.diagnostics(ref, cfg)
    for key in ("energy", "enstrophy", "max_u", "cfl_dt"):
        assert abs(d_gpu[key] - d[key]) <= 2e-6 * abs(d[key]), key
    assert abs(d_gpu["helicity"] - d["helicity"]) <= 2e-6 * 2 * math.sqrt(d["energy"] * d["enstrophy"])
