"""Pins of the oracle's MHD system (Eqs. uMHD, bMHD) against exact arithmetic
and the ideal invariants; CPU only."""

import math

import numpy as np
import pytest

import oracle
from oracle.spectral import Config
from paper_1808_01309_gb300 import inputs

from . import exact_fourier as xf

U_TERMS = [(0, 1, ("s", 1), ("c", 1), ("c", 1)), (1, -1, ("c", 1), ("s", 1), ("c", 1))]
# ABC-like magnetic field plus a uniform field along x (the k = 0 mode)
B_TERMS = [(0, 1, ("1", 0), ("1", 0), ("s", 1)), (1, 1, ("s", 1), ("1", 0), ("1", 0)),
           (2, 1, ("1", 0), ("s", 1), ("1", 0)), (0, 0.5, ("1", 0), ("1", 0), ("1", 0)),
           (2, 1, ("c", 2), ("1", 0), ("1", 0))]


def _to_array(modes, n):
    out = np.zeros((3, n, n, n // 2 + 1), dtype=np.complex128)
    for (p, q, r), v in modes.items():
        if p >= 0:
            out[:, r % n, q % n, p] = [complex(c) for c in v]
    return out


def _random_ub(n, seed):
    u = inputs.random_solenoidal_field(n, n, n, seed=seed)
    b = inputs.random_solenoidal_field(n, n, n, seed=seed + 50)
    return np.concatenate([u, b])


def test_mhd_tendency_matches_exact_advective_form():
    """u_t = -P[(u.grad)u - (B.grad)B], B_t = (B.grad)u - (u.grad)B summed
    exactly in rationals, vs the oracle's rotational, pseudospectral form."""
    u, b = xf.trig_modes(U_TERMS), xf.trig_modes(B_TERMS)
    ut = xf.scale(xf.project(xf.add(xf.advect(u, u), xf.scale(xf.advect(b, b), -1))), -1)
    bt = xf.add(xf.advect(b, u), xf.scale(xf.advect(u, b), -1))
    n = 16
    cfg = Config(n, n, n)
    ub = np.concatenate([_to_array(u, n), _to_array(b, n)])
    got = oracle.mhd_rhs(ub, cfg)
    exp = np.concatenate([_to_array(ut, n), _to_array(bt, n)])
    assert np.max(np.abs(exp)) > 0.1
    assert np.max(np.abs(got - exp)) < 1e-14


def test_zero_magnetic_field_reduces_to_hydrodynamics():
    n = 16
    cfg = Config(n, n, n, nu=0.01, eta=0.02)
    u = inputs.random_solenoidal_field(n, n, n, seed=3)
    ub = np.concatenate([u, np.zeros_like(u)])
    r = oracle.mhd_rhs(ub, cfg)
    assert np.max(np.abs(r[:3] - oracle.rhs(u, cfg))) < 1e-15
    assert np.max(np.abs(r[3:])) == 0.0
    s = oracle.mhd_rk_step(ub, 0.01, cfg)
    assert np.max(np.abs(s[:3] - oracle.rk_step(u, 0.01, cfg))) < 1e-15


def test_ideal_invariants_are_not_transferred():
    """Total energy, cross helicity and magnetic helicity are invariants of
    the ideal dealiased Galerkin system: their instantaneous transfer by the
    nonlinear terms vanishes."""
    n = 32
    cfg = Config(n, n, n)
    ub = _random_ub(n, 11)
    r = oracle.mhd_rhs(ub, cfg)
    w = oracle.hermitian_weight(cfg)
    u, b, ru, rb = ub[:3], ub[3:], r[:3], r[3:]

    def inner(a, c):
        return float(np.sum(w * np.real(np.sum(np.conj(a) * c, axis=0))))

    def scale(a, c):
        return float(np.sum(w * np.abs(a).sum(0) * np.abs(c).sum(0)))

    kx, ky, kz = oracle.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(k2 > 0, oracle.curl_hat(b, cfg) / np.where(k2 > 0, k2, 1.0), 0.0)
    assert abs(inner(u, ru) + inner(b, rb)) < 1e-14 * (scale(u, ru) + scale(b, rb))
    assert abs(inner(b, ru) + inner(u, rb)) < 1e-14 * (scale(b, ru) + scale(u, rb))
    assert abs(inner(a, rb)) < 1e-14 * scale(a, rb)
    # both right-hand sides are solenoidal
    for f in (ru, rb):
        assert np.max(np.abs(kx * f[0] + ky * f[1] + kz * f[2])) < 1e-13


def test_mhd_rk4_order():
    cfg = Config(16, 16, 16, nu=0.1, eta=0.3, rk_order=4)
    ub = _random_ub(16, 21) * 3.0
    T = 0.2

    def run(dt):
        v = ub
        for _ in range(int(round(T / dt))):
            v = oracle.mhd_rk_step(v, dt, cfg)
        return v

    ref = run(T / 64)
    e1 = np.linalg.norm(run(T / 4) - ref)
    e2 = np.linalg.norm(run(T / 8) - ref)
    assert 13.0 < e1 / e2 < 19.0


def test_mhd_diagnostics_closed_forms():
    n = 16
    cfg = Config(n, n, n)
    u = inputs.abc_flow(n, n, n)
    ub = np.concatenate([u, u])       # B = u, an Alfvenic ABC state
    d = oracle.mhd_diagnostics(ub, cfg)
    assert abs(d["energy"] - 1.5) < 1e-14 and abs(d["magnetic_energy"] - 1.5) < 1e-14
    assert abs(d["cross_helicity"] - 3.0) < 1e-14
    # curl B = B for ABC, so A = B/|k|^2 = B and H_m = <A.B> = 2 E_B
    assert abs(d["magnetic_helicity"] - 3.0) < 1e-14
    # u = B Beltrami: all nonlinear terms vanish
    assert np.max(np.abs(oracle.mhd_rhs(ub, cfg))) < 1e-14


def _beltrami(n, k):
    """ABC field of wavenumber k (unit coefficients): curl = k times the field."""
    return inputs.trig_field(n, n, n, [
        (0, 1.0, ("1", 0), ("1", 0), ("s", k)), (0, 1.0, ("1", 0), ("c", k), ("1", 0)),
        (1, 1.0, ("s", k), ("1", 0), ("1", 0)), (1, 1.0, ("1", 0), ("1", 0), ("c", k)),
        (2, 1.0, ("1", 0), ("s", k), ("1", 0)), (2, 1.0, ("c", k), ("1", 0), ("1", 0))])


@pytest.mark.parametrize("order", [2, 4])
def test_parallel_beltrami_fields_decay_exactly(order):
    """u and B multiples of one Beltrami field of |k| = 2: u x omega, j x B and
    u x B vanish, so u decays as exp(-nu |k|^2 t) and B as exp(-eta |k|^2 t)
    with no coupling, and a Lawson step is exact at any dt.  nu != eta tells
    the two rates apart."""
    n, nu, eta, dt = 16, 0.05, 0.02, 0.1
    cfg = Config(n, n, n, nu=nu, eta=eta, rk_order=order)
    f = _beltrami(n, 2)
    assert np.max(np.abs(oracle.curl_hat(f, cfg) - 2.0 * f)) < 1e-14
    ub = np.concatenate([f, 0.5 * f])
    r = oracle.mhd_rhs(ub, cfg)
    assert np.max(np.abs(r - np.concatenate([-4.0 * nu * f, -4.0 * eta * 0.5 * f]))) < 1e-15
    v = ub
    for _ in range(5):
        v = oracle.mhd_rk_step(v, dt, cfg)
    T = 5 * dt
    assert np.max(np.abs(v[:3] - f * math.exp(-4.0 * nu * T))) < 1e-15
    assert np.max(np.abs(v[3:] - 0.5 * f * math.exp(-4.0 * eta * T))) < 1e-15


def test_magnetic_helicity_of_a_wavenumber_two_field():
    """B a Beltrami field of |k| = 2: the Coulomb-gauge potential
    A = i k x B / |k|^2 is B/2, so the magnetic helicity sum w Re(A* . B)
    equals the magnetic energy 1/2 sum w |B|^2 = 1.5; with u = B/3 the cross
    helicity is 1/3 sum w |B|^2 = 1 and the kinetic energy 1.5/9."""
    n = 16
    cfg = Config(n, n, n)
    f = _beltrami(n, 2)
    d = oracle.mhd_diagnostics(np.concatenate([f / 3.0, f]), cfg)
    assert abs(d["magnetic_energy"] - 1.5) < 1e-14
    assert abs(d["magnetic_helicity"] - 1.5) < 1e-14
    assert abs(d["cross_helicity"] - 1.0) < 1e-14
    assert abs(d["energy"] - 1.5 / 9.0) < 1e-14
