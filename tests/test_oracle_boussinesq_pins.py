"""Pins of the oracle's Boussinesq system (Eqs. mom, temp, divv) against
exact arithmetic, closed-form internal gravity waves, a brute-force
convolution and the ideal invariants; CPU only."""

import math

import numpy as np
import pytest

import oracle
from oracle.spectral import Config
from paper_1808_01309_gb300 import inputs

from . import exact_fourier as xf

U_TERMS = [(0, 1, ("s", 1), ("c", 1), ("c", 1)), (1, -1, ("c", 1), ("s", 1), ("c", 1))]
TH_TERMS = [(0, 1, ("c", 1), ("1", 0), ("s", 1)), (0, 0.5, ("1", 0), ("s", 2), ("c", 1)),
            (0, 0.25, ("s", 1), ("c", 1), ("1", 0))]


def _to_array(modes, n, ncomp=3):
    out = np.zeros((ncomp, n, n, n // 2 + 1), dtype=np.complex128)
    for (p, q, r), v in modes.items():
        if p >= 0:
            out[:, r % n, q % n, p] = [complex(c) for c in v[:ncomp]]
    return out


def _random_state(n, seed, lx=2 * math.pi):
    u = inputs.random_solenoidal_field(n, n, n, seed=seed, lx=lx)
    th = inputs.random_scalar_field(n, n, n, seed=seed + 60, lx=lx)
    return np.concatenate([u, th])


def _plane_wave(n, p, q, r, A, th0):
    """Real single-mode state: u = A e cos(k.x), theta = th0 cos(k.x) with
    e the unit vector along z_hat - k k_z/|k|^2 (perpendicular to k)."""
    k = np.array([p, q, r], dtype=float)
    e = np.array([0.0, 0.0, 1.0]) - k * k[2] / k.dot(k)
    e /= np.linalg.norm(e)
    st = np.zeros((4, n, n, n // 2 + 1), dtype=np.complex128)
    st[:3, r % n, q % n, p] = 0.5 * A * e
    st[3, r % n, q % n, p] = 0.5 * th0
    if p == 0:  # the conjugate partner is stored too
        st[:3, (-r) % n, (-q) % n, 0] = 0.5 * A * e
        st[3, (-r) % n, (-q) % n, 0] = 0.5 * th0
    return st, e


def test_tendency_matches_exact_advective_form():
    """u_t = -P[(u.grad)u + N theta z_hat], theta_t = -(u.grad)theta + N w,
    summed exactly in rationals (advective form, convolution pair by pair),
    vs the oracle's rotational / divergence-form pseudospectral terms."""
    nbv = 2
    u, th = xf.trig_modes(U_TERMS), xf.trig_modes(TH_TERMS)
    buoy = {k: [xf.G(), xf.G(), v[0] * nbv] for k, v in th.items()}
    ut = xf.scale(xf.project(xf.add(xf.advect(u, u), buoy)), -1)
    tt = xf.add(xf.scale(xf.advect(u, th), -1), {k: [v[2] * nbv, xf.G(), xf.G()] for k, v in u.items()})
    n = 16
    cfg = Config(n, n, n, n_bv=float(nbv))
    st = np.concatenate([_to_array(u, n), _to_array(th, n, 1)])
    got = oracle.boussinesq_rhs(st, cfg)
    exp = np.concatenate([_to_array(ut, n), _to_array(tt, n, 1)])
    assert np.max(np.abs(exp[:3])) > 0.1 and np.max(np.abs(exp[3])) > 0.05
    assert np.max(np.abs(got - exp)) < 1e-14


def test_scalar_advection_matches_brute_force_convolution():
    """-(u.grad theta)^(k) = -sum_{p+q=k} u_hat(p) . (i q) theta_hat(q) over the
    full spectra of random band-limited fields (alias-free at 8^3), against
    the oracle's divergence form -i k . F[u theta]."""
    n = 8
    cfg = Config(n, n, n)
    st = _random_state(n, 5)
    full = lambda h: np.fft.fftn(oracle.inverse(h, cfg), axes=(-3, -2, -1), norm="forward")
    U, TH = full(st[:3]), full(st[3])
    idx = np.fft.fftfreq(n, 1.0 / n).astype(int)
    modes = [(a, b, c) for a in range(n) for b in range(n) for c in range(n) if np.abs(TH[a, b, c]) > 0]
    umodes = [(a, b, c) for a in range(n) for b in range(n) for c in range(n) if np.abs(U[:, a, b, c]).max() > 0]
    out = np.zeros((n, n, n), dtype=np.complex128)
    for (a, b, c) in umodes:
        for (d, e, f) in modes:
            qz, qy, qx = idx[d], idx[e], idx[f]
            s = U[0, a, b, c] * 1j * qx + U[1, a, b, c] * 1j * qy + U[2, a, b, c] * 1j * qz
            out[(a + d) % n, (b + e) % n, (c + f) % n] -= s * TH[d, e, f]
    D = oracle.dealias_mask(cfg)
    exp = out[:, :, : n // 2 + 1] * D
    _, got = oracle.boussinesq_nonlinear(st, cfg)
    assert np.max(np.abs(exp)) > 1e-3
    assert np.max(np.abs(got - exp)) < 1e-13


def test_ideal_total_energy_and_scalar_variance_are_conserved():
    """Without diffusion and forcing the right-hand side moves no total energy
    1/2 <|u|^2 + theta^2>: the nonlinear terms conserve kinetic energy and
    scalar variance separately and the two buoyancy terms exchange
    N <w theta> with opposite signs (a sign error in either breaks this)."""
    n = 16
    for nbv in (0.0, 1.7):
        cfg = Config(n, n, n, n_bv=nbv, lx=2 * math.pi * 1.5)
        st = _random_state(n, 11, lx=cfg.lx)
        r = oracle.boussinesq_rhs(st, cfg)
        w = oracle.hermitian_weight(cfg)
        dk = float(np.sum(w * np.real(np.sum(np.conj(st[:3]) * r[:3], axis=0))))
        dp = float(np.sum(w * np.real(np.conj(st[3]) * r[3])))
        exch = nbv * float(np.sum(w * np.real(np.conj(st[2]) * st[3])))
        assert abs(dk + dp) < 1e-13
        assert abs(dp - exch) < 1e-13  # advection moves no variance: dp is the exchange alone
        if nbv:
            assert abs(exch) > 1e-3


def test_internal_gravity_wave_tendency_and_frequency():
    """A single real plane wave (u along e, perpendicular to k, and theta) has
    no nonlinear term; its tendency is A_t = -Omega theta, theta_t = Omega A
    with Omega = N k_h/|k| (the buoyancy projected on e, and N w = N A e_z), so
    it rotates in the (A, theta) plane at the internal-wave frequency; with
    nu = kappa both decay by exp(-nu |k|^2 t)."""
    n, nbv, nu = 16, 3.0, 0.02
    p, q, r = 2, 1, 3
    A, th0 = 0.7, -0.4
    cfg = Config(n, n, n, n_bv=nbv, nu=nu, kappa=nu)
    st, e = _plane_wave(n, p, q, r, A, th0)
    k2 = p * p + q * q + r * r
    om = nbv * math.sqrt(p * p + q * q) / math.sqrt(k2)
    assert abs(e[2] - math.sqrt(p * p + q * q) / math.sqrt(k2)) < 1e-15
    R = oracle.boussinesq_rhs(st, cfg)
    exp = np.zeros_like(st)
    exp[:3, r, q, p] = 0.5 * (-om * th0 - nu * k2 * A) * e
    exp[3, r, q, p] = 0.5 * (om * A - nu * k2 * th0)
    assert np.max(np.abs(R - exp)) < 1e-14
    # RK4 against the exact damped rotation; error falls as dt^4
    T = 0.3
    errs = []
    for steps in (10, 20):
        dt = T / steps
        s = st.copy()
        for _ in range(steps):
            s = oracle.boussinesq_rk_step(s, dt, Config(n, n, n, n_bv=nbv, nu=nu, kappa=nu, rk_order=4))
        c, sn, d = math.cos(om * T), math.sin(om * T), math.exp(-nu * k2 * T)
        a_ex, t_ex = d * (A * c - th0 * sn), d * (th0 * c + A * sn)
        a_num = 2 * np.real(np.dot(s[:3, r, q, p], e))
        errs.append(abs(a_num - a_ex) + abs(2 * s[3, r, q, p].real - t_ex))
    assert errs[1] < 1e-6
    assert 12.0 < errs[0] / errs[1] < 20.0


def test_zero_scalar_reduces_to_hydrodynamics():
    n = 16
    cfg = Config(n, n, n, nu=0.01, kappa=0.03, n_bv=0.0)
    u = inputs.random_solenoidal_field(n, n, n, seed=3)
    f = inputs.forcing_field(n, n, n, seed=2)
    st = np.concatenate([u, np.zeros_like(u[:1])])
    r = oracle.boussinesq_rhs(st, cfg, forcing=f)
    assert np.max(np.abs(r[:3] - oracle.rhs(u, cfg, forcing=f))) < 1e-15
    assert np.max(np.abs(r[3])) == 0.0
    s = oracle.boussinesq_rk_step(st, 0.01, cfg, forcing=f)
    assert np.max(np.abs(s[:3] - oracle.rk_step(u, 0.01, cfg, forcing=f))) < 1e-15


def test_passive_scalar_diffusion_is_exact():
    """With u = 0 and N = 0 the scalar only diffuses: theta_hat(t) =
    exp(-kappa |k|^2 t) theta_hat(0) at any dt (Lawson form is exact for the
    linear part)."""
    n, kappa, dt = 16, 0.05, 0.1
    cfg = Config(n, n, n, kappa=kappa, nu=0.01)
    th = inputs.random_scalar_field(n, n, n, seed=9)
    st = np.concatenate([np.zeros((3,) + th.shape[1:], dtype=np.complex128), th])
    s = st
    for _ in range(3):
        s = oracle.boussinesq_rk_step(s, dt, cfg)
    kx, ky, kz = oracle.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    assert np.max(np.abs(s[3] - th[0] * np.exp(-kappa * k2 * 3 * dt))) < 1e-15
    assert np.max(np.abs(s[:3])) == 0.0


@pytest.mark.parametrize("order,ratio", [(4, 16.0), (2, 4.0)])
def test_rk_order_on_the_nonlinear_system(order, ratio):
    n = 16
    cfg = Config(n, n, n, nu=0.01, kappa=0.02, n_bv=2.0, rk_order=order)
    st = _random_state(n, 21)
    T = 0.2

    def run(steps):
        s = st
        for _ in range(steps):
            s = oracle.boussinesq_rk_step(s, T / steps, cfg)
        return s

    ref = run(64)
    e1 = np.linalg.norm(run(8) - ref)
    e2 = np.linalg.norm(run(16) - ref)
    assert 0.75 * ratio < e1 / e2 < 1.35 * ratio


def test_velocity_tendency_is_solenoidal_and_potential_energy_diagnostic():
    n = 16
    cfg = Config(n, n, n, n_bv=1.3, nu=0.01, kappa=0.01)
    st = _random_state(n, 31)
    r = oracle.boussinesq_rhs(st, cfg)
    kx, ky, kz = oracle.wavenumbers(cfg)
    assert np.max(np.abs(kx * r[0] + ky * r[1] + kz * r[2])) < 1e-14 * np.max(np.abs(r[:3]))
    d = oracle.boussinesq_diagnostics(st, cfg)
    th = oracle.inverse(st[3], cfg)
    assert abs(d["potential_energy"] - 0.5 * np.mean(th * th)) < 1e-15
    assert abs(d["potential_energy"] - 0.5) < 1e-14


def test_linear_terms_carry_their_own_diffusivities():
    """With the nonlinear terms off and N = 0 the right-hand side is
    -nu |k|^2 u_hat and -kappa |k|^2 theta_hat, and a Lawson step decays each
    by its own exp(-nu |k|^2 dt), exp(-kappa |k|^2 dt) (nu != kappa)."""
    n, nu, kappa, dt = 16, 0.01, 0.05, 0.1
    cfg = Config(n, n, n, nu=nu, kappa=kappa)
    st = _random_state(n, 11)
    kx, ky, kz = oracle.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    D = oracle.dealias_mask(cfg)
    r = oracle.boussinesq_rhs(st, cfg, nonlinear_on=False)
    assert np.max(np.abs(r[:3] + nu * k2 * st[:3] * D)) < 1e-15
    assert np.max(np.abs(r[3] + kappa * k2 * st[3] * D)) < 1e-15
    s = oracle.boussinesq_rk_step(st, dt, cfg, nonlinear_on=False)
    assert np.max(np.abs(s[:3] - st[:3] * D * np.exp(-nu * k2 * dt))) < 1e-15
    assert np.max(np.abs(s[3] - st[3] * D * np.exp(-kappa * k2 * dt))) < 1e-15
