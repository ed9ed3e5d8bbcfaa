"""Pins of the LES-closure oracle (oracle/les.py); CPU only."""

import math

import numpy as np
import pytest

import oracle
from oracle import les
from oracle.spectral import Config
from paper_1808_01309_gb300 import inputs


def test_gelu_derivative_matches_finite_differences():
    x = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (les.gelu(x + h) - les.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - les.gelu_grad(x))) < 1e-8
    # limits: gelu(x) -> x for large x, -> 0 for very negative x
    assert abs(les.gelu(10.0) - 10.0) < 1e-12 and abs(les.gelu(-10.0)) < 1e-12


def test_mlp_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    p = les.init_params(seed=1)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    X = rng.standard_normal((37, 5))
    T = rng.standard_normal((37, 6))
    _, g = les.mse_and_grads(p, X, T)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = les.mse_and_grads(p, X, T)
            flat[idx] = old - h
            lm, _ = les.mse_and_grads(p, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx)


def _inv(A):
    return les.invariants(np.asarray(A, dtype=np.float64)[:, :, None])[:, 0]


def test_invariants_closed_forms():
    a, b = 0.7, -0.3
    lam = _inv(np.diag([a, b, -a - b]))
    assert np.allclose(lam, [a * a + b * b + (a + b) ** 2, 0, a ** 3 + b ** 3 - (a + b) ** 3, 0, 0], atol=1e-15)
    w = 1.3
    lam = _inv([[0, -w, 0], [w, 0, 0], [0, 0, 0]])
    assert np.allclose(lam, [0, -2 * w * w, 0, 0, 0], atol=1e-15)
    g = 0.9
    lam = _inv([[0, g, 0], [0, 0, 0], [0, 0, 0]])
    assert np.allclose(lam, [g * g / 2, -g * g / 2, 0, 0, -g ** 4 / 8], atol=1e-15)
    # diagonal strain (a, b, c) with a rotation w about z: R^2 = diag(-w^2, -w^2, 0)
    a, b, w = 0.8, -0.3, 1.1
    c = -a - b
    lam = _inv([[a, -w, 0], [w, b, 0], [0, 0, c]])
    assert np.allclose(lam, [a * a + b * b + c * c, -2 * w * w, a ** 3 + b ** 3 + c ** 3,
                             -w * w * (a + b), -w * w * (a * a + b * b)], atol=1e-15)


def test_gradient_of_taylor_green_is_analytic():
    n = 16
    cfg = Config(n, n, n)
    A = les.gradient(inputs.taylor_green(n, n, n), cfg)
    z, y, x = np.meshgrid(*(np.arange(n) * 2 * math.pi / n,) * 3, indexing="ij")
    exp = np.zeros_like(A)
    exp[0, 0] = np.cos(x) * np.cos(y) * np.cos(z)
    exp[0, 1] = -np.sin(x) * np.sin(y) * np.cos(z)
    exp[0, 2] = -np.sin(x) * np.cos(y) * np.sin(z)
    exp[1, 0] = np.sin(x) * np.sin(y) * np.cos(z)
    exp[1, 1] = -np.cos(x) * np.cos(y) * np.cos(z)
    exp[1, 2] = np.cos(x) * np.sin(y) * np.sin(z)
    assert np.max(np.abs(A - exp)) < 1e-14


def test_subgrid_stress_closed_form():
    """u_y = cos(2x) + cos(30x) on a 128^3 DNS grid filtered at kc = 21:
    F[u_y^2] = 1 + cos(4x)/2 and u_y_bar^2 = 1/2 + cos(4x)/2, so tau_yy = 1/2
    and every other component vanishes."""
    n, kc, nl = 128, 21, 64
    uh = inputs.trig_field(n, n, n, [(1, 1.0, ("c", 2), ("1", 0), ("1", 0)),
                                     (1, 1.0, ("c", 30), ("1", 0), ("1", 0))])
    tau = les.sgs_stress_true(uh, n, nl, kc)
    expect = np.zeros_like(tau)
    expect[1] = 0.5
    assert np.max(np.abs(tau - expect)) < 1e-14


def test_subgrid_stress_of_a_resolved_mode_is_zero():
    """u_x = cos(12 y), a single mode inside the filter: F[u u] = F[ubar ubar]
    exactly, so tau vanishes (the product ubar ubar itself has a cos(24 y)
    part above kc that the LES truncates too)."""
    n, kc, nl = 128, 21, 64
    uh = inputs.trig_field(n, n, n, [(0, 1.0, ("1", 0), ("c", 12), ("1", 0))])
    tau = les.sgs_stress_true(uh, n, nl, kc)
    assert np.max(np.abs(tau)) < 1e-15


def test_subgrid_stress_vanishes_for_band_limited_fields():
    n, kc, nl = 64, 21, 64
    u = inputs.random_solenoidal_field(n, n, n, seed=5, kmax=(10, 10, 10))
    tau = les.sgs_stress_true(u, n, nl, kc)
    assert np.max(np.abs(tau)) < 1e-15 * 1e3


def test_zero_network_reduces_les_to_the_plain_method():
    n = 16
    cfg = Config(n, n, n, nu=1e-2)
    u = inputs.random_solenoidal_field(n, n, n, seed=7)
    p = les.init_params(seed=2)
    p["W3"][:] = 0
    p["b3"][:] = 0
    norm = dict(mean=np.zeros(5), std=np.ones(5), s_tau=1.0, s_A=1.0)
    assert np.max(np.abs(les.closure_term(u, cfg, p, norm))) == 0.0
    assert np.max(np.abs(les.les_rhs(u, cfg, p, norm) - oracle.rhs(u, cfg))) < 1e-15


def test_constant_strain_coefficient_is_an_eddy_viscosity():
    """g = (c, 0, ..., 0) for every input gives tau = s_tau c S / s_A; for a
    solenoidal field div S = (1/2) lap u, so the closure term is
    (s_tau c / (2 s_A)) |k|^2 u_hat on the retained modes."""
    n = 16
    cfg = Config(n, n, n, lx=2 * math.pi, ly=5.0, lz=3.0)
    u = inputs.random_solenoidal_field(n, n, n, seed=8, lx=2 * math.pi, ly=5.0, lz=3.0)
    norm = dict(mean=np.zeros(5), std=np.ones(5) * 10.0, s_tau=0.03, s_A=2.5)
    p = les.init_params(seed=3)
    p["W3"][:] = 0
    p["b3"][:] = [-0.7, 0, 0, 0, 0, 0]
    kx, ky, kz = oracle.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    expect = (0.03 * -0.7 / (2 * 2.5)) * k2 * u * oracle.dealias_mask(cfg)
    got = les.closure_term(u, cfg, p, norm)
    assert np.max(np.abs(got - expect)) < 1e-14 * np.max(np.abs(expect))
    # linear in the output layer
    p2 = les.init_params(seed=3)
    c1 = les.closure_term(u, cfg, p2, norm)
    p2["W3"] *= 2
    p2["b3"] *= 2
    assert np.max(np.abs(les.closure_term(u, cfg, p2, norm) - 2 * c1)) < 1e-14 * np.max(np.abs(c1))


def _tb(A, s_A=1.0):
    return les.tensor_basis(np.asarray(A, dtype=np.float64)[:, :, None], s_A)[:, :, 0]


def test_tensor_basis_closed_forms():
    """Hand-derived basis tensors for a simple shear and for a diagonal strain
    with a rotation about z (components 11, 22, 33, 12, 13, 23)."""
    g = 1.7
    T = _tb([[0, g, 0], [0, 0, 0], [0, 0, 0]])
    assert np.allclose(T[0], [0, 0, 0, g / 2, 0, 0], atol=1e-15)
    assert np.allclose(T[1], [-g * g / 2, g * g / 2, 0, 0, 0, 0], atol=1e-15)
    assert np.allclose(T[2], [g * g / 12, g * g / 12, -g * g / 6, 0, 0, 0], atol=1e-15)
    assert np.allclose(T[3], [-g * g / 12, -g * g / 12, g * g / 6, 0, 0, 0], atol=1e-15)
    assert np.allclose(T[4], 0, atol=1e-15)
    assert np.allclose(T[5], [0, 0, 0, -g ** 3 / 4, 0, 0], atol=1e-15)
    # the scale s_A divides S and R
    assert np.allclose(_tb([[0, g, 0], [0, 0, 0], [0, 0, 0]], 2.0), _tb([[0, g / 2, 0], [0, 0, 0], [0, 0, 0]]),
                       atol=1e-15)
    a, b, w = 0.8, -0.3, 1.1
    c = -a - b
    T = _tb([[a, -w, 0], [w, b, 0], [0, 0, c]])
    assert np.allclose(T[1], [0, 0, 0, w * (b - a), 0, 0], atol=1e-15)
    assert np.allclose(T[4], [0, 0, 0, w * (a * a - b * b), 0, 0], atol=1e-15)
    s6 = 2 * (a + b) / 3
    assert np.allclose(T[5], [w * w * (-2 * a + s6), w * w * (-2 * b + s6), w * w * s6, 0, 0, 0], atol=1e-15)


def test_tensor_basis_gradient_model_identity_and_equivariance():
    """-T2 + T3 - T4 is the deviatoric part of A A^T (the gradient model), and
    every basis tensor rotates with A while the invariants do not change."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((3, 3, 50))
    A -= np.einsum("ii...->...", A) / 3 * np.eye(3)[:, :, None]  # traceless
    T = les.tensor_basis(A)
    AAt = np.einsum("ik...,jk...->ij...", A, A)
    dev = AAt - np.einsum("ii...->...", AAt) / 3 * np.eye(3)[:, :, None]
    expect = np.stack([dev[i, j] for (i, j) in les.SYM])
    assert np.max(np.abs(-T[1] + T[2] - T[3] - expect)) < 1e-13
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Ar = np.einsum("ik,kl...,jl->ij...", Q, A, Q)
    Tr = les.tensor_basis(Ar)

    def full(t):
        F = np.zeros((3, 3) + t.shape[1:])
        for m, (i, j) in enumerate(les.SYM):
            F[i, j] = F[j, i] = t[m]
        return F

    for n in range(6):
        rot = np.einsum("ik,kl...,jl->ij...", Q, full(T[n]), Q)
        assert np.max(np.abs(full(Tr[n]) - rot)) < 1e-12, n
    assert np.max(np.abs(les.invariants(Ar) - les.invariants(A))) < 1e-12


def test_tensor_basis_fit_gradients_match_central_differences():
    rng = np.random.default_rng(6)
    p = les.init_params(seed=5)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    X = rng.standard_normal((29, 5))
    Bas = rng.standard_normal((29, 6, 6))
    T = rng.standard_normal((29, 6))
    _, g = les.mse_and_grads_tb(p, X, Bas, T)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = les.mse_and_grads_tb(p, X, Bas, T)
            flat[idx] = old - h
            lm, _ = les.mse_and_grads_tb(p, X, Bas, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx)
    # with the identity basis the fit is the plain fit
    eye = np.broadcast_to(np.eye(6), (29, 6, 6))
    l1, g1 = les.mse_and_grads_tb(p, X, eye, T)
    l2, g2 = les.mse_and_grads(p, X, T)
    assert abs(l1 - l2) < 1e-14 and all(np.allclose(g1[k], g2[k], rtol=1e-13, atol=1e-15) for k in p)


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.001953125, 1.0029296875, -3.14159265])
    r = les.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0  # 1 + 2^-8 is a tie: rounds to the even 1.0
    # round-to-nearest-even at the midpoint between 1 and 1 + 2^-7
    assert les.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert les.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert abs(r[4] + 3.140625) < 1e-12


def test_les_step_with_a_zero_network_is_the_plain_step():
    n = 16
    cfg = Config(n, n, n, nu=2e-2)
    u = inputs.random_solenoidal_field(n, n, n, seed=9)
    p = les.init_params(seed=4)
    p["W3"][:] = 0
    p["b3"][:] = 0
    norm = dict(mean=np.zeros(5), std=np.ones(5), s_tau=1.0, s_A=1.0)
    a = les.les_rk_step(u, 1e-2, cfg, p, norm)
    b = oracle.rk_step(u, 1e-2, cfg)
    assert np.max(np.abs(a - b)) < 1e-15
    # a nonzero network changes the step by dt times the projected closure (to first order)
    p = les.init_params(seed=4)
    norm = dict(mean=np.zeros(5), std=np.ones(5), s_tau=0.05, s_A=1.0)
    dt = 1e-6
    d = les.les_rk_step(u, dt, cfg, p, norm) - oracle.rk_step(u, dt, cfg)
    c = oracle.spectral.project(les.closure_term(u, cfg, p, norm), cfg)
    assert np.linalg.norm(d - dt * c) < 1e-3 * np.linalg.norm(dt * c)


def _force_case(seed=10, n=12):
    cfg = Config(n, n, n, lx=2 * math.pi, ly=4.0, lz=5.0)
    u = inputs.random_solenoidal_field(n, n, n, seed=seed, lx=2 * math.pi, ly=4.0, lz=5.0)
    rng = np.random.default_rng(seed)
    p = les.init_params(seed=seed)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    p["W3"] *= 5
    lam = les.invariants(les.gradient(u, cfg)).reshape(5, -1)
    norm = dict(mean=lam.mean(1), std=lam.std(1), s_tau=0.05, s_A=3.0)
    f = oracle.spectral.project(inputs.forcing_field(n, n, n, seed=3, kmax_shell=5.0, rms=0.01, lx=2 * math.pi,
                                                     ly=4.0, lz=5.0), cfg) * oracle.dealias_mask(cfg)
    return cfg, u, p, norm, f


def test_force_loss_is_the_grid_mean_of_the_residual():
    cfg, u, p, norm, f = _force_case()
    L, _ = les.force_loss_and_grads(u, cfg, p, norm, f)
    r_hat = oracle.spectral.project(les.closure_term(u, cfg, p, norm), cfg) - f
    r = oracle.spectral.inverse(r_hat, cfg)
    assert abs(L - np.mean(np.sum(r * r, axis=0))) < 1e-13 * L
    assert L > 0


def test_force_loss_gradients_match_central_differences():
    cfg, u, p, norm, f = _force_case()
    _, g = les.force_loss_and_grads(u, cfg, p, norm, f)
    rng = np.random.default_rng(12)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = les.force_loss_and_grads(u, cfg, p, norm, f)
            flat[idx] = old - h
            lm, _ = les.force_loss_and_grads(u, cfg, p, norm, f)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            scale = max(np.max(np.abs(g[name])), 1e-30)
            assert abs(fd - an) <= 1e-5 * scale, (name, idx, fd, an)


def test_transfer_spectrum_sums_to_the_energy_rate():
    """Summed over all shells, T(K) of a force is sum w Re(u* . f), the rate
    of change of the energy 1/2 sum w |u|^2 under du/dt = f (Parseval)."""
    cfg, u, p, norm, f = _force_case()
    T = les.transfer_spectrum(u, f, cfg, 64)
    r = oracle.spectral.inverse(u, cfg)
    q = oracle.spectral.inverse(f, cfg)
    assert abs(T.sum() - np.mean(np.sum(r * q, axis=0))) < 1e-13 * abs(T.sum())


def test_transfer_loss_gradients_match_central_differences():
    cfg, u, p, norm, f = _force_case()
    Te = les.transfer_spectrum(u, f, cfg, 12)
    L, g = les.transfer_loss_and_grads(u, cfg, p, norm, Te)
    assert L > 0
    rng = np.random.default_rng(13)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = les.transfer_loss_and_grads(u, cfg, p, norm, Te)
            flat[idx] = old - h
            lm, _ = les.transfer_loss_and_grads(u, cfg, p, norm, Te)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            scale = max(np.max(np.abs(g[name])), 1e-30)
            assert abs(fd - an) <= 1e-5 * scale, (name, idx, fd, an)
