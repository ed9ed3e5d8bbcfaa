"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here runs on the CPU.  None re-types an oracle formula: each checks
it against a different route (a direct O(N^6) sum, exact rational Fourier
arithmetic in advective form, closed-form flows, conservation laws, brute-force
convolution, convergence order, or a third-party FFT)."""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.spectral import CUBIC, NONE, SPHERICAL, Config, mode_indices
from paper_1808_01309_gb300 import inputs

from . import exact_fourier as xf

TWO_PI = 2.0 * math.pi


def grid(cfg):
    z = np.arange(cfg.nz) * cfg.lz / cfg.nz
    y = np.arange(cfg.ny) * cfg.ly / cfg.ny
    x = np.arange(cfg.nx) * cfg.lx / cfg.nx
    return np.meshgrid(z, y, x, indexing="ij")  # Z, Y, X with shape (nz, ny, nx)


def relerr(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# --------------------------------------------------------------------------
# Transform (Eq. fftsum, readings R1-R3)
# --------------------------------------------------------------------------

def _dft_kernel(nz, ny, nx, sign):
    """exp(sign 2 pi i (p i/nx + q j/ny + r k/nz)) as a dense 6-index tensor
    [r, q, p, k, j, i] over the full index ranges."""
    r = np.arange(nz).reshape(-1, 1, 1, 1, 1, 1)
    q = np.arange(ny).reshape(1, -1, 1, 1, 1, 1)
    p = np.arange(nx).reshape(1, 1, -1, 1, 1, 1)
    k = np.arange(nz).reshape(1, 1, 1, -1, 1, 1)
    j = np.arange(ny).reshape(1, 1, 1, 1, -1, 1)
    i = np.arange(nx).reshape(1, 1, 1, 1, 1, -1)
    return np.exp(sign * 2j * math.pi * (p * i / nx + q * j / ny + r * k / nz))


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 6, 6), (10, 6, 8), (4, 12, 10)])
def test_forward_is_the_direct_sum(shape):
    nz, ny, nx = shape
    u = inputs.random_real_field((3, nz, ny, nx), seed=11)
    ker = _dft_kernel(nz, ny, nx, -1.0)
    direct = np.einsum("rqpkji,ckji->crqp", ker, u) / (nx * ny * nz)
    got = oracle.forward(u)
    assert got.shape == (3, nz, ny, nx // 2 + 1)
    assert relerr(got, direct[..., : nx // 2 + 1]) < 1e-14


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 12)])
def test_inverse_is_the_unnormalised_direct_sum(shape):
    nz, ny, nx = shape
    cfg = Config(nx, ny, nz)
    u = inputs.random_real_field((3, nz, ny, nx), seed=12)
    full = np.einsum("rqpkji,ckji->crqp", _dft_kernel(nz, ny, nx, -1.0), u) / (nx * ny * nz)
    # backward sum over the FULL spectrum, then compare with the oracle fed the half spectrum
    back = np.einsum("rqpkji,crqp->ckji", _dft_kernel(nz, ny, nx, +1.0), full)
    assert np.max(np.abs(back.imag)) < 1e-12
    got = oracle.inverse(full[..., : nx // 2 + 1], cfg)
    assert relerr(got, back.real) < 1e-14
    assert relerr(got, u) < 1e-14


def test_parseval_with_hermitian_weights():
    cfg = Config(16, 8, 12)
    u = inputs.random_real_field((3, cfg.nz, cfg.ny, cfg.nx), seed=3)
    uh = oracle.forward(u)
    w = oracle.hermitian_weight(cfg)
    lhs = np.mean(np.sum(u * u, axis=0))
    rhs = np.sum(w * np.sum(np.abs(uh) ** 2, axis=0))
    assert abs(lhs - rhs) / lhs < 1e-14


def test_third_party_fft_agrees():
    torch = pytest.importorskip("torch")
    cfg = Config(32, 32, 32)
    u = inputs.random_real_field((3, 32, 32, 32), seed=5)
    ref = torch.fft.rfftn(torch.from_numpy(u), dim=(-3, -2, -1), norm="forward").numpy()
    assert relerr(oracle.forward(u), ref) < 1e-14
    assert relerr(oracle.inverse(ref, cfg), u) < 1e-14


# --------------------------------------------------------------------------
# Mask (reading R4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,k", [(32, 10), (64, 21), (96, 31), (128, 42), (256, 85),
                                 (512, 170), (1024, 341), (12, 3), (8, 2)])
def test_two_thirds_halfwidth(n, k):
    assert oracle.retained_halfwidth(n, CUBIC) == k
    # alias-free (a product of two kept modes cannot fold back onto a kept mode)
    # and maximal
    assert 3 * k < n and 3 * (k + 1) >= n
    assert oracle.retained_halfwidth(n, NONE) == n // 2 - 1


def test_spherical_mask_is_inside_cube():
    cfg = Config(32, 32, 32, dealias=SPHERICAL)
    p, q, r = mode_indices(cfg)
    m = oracle.dealias_mask(cfg)
    rho2 = (p * p + q * q + r * r) + 0 * m
    assert np.all(rho2[m] < (32 / 3) ** 2)
    assert np.all(~m[rho2 >= (32 / 3) ** 2])
    assert m.sum() < oracle.dealias_mask(Config(32, 32, 32)).sum()


# --------------------------------------------------------------------------
# Curl, nonlinear term, projection
# --------------------------------------------------------------------------

def test_curl_of_taylor_green_is_analytic():
    cfg = Config(16, 16, 16)
    Z, Y, X = grid(cfg)
    om = oracle.inverse(oracle.curl_hat(inputs.taylor_green(16, 16, 16), cfg), cfg)
    expect = np.stack([-np.cos(X) * np.sin(Y) * np.sin(Z),
                       -np.sin(X) * np.cos(Y) * np.sin(Z),
                       2.0 * np.sin(X) * np.sin(Y) * np.cos(Z)])
    assert np.max(np.abs(om - expect)) < 1e-14


@pytest.mark.parametrize("lx,ly,lz", [(TWO_PI, TWO_PI, TWO_PI), (4.0, 9.0, 2.5)])
def test_rhs_of_crossed_shear_is_closed_form(lx, ly, lz):
    """u = (sin(a y), 0, sin(b x)): (u.grad)u = (0, 0, b sin(a y) cos(b x)) is
    solenoidal, so the projected rotational term is its negative; the viscous
    term is nu Laplacian u."""
    nu = 0.03
    cfg = Config(16, 8, 12, lx=lx, ly=ly, lz=lz, nu=nu)
    a, b = TWO_PI / ly, TWO_PI / lx
    Z, Y, X = grid(cfg)
    uh = inputs.crossed_shear(16, 8, 12)
    got = oracle.inverse(oracle.rhs(uh, cfg), cfg)
    expect = np.stack([-nu * a * a * np.sin(a * Y),
                       0.0 * X,
                       -b * np.sin(a * Y) * np.cos(b * X) - nu * b * b * np.sin(b * X)])
    assert np.max(np.abs(got - expect)) < 1e-13


def _full_spectrum(uh, cfg):
    """dict (p,q,r) -> complex 3-vector for every mode of the full spectrum."""
    nz, ny, nx = cfg.nz, cfg.ny, cfg.nx
    out = {}
    for r in range(nz):
        for q in range(ny):
            for p in range(nx // 2 + 1):
                v = uh[:, r, q, p]
                if not np.any(v):
                    continue
                rs = r if r < (nz + 1) // 2 else r - nz
                qs = q if q < (ny + 1) // 2 else q - ny
                out[(p, qs, rs)] = v
                if 0 < p < nx - p:
                    out[(-p, -qs, -rs)] = np.conj(v)
    return out


def _halfwidth(n):
    k = 0
    while 3 * (k + 1) < n:
        k += 1
    return k


@pytest.mark.parametrize("n3", [(8, 8, 8), (12, 12, 12), (8, 12, 16)])
def test_rhs_equals_bruteforce_truncated_convolution(n3):
    """-D P[(u.grad)u] summed pair by pair over the kept modes, with the kept
    set recomputed here from 3K < N, equals the oracle's pseudospectral,
    dealiased rotational-form term."""
    nx, ny, nz = n3
    cfg = Config(nx, ny, nz, lx=TWO_PI, ly=3.0, lz=5.0)
    uh = inputs.random_solenoidal_field(nx, ny, nz, seed=21, kmax=(nx, ny, nz))
    Kx, Ky, Kz = _halfwidth(nx), _halfwidth(ny), _halfwidth(nz)
    sx, sy, sz = TWO_PI / cfg.lx, TWO_PI / cfg.ly, TWO_PI / cfg.lz

    def kept(m):
        return abs(m[0]) <= Kx and abs(m[1]) <= Ky and abs(m[2]) <= Kz

    full = {m: v for m, v in _full_spectrum(uh, cfg).items() if kept(m)}
    keys = list(full)
    K = np.array(keys, dtype=np.float64) * np.array([sx, sy, sz])
    U = np.array([full[m] for m in keys])
    # (u.grad)u at mode p+q: (u(p) . i k(q)) u(q)
    coef = 1j * (U @ K.T)                         # [p, q] = u(p) . k(q)
    sums = {}
    for a, pa in enumerate(keys):
        for b, qb in enumerate(keys):
            m = (pa[0] + qb[0], pa[1] + qb[1], pa[2] + qb[2])
            if m[0] < 0 or not kept(m):
                continue
            sums[m] = sums.get(m, 0.0) + coef[a, b] * U[b]
    expect = np.zeros_like(uh)
    for m, v in sums.items():
        k = np.array(m, dtype=np.float64) * np.array([sx, sy, sz])
        k2 = k @ k
        if k2 == 0:
            continue
        v = -(v - k * (k @ v) / k2)
        expect[:, m[2] % nz, m[1] % ny, m[0]] = v
    got = oracle.rhs(uh, cfg)
    assert relerr(got, expect) < 1e-13


def test_projected_rhs_is_divergence_free_with_zero_mean():
    cfg = Config(32, 16, 24, lx=3.0, ly=TWO_PI, lz=7.0, nu=1e-2)
    uh = inputs.random_solenoidal_field(32, 16, 24, seed=4, lx=3.0, lz=7.0)
    f = inputs.forcing_field(32, 16, 24, seed=5, lx=3.0, lz=7.0)
    out = oracle.rhs(uh, cfg, forcing=f)
    kx, ky, kz = oracle.wavenumbers(cfg)
    div = kx * out[0] + ky * out[1] + kz * out[2]
    assert np.max(np.abs(div)) <= 1e-14 * np.max(np.abs(out)) * np.max(np.abs(kz))
    assert np.all(out[:, 0, 0, 0] == 0)
    assert np.all(out[:, ~oracle.dealias_mask(cfg)] == 0)


def test_nonlinear_transfer_conserves_energy_and_helicity():
    """u.(u x w) = 0 and w.(u x w) = 0 pointwise, so with Parseval the
    projected, dealiased term transfers no energy and no helicity."""
    cfg = Config(32, 32, 32)
    uh = inputs.random_solenoidal_field(32, 32, 32, seed=9)
    nl = oracle.rhs(uh, cfg)
    w = oracle.hermitian_weight(cfg)
    om = oracle.curl_hat(uh, cfg)
    de = np.sum(w * np.real(np.sum(np.conj(uh) * nl, axis=0)))
    dh = np.sum(w * np.real(np.sum(np.conj(om) * nl, axis=0)))
    scale_e = np.sum(w * np.abs(uh).sum(0) * np.abs(nl).sum(0))
    scale_h = np.sum(w * np.abs(om).sum(0) * np.abs(nl).sum(0))
    assert abs(de) < 1e-14 * scale_e
    assert abs(dh) < 1e-14 * scale_h


def test_hermitian_output_plane():
    cfg = Config(16, 16, 16)
    out = oracle.rhs(inputs.random_solenoidal_field(16, 16, 16, seed=8), cfg)
    plane = out[:, :, :, 0]
    r = (-np.arange(16)) % 16
    mirror = np.conj(plane[:, r][:, :, r])
    assert np.max(np.abs(plane - mirror)) < 1e-15 * np.max(np.abs(out)) + 1e-300


# --------------------------------------------------------------------------
# Exact rational Taylor coefficients of the Taylor-Green vortex
# --------------------------------------------------------------------------

TG_TERMS = [(0, 1, ("s", 1), ("c", 1), ("c", 1)), (1, -1, ("c", 1), ("s", 1), ("c", 1))]


def test_taylor_green_tendency_matches_exact_rational_advection():
    u0 = xf.trig_modes(TG_TERMS)
    ut = xf.euler_rate(u0)
    cfg = Config(16, 16, 16)
    got = oracle.rhs(inputs.taylor_green(16, 16, 16), cfg)
    expect = np.zeros_like(got)
    for (p, q, r), v in ut.items():
        if p >= 0:
            expect[:, r % 16, q % 16, p] = [complex(c) for c in v]
    assert np.max(np.abs(expect)) > 0.03
    assert np.max(np.abs(got - expect)) < 1e-15


def test_taylor_green_initial_invariants_and_enstrophy_growth():
    u0 = xf.trig_modes(TG_TERMS)
    w0 = xf.curl(u0)
    E0 = xf.inner(u0, u0) / 2
    W0 = xf.inner(w0, w0) / 2
    assert (E0, W0) == (Fraction(1, 8), Fraction(3, 8))
    ut = xf.euler_rate(u0)
    utt = xf.scale(xf.project(xf.add(xf.advect(ut, u0), xf.advect(u0, ut))), -1)
    wt, wtt = xf.curl(ut), xf.curl(utt)
    assert xf.inner(w0, wt) == 0                    # no vortex stretching at t = 0
    c2 = (xf.inner(wt, wt) + xf.inner(w0, wtt)) / (2 * W0)   # Omega/Omega0 = 1 + c2 t^2
    assert c2 == Fraction(5, 48)

    cfg = Config(32, 32, 32, nu=0.0, rk_order=4)
    uh = inputs.taylor_green(32, 32, 32)
    d0 = oracle.diagnostics(uh, cfg)
    assert abs(d0["energy"] - 0.125) < 1e-15 and abs(d0["enstrophy"] - 0.375) < 1e-15

    def f_of(t_end, dt=1e-3):
        u = uh.copy()
        for _ in range(int(round(t_end / dt))):
            u = oracle.rk_step(u, dt, cfg)
        W = oracle.diagnostics(u, cfg)["enstrophy"]
        return (W / 0.375 - 1.0) / t_end ** 2

    f1, f2 = f_of(0.02), f_of(0.04)
    c2_num = (4.0 * f1 - f2) / 3.0           # Richardson: removes the t^2 term of f
    assert abs(c2_num - 5.0 / 48.0) < 1e-6


# --------------------------------------------------------------------------
# Closed-form time evolutions (reading R8)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("order", [2, 4])
def test_abc_flow_decays_exactly(order):
    """Beltrami: w = u so u x w = 0 and each mode decays as exp(-nu |k|^2 t);
    a Lawson step is exact for it at any dt."""
    nu, dt = 0.05, 0.1
    cfg = Config(16, 16, 16, nu=nu, rk_order=order)
    uh = inputs.abc_flow(16, 16, 16)
    assert np.max(np.abs(oracle.curl_hat(uh, cfg) - uh)) < 1e-15
    d = oracle.diagnostics(uh, cfg)
    assert abs(d["energy"] - 1.5) < 1e-14 and abs(d["helicity"] - 3.0) < 1e-14
    assert np.max(np.abs(oracle.rhs(uh, Config(16, 16, 16)))) < 1e-15
    u = uh
    for _ in range(5):
        u = oracle.rk_step(u, dt, cfg)
    assert np.max(np.abs(u - uh * math.exp(-nu * 5 * dt))) < 1e-15


def test_kolmogorov_shear_decays_exactly():
    nu, dt = 0.02, 0.25
    cfg = Config(16, 16, 16, nu=nu, rk_order=4)
    uh = inputs.kolmogorov_flow(16, 16, 16)
    u = uh
    for _ in range(4):
        u = oracle.rk_step(u, dt, cfg)
    assert np.max(np.abs(u - uh * math.exp(-nu * 1.0))) < 1e-15


@pytest.mark.parametrize("order", [2, 4])
def test_linear_forced_response(order):
    """u0 = 0, nonlinear term off: u_hat(t) = f (1 - exp(-nu k^2 t))/(nu k^2)."""
    nu, dt, steps = 0.01, 0.01, 20
    cfg = Config(16, 16, 16, nu=nu, rk_order=order)
    f = inputs.forcing_field(16, 16, 16, seed=2)
    u = np.zeros_like(f)
    for _ in range(steps):
        u = oracle.rk_step(u, dt, cfg, forcing=f, nonlinear_on=False)
    kx, ky, kz = oracle.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    t = steps * dt
    with np.errstate(divide="ignore", invalid="ignore"):
        expect = np.where(k2 > 0, f * (1 - np.exp(-nu * k2 * t)) / (nu * k2), 0)
    tol = 1e-12 if order == 4 else 1e-7
    assert relerr(u, expect) < tol


@pytest.mark.parametrize("order,rate", [(4, 16.0), (2, 4.0)])
def test_runge_kutta_order(order, rate):
    # nu is large enough that a misplaced integrating factor lowers the order
    cfg = Config(16, 16, 16, nu=0.2, rk_order=order)
    uh = inputs.random_solenoidal_field(16, 16, 16, seed=31) * 4.0
    T = 0.2

    def run(dt):
        u = uh
        for _ in range(int(round(T / dt))):
            u = oracle.rk_step(u, dt, cfg)
        return u

    ref = run(T / 64)
    e1 = np.linalg.norm(run(T / 4) - ref)
    e2 = np.linalg.norm(run(T / 8) - ref)
    assert 0.85 * rate < e1 / e2 < 1.2 * rate


def test_inviscid_energy_drift_is_at_the_scheme_order():
    """For an energy-conserving system the RK4 amplification factor satisfies
    |R(iy)|^2 = 1 - y^6/72 + y^8/576, so the energy error after a fixed time
    is O(dt^5): halving dt divides the drift by about 32."""
    cfg = Config(16, 16, 16, nu=0.0, rk_order=4)
    uh = inputs.random_solenoidal_field(16, 16, 16, seed=41) * 4.0
    E0 = oracle.diagnostics(uh, cfg)["energy"]

    def drift(dt):
        u = uh
        for _ in range(int(round(0.2 / dt))):
            u = oracle.rk_step(u, dt, cfg)
        return abs(oracle.diagnostics(u, cfg)["energy"] - E0)

    d1, d2 = drift(0.025), drift(0.0125)
    assert d1 < 1e-4 * E0
    assert 24.0 < d1 / d2 < 40.0


# --------------------------------------------------------------------------
# Diagnostics (reading R9) and the synthetic inputs
# --------------------------------------------------------------------------

def test_diagnostics_match_physical_space():
    cfg = Config(24, 16, 32, lx=5.0, ly=TWO_PI, lz=3.0)
    uh = inputs.random_solenoidal_field(24, 16, 32, seed=13, lx=5.0, lz=3.0)
    d = oracle.diagnostics(uh, cfg, cfl=0.7)
    u = oracle.inverse(uh, cfg)
    w = oracle.inverse(oracle.curl_hat(uh, cfg), cfg)
    assert abs(d["energy"] - 0.5 * np.mean(np.sum(u * u, 0))) < 1e-14
    assert abs(d["enstrophy"] - 0.5 * np.mean(np.sum(w * w, 0))) < 1e-12 * d["enstrophy"]
    assert abs(d["helicity"] - np.mean(np.sum(u * w, 0))) < 1e-12 * d["enstrophy"]
    assert abs(np.sum(d["spectrum"]) - d["energy"]) < 1e-14
    umax = np.sqrt(np.max(np.sum(u * u, 0)))
    assert abs(d["max_u"] - umax) < 1e-15
    assert abs(d["cfl_dt"] - 0.7 * min(5.0 / 24, TWO_PI / 16, 3.0 / 32) / umax) < 1e-15
    assert d["max_div"] < 1e-13


def test_shell_spectrum_of_closed_form_fields():
    """Shells K = floor(|k| + 1/2): the Taylor-Green modes (|k| = sqrt 3) put
    their energy 1/8 in shell 2, u = (0, 0, sin 2x cos 2y) (|k| = sqrt 8) its
    1/8 in shell 3, the ABC flow (|k| = 1) its 3/2 in shell 1; on a box of
    length 4 pi along x, sin(2 * 2 pi x / Lx) = sin x sits in shell 1."""
    n = 16
    cfg = Config(n, n, n)
    cases = [(inputs.taylor_green(n, n, n), 2, 0.125),
             (inputs.trig_field(n, n, n, [(2, 1.0, ("s", 2), ("c", 2), ("1", 0))]), 3, 0.125),
             (inputs.abc_flow(n, n, n), 1, 1.5)]
    for uh, shell, e in cases:
        sp = oracle.diagnostics(uh, cfg)["spectrum"]
        assert abs(sp[shell] - e) < 1e-15
        assert np.sum(np.abs(np.delete(sp, shell))) < 1e-15
    box = Config(n, n, n, lx=2 * TWO_PI)
    uh = inputs.trig_field(n, n, n, [(2, 1.0, ("s", 2), ("1", 0), ("1", 0))])
    sp = oracle.diagnostics(uh, box)["spectrum"]
    assert abs(sp[1] - 0.25) < 1e-15 and np.sum(np.abs(np.delete(sp, 1))) < 1e-15


def test_taylor_green_cfl_closed_form():
    cfg = Config(32, 32, 32)
    d = oracle.diagnostics(inputs.taylor_green(32, 32, 32), cfg, cfl=0.5)
    assert abs(d["max_u"] - 1.0) < 1e-15
    assert abs(d["cfl_dt"] - 0.5 * TWO_PI / 32) < 1e-15


def test_random_field_properties():
    n = 32
    cfg = Config(n, n, n)
    uh = inputs.random_solenoidal_field(n, n, n, seed=1)
    d = oracle.diagnostics(uh, cfg)
    assert abs(d["energy"] - 0.5) < 1e-14
    assert d["max_div"] < 1e-14
    # Hermitian kx = 0 plane, zero mean
    r = (-np.arange(n)) % n
    plane = uh[:, :, :, 0]
    assert np.max(np.abs(plane - np.conj(plane[:, r][:, :, r]))) == 0.0
    assert np.all(uh[:, 0, 0, 0] == 0)
    # spectrum shape K^4 exp(-2 (K/4)^2) on the shells inside the cube
    K = np.arange(1, 10)
    target = K ** 4.0 * np.exp(-2.0 * (K / 4.0) ** 2)
    ratio = d["spectrum"][1:10] / target
    assert np.max(ratio) / np.min(ratio) - 1.0 < 1e-12
    # seeded: same bytes every call, and the low modes do not depend on the grid
    assert np.array_equal(uh, inputs.random_solenoidal_field(n, n, n, seed=1))


def test_forcing_properties():
    n = 32
    cfg = Config(n, n, n)
    f = inputs.forcing_field(n, n, n, seed=2)
    w = oracle.hermitian_weight(cfg)
    kx, ky, kz = oracle.wavenumbers(cfg)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz) + 0 * f[0].real
    mod = np.sqrt(np.sum(np.abs(f) ** 2, 0))
    on = mod > 0
    assert np.all((kk[on] >= 2 - 1e-12) & (kk[on] <= 3 + 1e-12))
    assert np.max(mod[on]) / np.min(mod[on]) - 1 < 1e-12
    assert abs(math.sqrt(np.sum(w * mod ** 2)) - 0.25) < 1e-15
    assert np.max(np.abs(kx * f[0] + ky * f[1] + kz * f[2])) < 1e-15
    fphys = oracle.inverse(f, cfg)
    assert abs(math.sqrt(np.mean(np.sum(fphys ** 2, 0))) - 0.25) < 1e-15
