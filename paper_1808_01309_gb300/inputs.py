"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no step of the method (no transform, product, projection or
time step): it only synthesises spectral fields in the state layout
(3, nz, ny, nx//2+1), complex128, kx fastest, ky/kz in FFT order, so that the
same bytes can be fed to the FP64 oracle and to the CUDA path.

Random numbers come from a counter-based generator keyed by the signed mode
index (p, q, r), the component and the seed, so a mode's draw does not depend
on the grid size or on the order in which modes are visited:

  splitmix64(x):  z = x + 0x9E3779B97F4A7C15
                  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
                  z = (z ^ (z >> 27)) * 0x94D049BB133111EB
                  return z ^ (z >> 31)             (all mod 2^64)
  key  = splitmix64(splitmix64(splitmix64(seed) ^ enc(p, q, r)) ^ (2*comp + j))
  enc  = ((p + 2^20) << 42) | ((q + 2^20) << 21) | (r + 2^20)
  unif = ((key >> 11) + 1) * 2^-53          in (0, 1]
  a complex normal deviate per (mode, comp): Box-Muller on the uniforms of
  j = 0 and j = 1.
"""

from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def _uniform(seed: int, p, q, r, stream: int) -> np.ndarray:
    off = np.int64(1 << 20)
    enc = (((np.asarray(p, np.int64) + off) << np.int64(42))
           | ((np.asarray(q, np.int64) + off) << np.int64(21))
           | (np.asarray(r, np.int64) + off)).astype(np.uint64)
    s = _splitmix64(np.array([seed], dtype=np.uint64))[0]
    k = _splitmix64(_splitmix64(s ^ enc) ^ np.uint64(stream))
    return ((k >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53


def complex_normal(seed: int, p, q, r, comp: int) -> np.ndarray:
    """One standard complex normal deviate per mode (Box-Muller)."""
    u1 = _uniform(seed, p, q, r, 2 * comp)
    u2 = _uniform(seed, p, q, r, 2 * comp + 1)
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2.0 * math.pi * u2) + 1j * rad * np.sin(2.0 * math.pi * u2)


def cube_halfwidth(n: int) -> int:
    """Largest |index| strictly below n/3 (the 2/3-rule cube), ceil(n/3) - 1."""
    return -(-n // 3) - 1


def _signed(n: int) -> np.ndarray:
    i = np.arange(n)
    return np.where(i < (n + 1) // 2, i, i - n)


def _cube_indices(nx, ny, nz, kmax):
    """Storage indices and signed indices of the modes with |p|<=Kx, |q|<=Ky,
    |r|<=Kz, p >= 0, excluding Nyquist rows."""
    kx, ky, kz = kmax
    kx = min(kx, nx // 2 - 1)
    ky = min(ky, ny // 2 - 1)
    kz = min(kz, nz // 2 - 1)
    p = np.arange(0, kx + 1)
    q = np.concatenate([np.arange(0, ky + 1), np.arange(-ky, 0)])
    r = np.concatenate([np.arange(0, kz + 1), np.arange(-kz, 0)])
    iq = np.where(q >= 0, q, q + ny)
    ir = np.where(r >= 0, r, r + nz)
    return p, q, r, iq, ir


def _hermitian_kx0(f: np.ndarray) -> None:
    """Make the kx = 0 plane Hermitian in (ky, kz): f(0,-q,-r) = conj f(0,q,r),
    keeping the half with r > 0 or (r == 0 and q > 0); the mean is zeroed."""
    nz, ny = f.shape[1], f.shape[2]
    q = _signed(ny).reshape(1, -1)
    r = _signed(nz).reshape(-1, 1)
    neg = (r < 0) | ((r == 0) & (q < 0))
    src_r = (-r) % nz
    src_q = (-q) % ny
    plane = f[:, :, :, 0].copy()
    mirrored = np.conj(plane[:, src_r, src_q])
    plane = np.where(neg[None], mirrored, plane)
    plane[:, 0, 0] = 0.0
    f[:, :, :, 0] = plane


def _kvec(p, q, r, lx, ly, lz):
    return (2.0 * math.pi / lx) * p, (2.0 * math.pi / ly) * q, (2.0 * math.pi / lz) * r


def random_solenoidal_field(nx, ny, nz, seed=1, kmax=None, lx=2 * math.pi,
                            ly=2 * math.pi, lz=2 * math.pi, energy=0.5, k_peak=4.0):
    """Random divergence-free velocity with shell spectrum
    E(K) proportional to K^4 exp(-2 (K/k_peak)^2), total energy `energy`.

    Each stored mode inside the cube |p|<=Kx, |q|<=Ky, |r|<=Kz gets
    u_hat = (k x a)/|k| with a a seeded complex normal 3-vector (so k.u_hat = 0),
    the kx = 0 plane is made Hermitian, each shell K = floor(|k| + 1/2) is
    rescaled to the target shape and the whole field to the requested energy
    (energy = 1/2 sum w |u_hat|^2, w = 1 on kx = 0, else 2).
    """
    if kmax is None:
        kmax = (cube_halfwidth(nx), cube_halfwidth(ny), cube_halfwidth(nz))
    nh = nx // 2 + 1
    p, q, r, iq, ir = _cube_indices(nx, ny, nz, kmax)
    P, Q, R = np.meshgrid(p, q, r, indexing="ij")          # (cx, cy, cz)
    P, Q, R = P.transpose(2, 1, 0), Q.transpose(2, 1, 0), R.transpose(2, 1, 0)  # (cz, cy, cx)
    a = [complex_normal(seed, P, Q, R, c) for c in range(3)]
    kx, ky, kz = _kvec(P, Q, R, lx, ly, lz)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    kk_safe = np.where(kk > 0, kk, 1.0)
    ux = (ky * a[2] - kz * a[1]) / kk_safe
    uy = (kz * a[0] - kx * a[2]) / kk_safe
    uz = (kx * a[1] - ky * a[0]) / kk_safe
    f = np.zeros((3, nz, ny, nh), dtype=np.complex128)
    sel = np.ix_(ir, iq, p)
    for c, v in enumerate((ux, uy, uz)):
        f[c][sel] = np.where(kk > 0, v, 0.0)
    _hermitian_kx0(f)
    # shell rescaling
    Pf = np.arange(nh).reshape(1, 1, -1)
    Qf = _signed(ny).reshape(1, -1, 1)
    Rf = _signed(nz).reshape(-1, 1, 1)
    kxf, kyf, kzf = _kvec(Pf, Qf, Rf, lx, ly, lz)
    kmag = np.sqrt(kxf ** 2 + kyf ** 2 + kzf ** 2) + np.zeros((nz, ny, nh))
    shell = np.floor(kmag + 0.5).astype(np.int64)
    w = np.full(nh, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[-1] = 1.0
    e_mode = 0.5 * w.reshape(1, 1, -1) * np.sum(np.abs(f) ** 2, axis=0)
    ns = int(shell.max()) + 1
    e_shell = np.bincount(shell.ravel(), weights=e_mode.ravel(), minlength=ns)
    K = np.arange(ns, dtype=np.float64)
    target = K ** 4 * np.exp(-2.0 * (K / k_peak) ** 2)
    scale = np.where(e_shell > 0, np.sqrt(target / np.where(e_shell > 0, e_shell, 1.0)), 0.0)
    f *= scale[shell][None]
    e_tot = float(np.sum(0.5 * w.reshape(1, 1, -1) * np.sum(np.abs(f) ** 2, axis=0)))
    if e_tot > 0:
        f *= math.sqrt(energy / e_tot)
    return f


def random_scalar_field(nx, ny, nz, seed=61, kmax=None, lx=2 * math.pi,
                        ly=2 * math.pi, lz=2 * math.pi, variance=0.5, k_peak=4.0):
    """Random real scalar (Boussinesq temperature) of shape (1, nz, ny, nx/2+1)
    with shell spectrum proportional to K^4 exp(-2 (K/k_peak)^2) and
    1/2 sum w |theta_hat|^2 = variance: a seeded complex normal per stored
    mode of the cube (stream component 3), Hermitian kx = 0 plane, per-shell
    rescaling as for the velocity."""
    if kmax is None:
        kmax = (cube_halfwidth(nx), cube_halfwidth(ny), cube_halfwidth(nz))
    nh = nx // 2 + 1
    p, q, r, iq, ir = _cube_indices(nx, ny, nz, kmax)
    P, Q, R = np.meshgrid(p, q, r, indexing="ij")
    P, Q, R = P.transpose(2, 1, 0), Q.transpose(2, 1, 0), R.transpose(2, 1, 0)
    a = complex_normal(seed, P, Q, R, 3)
    f = np.zeros((1, nz, ny, nh), dtype=np.complex128)
    f[0][np.ix_(ir, iq, p)] = np.where((P == 0) & (Q == 0) & (R == 0), 0.0, a)
    _hermitian_kx0(f)
    Pf = np.arange(nh).reshape(1, 1, -1)
    Qf = _signed(ny).reshape(1, -1, 1)
    Rf = _signed(nz).reshape(-1, 1, 1)
    kxf, kyf, kzf = _kvec(Pf, Qf, Rf, lx, ly, lz)
    kmag = np.sqrt(kxf ** 2 + kyf ** 2 + kzf ** 2) + np.zeros((nz, ny, nh))
    shell = np.floor(kmag + 0.5).astype(np.int64)
    w = np.full(nh, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[-1] = 1.0
    e_mode = 0.5 * w.reshape(1, 1, -1) * np.abs(f[0]) ** 2
    ns = int(shell.max()) + 1
    e_shell = np.bincount(shell.ravel(), weights=e_mode.ravel(), minlength=ns)
    K = np.arange(ns, dtype=np.float64)
    target = K ** 4 * np.exp(-2.0 * (K / k_peak) ** 2)
    scale = np.where(e_shell > 0, np.sqrt(target / np.where(e_shell > 0, e_shell, 1.0)), 0.0)
    f *= scale[shell][None]
    e_tot = float(np.sum(0.5 * w.reshape(1, 1, -1) * np.abs(f[0]) ** 2))
    if e_tot > 0:
        f *= math.sqrt(variance / e_tot)
    return f


def forcing_field(nx, ny, nz, seed=2, kmin=2.0, kmax_shell=3.0, rms=0.25, kmax=None,
                  lx=2 * math.pi, ly=2 * math.pi, lz=2 * math.pi):
    """Constant-in-time solenoidal forcing on kmin <= |k| <= kmax_shell: every
    forced mode has the same modulus |f_hat| and a seeded random direction and
    phase, the kx = 0 plane is Hermitian and the field is scaled so that the
    physical rms <|f|^2>^(1/2) = sqrt(sum w |f_hat|^2) equals `rms`."""
    if kmax is None:
        kmax = (cube_halfwidth(nx), cube_halfwidth(ny), cube_halfwidth(nz))
    nh = nx // 2 + 1
    p, q, r, iq, ir = _cube_indices(nx, ny, nz, kmax)
    P, Q, R = np.meshgrid(p, q, r, indexing="ij")
    P, Q, R = P.transpose(2, 1, 0), Q.transpose(2, 1, 0), R.transpose(2, 1, 0)
    a = [complex_normal(seed, P, Q, R, c) for c in range(3)]
    kx, ky, kz = _kvec(P, Q, R, lx, ly, lz)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    band = (kk >= kmin - 1e-12) & (kk <= kmax_shell + 1e-12)
    kk_safe = np.where(kk > 0, kk, 1.0)
    v = [(ky * a[2] - kz * a[1]) / kk_safe, (kz * a[0] - kx * a[2]) / kk_safe,
         (kx * a[1] - ky * a[0]) / kk_safe]
    norm = np.sqrt(sum(np.abs(x) ** 2 for x in v))
    norm = np.where(norm > 0, norm, 1.0)
    f = np.zeros((3, nz, ny, nh), dtype=np.complex128)
    sel = np.ix_(ir, iq, p)
    for c in range(3):
        f[c][sel] = np.where(band, v[c] / norm, 0.0)
    _hermitian_kx0(f)
    w = np.full(nh, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[-1] = 1.0
    ms = float(np.sum(w.reshape(1, 1, -1) * np.sum(np.abs(f) ** 2, axis=0)))
    if ms > 0:
        f *= rms / math.sqrt(ms)
    return f


def _axis_terms(kind: str, m: int):
    """Fourier expansion of cos(m t), sin(m t) or 1 as (index, coefficient)."""
    if kind == "1" or m == 0:
        return [(0, 1.0 + 0j)] if kind != "s" else []
    if kind == "c":
        return [(m, 0.5 + 0j), (-m, 0.5 + 0j)]
    if kind == "s":
        return [(m, -0.5j), (-m, 0.5j)]
    raise ValueError(kind)


def trig_field(nx, ny, nz, terms):
    """Exact spectral coefficients of a real field given as a sum of products
    of trigonometric functions of the box's fundamental wavenumbers.

    `terms` is a list of (component, amplitude, (kind_x, mx), (kind_y, my),
    (kind_z, mz)) with kind in {"c", "s", "1"}: the term amplitude *
    f_x(mx 2 pi x/Lx) f_y(my 2 pi y/Ly) f_z(mz 2 pi z/Lz)."""
    nh = nx // 2 + 1
    f = np.zeros((3, nz, ny, nh), dtype=np.complex128)
    for comp, amp, (kx_, mx), (ky_, my), (kz_, mz) in terms:
        for p, cx in _axis_terms(kx_, mx):
            if p < 0:
                continue
            for q, cy in _axis_terms(ky_, my):
                for r, cz in _axis_terms(kz_, mz):
                    f[comp, r % nz, q % ny, p] += amp * cx * cy * cz
    return f


def taylor_green(nx, ny, nz):
    """u = (sin x cos y cos z, -cos x sin y cos z, 0)."""
    return trig_field(nx, ny, nz, [
        (0, 1.0, ("s", 1), ("c", 1), ("c", 1)),
        (1, -1.0, ("c", 1), ("s", 1), ("c", 1)),
    ])


def abc_flow(nx, ny, nz, A=1.0, B=1.0, C=1.0):
    """Arnold-Beltrami-Childress flow
    u = (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x)."""
    return trig_field(nx, ny, nz, [
        (0, A, ("1", 0), ("1", 0), ("s", 1)), (0, C, ("1", 0), ("c", 1), ("1", 0)),
        (1, B, ("s", 1), ("1", 0), ("1", 0)), (1, A, ("1", 0), ("1", 0), ("c", 1)),
        (2, C, ("1", 0), ("s", 1), ("1", 0)), (2, B, ("c", 1), ("1", 0), ("1", 0)),
    ])


def kolmogorov_flow(nx, ny, nz):
    """Shear u = (sin y, 0, 0)."""
    return trig_field(nx, ny, nz, [(0, 1.0, ("1", 0), ("s", 1), ("1", 0))])


def crossed_shear(nx, ny, nz):
    """u = (sin y, 0, sin x): a solenoidal field whose advection
    (u . grad) u = (0, 0, b sin(a y) cos(b x)) is itself solenoidal."""
    return trig_field(nx, ny, nz, [
        (0, 1.0, ("1", 0), ("s", 1), ("1", 0)),
        (2, 1.0, ("s", 1), ("1", 0), ("1", 0)),
    ])


def ensemble_viscosity(i: int) -> float:
    """nu_i = 1e-3 + 4e-3 U, U the first uniform of seed 2000 + i."""
    u = float(_uniform(2000 + i, 0, 0, 0, 0))
    return 1e-3 + 4e-3 * u


def random_real_field(shape, seed=7):
    """Seeded real normal samples (for transform tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape)
