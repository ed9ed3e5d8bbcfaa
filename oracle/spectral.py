"""Plain float64 restatement of the pseudospectral Navier-Stokes RHS and its
integrating-factor Runge-Kutta step (arXiv:1808.01309, Sec. 2).

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Array conventions (shared by the C-ABI, written independently there):
  * a vector field in spectral space is a complex array of shape
    (3, nz, ny, nx//2 + 1): component, kz, ky, kx with kx fastest; ky and kz in
    FFT order (0..n/2-1, -n/2..-1): the half spectrum of a real array of
    shape (nz, ny, nx) with the x axis halved.
  * a vector field in physical space is a real array of shape (3, nz, ny, nx)
    sampled at x_i = Lx i / nx (and likewise in y, z).

Readings of the paper (each one is repeated where it is used):
  R1 (Eq. fftsum, garbled): the phase is 2 pi (p i/Nx + q j/Ny + r k/Nz) with
     (i, j, k) the grid index; the box lengths only enter the wavenumbers
     k = 2 pi p / Lx etc.
  R2 (Sec. 2, "neglect any normalization"): forward transform carries
     1/(Nx Ny Nz), backward transform none, so coefficients are Fourier-series
     coefficients and E = 1/2 sum w |u_hat|^2.
  R3 (Sec. 2, Hermitian relation printed with a minus sign): for real data
     u_hat(-k) = conj(u_hat(k)); only kx >= 0 is stored.
  R4 (dealiasing, not in the paper): cubic Orszag 2/3 rule, a mode is kept
     iff |p| < Nx/3, |q| < Ny/3 and |r| < Nz/3, i.e. |p| <= ceil(N/3) - 1.
     SPHERICAL additionally requires (p/(Nx/3))^2 + (q/(Ny/3))^2 +
     (r/(Nz/3))^2 < 1.  NONE keeps every mode except the Nyquist ones
     (|p| <= N/2 - 1), because a Nyquist mode cannot carry a Hermitian-
     consistent derivative or projection.
  R5 (state space): the method advances the truncated (Galerkin) system, so
     every operation first applies the dealias mask D to its input; modes
     outside D are ignored on input and are zero on output.
  R6 (Sec. 2, pressure as a Lagrange multiplier): the projection
     P(k) = I - k k^T/|k|^2 acts on the whole non-viscous right-hand side
     (nonlinear term plus forcing); at k = 0 the projected term is 0, so the
     mean flow is conserved.
  R7 (nonlinear term, "computed in physical space"): rotational form
     n = u x omega; the gradient part of the advection is absorbed by P.
  R8 (Sec. 2, "explicit Runge-Kutta of 2nd-4th order"): Lawson (integrating
     factor) RK2 (Heun) and RK4 (classical) with E = exp(-nu |k|^2 dt/2)
     (exp(-eta |k|^2 dt/2) for the magnetic field).
  R9 (diagnostics, not in the paper): Hermitian weight w = 1 on the planes
     kx = 0 and kx = Nx/2, else 2; shells K = floor(|k| + 1/2).
  R10 (forcing, not in the paper): a constant-in-time solenoidal forcing
     f_hat, supplied by the caller (the seeded recipe lives with the input
     generators); it is masked and added before the projection (R6).
  R11 (time): the forcing is constant, so the right-hand side does not
     depend on t.
  R12 (MHD, Eqs. uMHD, bMHD; the forms are not stated): rotational forms
     N_u = P F[u x omega + j x B] with j = curl B (the magnetic pressure
     gradient is removed by P) and N_B = i k x F[u x B] = F[curl(u x B)];
     B stays divergence-free without a projection.
  R13 (Boussinesq, Eqs. mom, temp, divv; the advection forms are not stated):
     velocity in rotational form as in R7 with the buoyancy -N theta z_hat
     added before the projection; scalar advection in divergence form
     u . grad theta = div(u theta) (equal for divergence-free u), i.e.
     -i k . F[u theta] (the CUDA path forms u . grad theta from the spectral
     gradient instead: the same Galerkin term, with its FP32 rounding relative
     to the advection term rather than to u theta); the source N w of Eq. temp uses the vertical velocity
     of the same state; theta is not forced; Lawson factors
     exp(-nu |k|^2 dt/2) on u and exp(-kappa |k|^2 dt/2) on theta, the
     buoyancy coupling is part of the explicit right-hand side.
  (R14 concerns the FP32 twiddles of the CUDA path only; this module is
  float64 throughout.)
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import fft as _fft

CUBIC, SPHERICAL, NONE = 0, 1, 2


@dataclasses.dataclass
class Config:
    """Grid, box, viscosity and scheme of one solve (Sec. 2: anisotropic boxes
    (Lx, Ly, Lz) and grids (Nx, Ny, Nz) are allowed)."""

    nx: int
    ny: int
    nz: int
    lx: float = 2.0 * math.pi
    ly: float = 2.0 * math.pi
    lz: float = 2.0 * math.pi
    nu: float = 0.0
    dealias: int = CUBIC
    rk_order: int = 4
    eta: float = 0.0  # magnetic diffusivity (MHD)
    n_bv: float = 0.0  # Brunt-Vaisala frequency (Boussinesq)
    kappa: float = 0.0  # scalar diffusivity (Boussinesq)

    @property
    def nh(self) -> int:
        return self.nx // 2 + 1


def retained_halfwidth(n: int, dealias: int) -> int:
    """Largest |index| kept along an axis of n points (reading R4)."""
    if dealias == NONE:
        return n // 2 - 1
    return -(-n // 3) - 1  # ceil(n/3) - 1: the largest integer strictly below n/3


def _signed(n: int) -> np.ndarray:
    """Signed wavenumber index in FFT order: 0..n/2-1, -n/2..-1 (Eq. fftsum)."""
    i = np.arange(n)
    return np.where(i < (n + 1) // 2, i, i - n)


def mode_indices(cfg: Config):
    """Integer indices (p, q, r) broadcast to shape (nz, ny, nh)."""
    p = np.arange(cfg.nh).reshape(1, 1, -1)
    q = _signed(cfg.ny).reshape(1, -1, 1)
    r = _signed(cfg.nz).reshape(-1, 1, 1)
    return p, q, r


def wavenumbers(cfg: Config):
    """Physical wavenumbers k = 2 pi p / L (reading R1), broadcastable arrays
    (kx of shape (1,1,nh), ky (1,ny,1), kz (nz,1,1))."""
    p, q, r = mode_indices(cfg)
    return (2.0 * math.pi / cfg.lx) * p, (2.0 * math.pi / cfg.ly) * q, (2.0 * math.pi / cfg.lz) * r


def dealias_mask(cfg: Config) -> np.ndarray:
    """Boolean mask D(k) of kept modes, shape (nz, ny, nh) (reading R4)."""
    p, q, r = mode_indices(cfg)
    kx = retained_halfwidth(cfg.nx, cfg.dealias)
    ky = retained_halfwidth(cfg.ny, cfg.dealias)
    kz = retained_halfwidth(cfg.nz, cfg.dealias)
    keep = (np.abs(p) <= kx) & (np.abs(q) <= ky) & (np.abs(r) <= kz)
    if cfg.dealias == SPHERICAL:
        rho = (3.0 * p / cfg.nx) ** 2 + (3.0 * q / cfg.ny) ** 2 + (3.0 * r / cfg.nz) ** 2
        keep = keep & (rho < 1.0)
    return keep


def hermitian_weight(cfg: Config) -> np.ndarray:
    """Multiplicity of a stored mode in the full spectrum (reading R9)."""
    w = np.full(cfg.nh, 2.0)
    w[0] = 1.0
    if cfg.nx % 2 == 0:
        w[-1] = 1.0
    return w.reshape(1, 1, -1)


def forward(u: np.ndarray) -> np.ndarray:
    """Forward transform of real data over the last three axes:
    u_hat(p,q,r) = (1/(Nx Ny Nz)) sum_ijk u_ijk exp(-2 pi i (p i/Nx + q j/Ny + r k/Nz)).
    Eq. (fftsum) with readings R1, R2, by the plain mixed-radix Cooley-Tukey
    transform of oracle/fft.py."""
    return _fft.rfft3(u)


def inverse(uh: np.ndarray, cfg: Config) -> np.ndarray:
    """Backward transform, the unnormalised sum with the opposite sign
    (Sec. 2, text after Eq. fftsum; reading R2), to real data on the grid."""
    return _fft.irfft3(uh, cfg.nz, cfg.ny, cfg.nx)


def curl_hat(uh: np.ndarray, cfg: Config) -> np.ndarray:
    """Vorticity coefficients omega_hat = i k x u_hat (spectral derivatives of
    the Galerkin system, Sec. 2)."""
    kx, ky, kz = wavenumbers(cfg)
    ux, uy, uz = uh
    return 1j * np.stack([ky * uz - kz * uy, kz * ux - kx * uz, kx * uy - ky * ux])


def project(vh: np.ndarray, cfg: Config) -> np.ndarray:
    """Leray projection v - k (k . v)/|k|^2 onto divergence-free fields, with
    the k = 0 mode set to zero (Sec. 2, pressure as Lagrange multiplier;
    reading R6)."""
    kx, ky, kz = wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    kdotv = kx * vh[0] + ky * vh[1] + kz * vh[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(k2 > 0.0, kdotv / np.where(k2 > 0.0, k2, 1.0), 0.0)
    out = np.stack([vh[0] - kx * s, vh[1] - ky * s, vh[2] - kz * s])
    out[:, k2 == 0.0] = 0.0
    return out


def nonlinear(uh: np.ndarray, cfg: Config) -> np.ndarray:
    """Unprojected, masked nonlinear term D F[u x omega] (Sec. 2: nonlinear
    terms formed in physical space and transformed; readings R4, R5, R7)."""
    D = dealias_mask(cfg)
    u_hat = uh * D
    u = inverse(u_hat, cfg)
    om = inverse(curl_hat(u_hat, cfg), cfg)
    n = np.cross(u, om, axis=0)
    return forward(n) * D


def _forcing_or_zero(forcing, cfg: Config, like: np.ndarray) -> np.ndarray:
    if forcing is None:
        return np.zeros_like(like)
    return np.asarray(forcing, dtype=np.complex128) * dealias_mask(cfg)


def _nonviscous(uh: np.ndarray, cfg: Config, forcing, nonlinear_on: bool) -> np.ndarray:
    """R(u_hat) = D P(N + f): the right-hand side without the viscous term
    (readings R5, R6)."""
    v = _forcing_or_zero(forcing, cfg, uh)
    if nonlinear_on:
        v = v + nonlinear(uh, cfg)
    return project(v, cfg) * dealias_mask(cfg)


def rhs(uh: np.ndarray, cfg: Config, forcing=None, nonlinear_on: bool = True) -> np.ndarray:
    """d u_hat/dt = D P(F[u x omega] + f_hat) - nu |k|^2 D u_hat
    (Eq. mom with theta = 0 and Eq. divv, HD case of Sec. 2)."""
    kx, ky, kz = wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    D = dealias_mask(cfg)
    return _nonviscous(uh, cfg, forcing, nonlinear_on) - cfg.nu * k2 * (uh * D)


def _lawson_step(u, E, R, dt: float, order: int):
    """One explicit Runge-Kutta step (Sec. 2, 2nd or 4th order) in Lawson
    (integrating-factor) form, reading R8.  u and E are arrays of the same
    shape (E the per-mode half-step factor exp(-rate |k|^2 dt/2)), R the
    right-hand side without the linear damping:

      RK4: k1 = R(u), k2 = R(E (u + dt/2 k1)), k3 = R(E u + dt/2 k2),
           k4 = R(E^2 u + dt E k3),
           u+ = E^2 u + dt/6 (E^2 k1 + 2 E (k2 + k3) + k4)
      RK2: k1 = R(u), k2 = R(E^2 (u + dt k1)),
           u+ = E^2 (u + dt/2 k1) + dt/2 k2
    """
    if order == 4:
        k1 = R(u)
        k2_ = R(E * (u + 0.5 * dt * k1))
        k3 = R(E * u + 0.5 * dt * k2_)
        k4 = R(E * E * u + dt * E * k3)
        return E * E * u + (dt / 6.0) * (E * E * k1 + 2.0 * E * (k2_ + k3) + k4)
    if order == 2:
        k1 = R(u)
        k2_ = R(E * E * (u + dt * k1))
        return E * E * (u + 0.5 * dt * k1) + 0.5 * dt * k2_
    raise ValueError("rk_order must be 2 or 4")


def rk_step(uh: np.ndarray, dt: float, cfg: Config, forcing=None,
            nonlinear_on: bool = True) -> np.ndarray:
    """One IF-RK step of the HD system (Sec. 2; reading R8, see _lawson_step)
    with E = exp(-nu |k|^2 dt/2)."""
    kx, ky, kz = wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    E = np.exp(-cfg.nu * k2 * dt / 2.0) + np.zeros_like(uh, dtype=np.float64)
    u = uh * dealias_mask(cfg)
    return _lawson_step(u, E, lambda v: _nonviscous(v, cfg, forcing, nonlinear_on), dt, cfg.rk_order)


# --------------------------------------------------------------------------
# MHD (Eqs. uMHD, bMHD): state = 6 components (u_x, u_y, u_z, B_x, B_y, B_z)
# --------------------------------------------------------------------------

def mhd_nonlinear(ub: np.ndarray, cfg: Config):
    """Masked nonlinear terms of the MHD system in rotational form:
    N_u = D F[u x omega + j x B] (pressure and magnetic pressure gradients
    are removed by the projection) and N_B = D (i k x F[u x B]) = F[curl(u x B)]
    (Eqs. uMHD, bMHD with j = curl B; readings R4, R5, R7)."""
    D = dealias_mask(cfg)
    u_hat, b_hat = ub[:3] * D, ub[3:] * D
    u = inverse(u_hat, cfg)
    om = inverse(curl_hat(u_hat, cfg), cfg)
    b = inverse(b_hat, cfg)
    j = inverse(curl_hat(b_hat, cfg), cfg)
    nu_ = forward(np.cross(u, om, axis=0) + np.cross(j, b, axis=0)) * D
    nb = curl_hat(forward(np.cross(u, b, axis=0)), cfg) * D
    return nu_, nb


def _mhd_nonviscous(ub, cfg: Config, forcing, nonlinear_on=True):
    D = dealias_mask(cfg)
    nu_ = _forcing_or_zero(forcing, cfg, ub[:3])
    nb = np.zeros_like(ub[3:])
    if nonlinear_on:
        n1, n2 = mhd_nonlinear(ub, cfg)
        nu_ = nu_ + n1
        nb = n2
    return np.concatenate([project(nu_, cfg) * D, nb * D])


def mhd_rhs(ub: np.ndarray, cfg: Config, forcing=None) -> np.ndarray:
    """d/dt of (u_hat, B_hat): D P(N_u + f) - nu |k|^2 D u_hat and
    N_B - eta |k|^2 D B_hat (Eqs. uMHD, bMHD, divergence-free u and B)."""
    kx, ky, kz = wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    D = dealias_mask(cfg)
    lin = np.concatenate([cfg.nu * k2 * ub[:3] * D, cfg.eta * k2 * ub[3:] * D])
    return _mhd_nonviscous(ub, cfg, forcing) - lin


def mhd_rk_step(ub: np.ndarray, dt: float, cfg: Config, forcing=None) -> np.ndarray:
    """One IF-RK step of the MHD system: the same Lawson scheme with
    E = exp(-nu |k|^2 dt/2) on u and exp(-eta |k|^2 dt/2) on B."""
    kx, ky, kz = wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz + np.zeros(ub.shape[1:])
    E = np.concatenate([np.broadcast_to(np.exp(-cfg.nu * k2 * dt / 2.0), (3,) + k2.shape),
                        np.broadcast_to(np.exp(-cfg.eta * k2 * dt / 2.0), (3,) + k2.shape)])
    u = ub * dealias_mask(cfg)
    return _lawson_step(u, E, lambda v: _mhd_nonviscous(v, cfg, forcing), dt, cfg.rk_order)


def mhd_diagnostics(ub: np.ndarray, cfg: Config, cfl: float = 0.5) -> dict:
    """HD diagnostics of u plus magnetic energy 1/2 sum w |B|^2, cross helicity
    sum w Re(u* . B) and magnetic helicity sum w Re(A* . B), A = i k x B / |k|^2
    the Coulomb-gauge vector potential (reading R9)."""
    d = diagnostics(ub[:3], cfg, cfl)
    D = dealias_mask(cfg)
    u, b = ub[:3] * D, ub[3:] * D
    w = hermitian_weight(cfg)
    kx, ky, kz = wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(k2 > 0, curl_hat(b, cfg) / np.where(k2 > 0, k2, 1.0), 0.0)
    d["magnetic_energy"] = float(np.sum(0.5 * w * np.sum(np.abs(b) ** 2, axis=0)))
    d["cross_helicity"] = float(np.sum(w * np.real(np.sum(np.conj(u) * b, axis=0))))
    d["magnetic_helicity"] = float(np.sum(w * np.real(np.sum(np.conj(a) * b, axis=0))))
    return d


# --------------------------------------------------------------------------
# Boussinesq (Eqs. mom, temp, divv): state = 4 components (u_x, u_y, u_z, theta)
# --------------------------------------------------------------------------

def boussinesq_nonlinear(ut: np.ndarray, cfg: Config):
    """Masked nonlinear terms of the Boussinesq system (reading R13):
    N_u = D F[u x omega] (the gradient part of the advection is removed by the
    projection) and N_theta = -D (i k . F[u theta]) = -D F[u . grad theta]."""
    D = dealias_mask(cfg)
    u_hat, th_hat = ut[:3] * D, ut[3] * D
    u = inverse(u_hat, cfg)
    om = inverse(curl_hat(u_hat, cfg), cfg)
    th = inverse(th_hat, cfg)
    n_u = forward(np.cross(u, om, axis=0)) * D
    g = forward(u * th)  # F[u theta], three components
    kx, ky, kz = wavenumbers(cfg)
    n_th = -1j * (kx * g[0] + ky * g[1] + kz * g[2]) * D
    return n_u, n_th


def _bq_nonviscous(ut, cfg: Config, forcing, nonlinear_on=True):
    """R = (D P(N_u + f - N theta z_hat), D (N_theta + N w)): the right-hand side
    without the diffusion terms (Eqs. mom, temp with reading R13)."""
    D = dealias_mask(cfg)
    u_hat, th_hat = ut[:3] * D, ut[3] * D
    v = _forcing_or_zero(forcing, cfg, u_hat)
    v[2] = v[2] - cfg.n_bv * th_hat
    r_th = cfg.n_bv * u_hat[2]
    if nonlinear_on:
        n_u, n_th = boussinesq_nonlinear(ut, cfg)
        v = v + n_u
        r_th = r_th + n_th
    return np.concatenate([project(v, cfg) * D, (r_th * D)[None]])


def boussinesq_rhs(ut: np.ndarray, cfg: Config, forcing=None, nonlinear_on: bool = True) -> np.ndarray:
    """d/dt of (u_hat, theta_hat): D P(N_u + f - N theta z_hat) - nu |k|^2 D u_hat
    and D (N_theta + N w_hat) - kappa |k|^2 D theta_hat (Eqs. mom, temp, divv)."""
    kx, ky, kz = wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    D = dealias_mask(cfg)
    lin = np.concatenate([cfg.nu * k2 * ut[:3] * D, (cfg.kappa * k2 * ut[3] * D)[None]])
    return _bq_nonviscous(ut, cfg, forcing, nonlinear_on) - lin


def boussinesq_rk_step(ut: np.ndarray, dt: float, cfg: Config, forcing=None,
                       nonlinear_on: bool = True) -> np.ndarray:
    """One IF-RK step of the Boussinesq system: the Lawson scheme of
    _lawson_step with E = exp(-nu |k|^2 dt/2) on u and exp(-kappa |k|^2 dt/2)
    on theta (reading R13)."""
    kx, ky, kz = wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz + np.zeros(ut.shape[1:])
    E = np.concatenate([np.broadcast_to(np.exp(-cfg.nu * k2 * dt / 2.0), (3,) + k2.shape),
                        np.exp(-cfg.kappa * k2 * dt / 2.0)[None]])
    u = ut * dealias_mask(cfg)
    return _lawson_step(u, E, lambda v: _bq_nonviscous(v, cfg, forcing, nonlinear_on), dt, cfg.rk_order)


def boussinesq_diagnostics(ut: np.ndarray, cfg: Config, cfl: float = 0.5) -> dict:
    """HD diagnostics of u plus the potential energy 1/2 sum w |theta_hat|^2
    (reading R9); energy + potential_energy is the quantity Eqs. mom and temp
    conserve without diffusion, forcing and (by the truncation) aliasing."""
    d = diagnostics(ut[:3], cfg, cfl)
    th = ut[3] * dealias_mask(cfg)
    w = hermitian_weight(cfg)
    d["potential_energy"] = float(np.sum(0.5 * w * np.abs(th) ** 2))
    return d


def diagnostics(uh: np.ndarray, cfg: Config, cfl: float = 0.5) -> dict:
    """Global quantities of the retained state D u_hat (readings R5, R9):
    energy E = 1/2 sum w |u|^2, enstrophy 1/2 sum w |omega|^2, helicity
    sum w Re(u* . omega), max |k . u_hat|, shell spectrum E(K), max |u(x)| over
    the grid and the CFL step cfl * min(dx, dy, dz) / max|u|."""
    D = dealias_mask(cfg)
    u = uh * D
    om = curl_hat(u, cfg)
    w = hermitian_weight(cfg)
    kx, ky, kz = wavenumbers(cfg)
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz) + 0.0 * D
    e_mode = 0.5 * w * np.sum(np.abs(u) ** 2, axis=0)
    energy = float(np.sum(e_mode))
    enstrophy = float(np.sum(0.5 * w * np.sum(np.abs(om) ** 2, axis=0)))
    helicity = float(np.sum(w * np.real(np.sum(np.conj(u) * om, axis=0))))
    max_div = float(np.max(np.abs(kx * u[0] + ky * u[1] + kz * u[2])))
    shell = np.floor(kmag + 0.5).astype(np.int64)
    nshells = int(shell[D].max()) + 1 if D.any() else 1
    spectrum = np.bincount(shell[D], weights=e_mode[D], minlength=nshells)
    uphys = inverse(u, cfg)
    max_u = float(np.sqrt(np.max(np.sum(uphys * uphys, axis=0))))
    dmin = min(cfg.lx / cfg.nx, cfg.ly / cfg.ny, cfg.lz / cfg.nz)
    cfl_dt = cfl * dmin / max_u if max_u > 0.0 else math.inf
    return dict(energy=energy, enstrophy=enstrophy, helicity=helicity, max_div=max_div,
                max_u=max_u, cfl_dt=cfl_dt, spectrum=spectrum)
