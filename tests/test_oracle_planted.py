"""Planted mistakes: each plausible error in the oracle must fail a pin.

Every case below replaces one function of the oracle (oracle/fft.py,
oracle/spectral.py with its MHD and Boussinesq systems, oracle/les.py) by a copy with one mistake planted (a
flipped sign, a transposed index, a dropped term, a wrong coefficient) and
runs the CPU pins of tests/test_oracle_*pins.py until one of them fails.  A
case passes when some pin fails; a mistake that no pin notices fails the case.
CPU only; nothing here touches the CUDA path."""

import dataclasses
import math

import numpy as np
import pytest

import oracle
from oracle import fft as offt
from oracle import les
from oracle import spectral as sp

from . import test_oracle_fft_pins as FP
from . import test_oracle_boussinesq_pins as BP
from . import test_oracle_les_pins as LP
from . import test_oracle_mhd_pins as MP
from . import test_oracle_pins as P


def _patch(monkeypatch, name, fn, mods):
    for m in mods:
        if hasattr(m, name):
            monkeypatch.setattr(m, name, fn)


def some_pin_fails(pins):
    for pin in pins:
        try:
            pin()
        except (AssertionError, FloatingPointError, ValueError, IndexError):
            return pin
    return None


# ---------------------------------------------------------------------------
# the transform (oracle/fft.py) and the right-hand side (oracle/spectral.py)
# ---------------------------------------------------------------------------

HD_PINS = [
    lambda: FP.test_matches_the_direct_sum(12, -1),
    lambda: FP.test_matches_the_direct_sum(96, +1),
    lambda: FP.test_real_transforms_match_the_direct_sum((8, 6, 10)),
    lambda: P.test_forward_is_the_direct_sum((8, 8, 8)),
    lambda: P.test_inverse_is_the_unnormalised_direct_sum((6, 10, 12)),
    P.test_parseval_with_hermitian_weights,
    lambda: P.test_two_thirds_halfwidth(96, 31),
    P.test_curl_of_taylor_green_is_analytic,
    lambda: P.test_rhs_of_crossed_shear_is_closed_form(4.0, 9.0, 2.5),
    P.test_projected_rhs_is_divergence_free_with_zero_mean,
    P.test_taylor_green_tendency_matches_exact_rational_advection,
    lambda: P.test_rhs_equals_bruteforce_truncated_convolution((8, 12, 16)),
    lambda: P.test_abc_flow_decays_exactly(4),
    lambda: P.test_abc_flow_decays_exactly(2),
    lambda: P.test_linear_forced_response(4),
    lambda: P.test_linear_forced_response(2),
    lambda: P.test_runge_kutta_order(4, 16.0),
    lambda: P.test_runge_kutta_order(2, 4.0),
    P.test_diagnostics_match_physical_space,
    P.test_shell_spectrum_of_closed_form_fields,
]


def _fft_first_output_transposed(x, sign):
    """Output read with k2 fastest instead of k1 (index slip)."""
    n, B = x.shape
    if n == 1:
        return np.array(x, dtype=np.complex128)
    r = offt._radix(n)
    if r == n:
        return offt.dft_matrix(n, sign) @ x
    m = n // r
    y = offt.dft_matrix(r, sign) @ x.reshape(r, m * B)
    y = y.reshape(r, m, B) * offt._twiddles(r, m, sign)
    y = np.ascontiguousarray(y.transpose(1, 0, 2))
    z = _fft_first_output_transposed(y.reshape(m, r * B), sign)
    return np.ascontiguousarray(z.reshape(m, r, B).transpose(1, 0, 2)).reshape(n, B)


def _twiddles_conjugated(r, m, sign):
    k1 = np.arange(r).reshape(-1, 1)
    n2 = np.arange(m).reshape(1, -1)
    return offt._roots(k1 * n2, r * m, -sign).reshape(r, m, 1)


def _irfft3_without_conj(uh, nz, ny, nx):
    nh = nx // 2 + 1
    out = np.empty(uh.shape[:-3] + (nz, ny, nx))
    for idx in np.ndindex(*uh.shape[:-3]):
        a = offt.fft_axis(offt.fft_axis(uh[idx], -3, +1), -2, +1)
        full = np.empty((nz, ny, nx), dtype=np.complex128)
        full[..., :nh] = a
        full[..., nh:] = a[..., nx - nh:0:-1]  # the conjugate is missing
        out[idx] = offt.fft_axis(full, -1, +1).real
    return out


_orig_rfft3 = offt.rfft3
_orig_curl = sp.curl_hat
_orig_project = sp.project
_orig_wavenumbers = sp.wavenumbers
_orig_rhs = sp.rhs


def _nonlinear_omega_cross_u(uh, cfg):
    D = sp.dealias_mask(cfg)
    u_hat = uh * D
    u = sp.inverse(u_hat, cfg)
    om = sp.inverse(sp.curl_hat(u_hat, cfg), cfg)
    return sp.forward(np.cross(om, u, axis=0)) * D  # operands swapped


def _project_drops_z(vh, cfg):
    out = _orig_project(vh, cfg)
    kx, ky, kz = sp.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(k2 > 0, (kx * vh[0] + ky * vh[1] + kz * vh[2]) / np.where(k2 > 0, k2, 1), 0)
    out[2] = out[2] + kz * s  # the k_z (k . v)/|k|^2 term is lost
    return out


def _lawson_rk4_weight_one(u, E, R, dt, order):
    if order != 4:
        return _orig_lawson(u, E, R, dt, order)
    k1 = R(u)
    k2 = R(E * (u + 0.5 * dt * k1))
    k3 = R(E * u + 0.5 * dt * k2)
    k4 = R(E * E * u + dt * E * k3)
    return E * E * u + (dt / 6.0) * (E * E * k1 + E * (k2 + k3) + k4)  # weight 1 instead of 2


def _lawson_rk2_full_first_stage(u, E, R, dt, order):
    if order != 2:
        return _orig_lawson(u, E, R, dt, order)
    k1 = R(u)
    k2 = R(E * E * (u + dt * k1))
    return E * E * (u + dt * k1) + 0.5 * dt * k2  # dt instead of dt/2 on k1


_orig_lawson = sp._lawson_step


def _rk_step_full_step_factor(uh, dt, cfg, forcing=None, nonlinear_on=True):
    kx, ky, kz = sp.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    E = np.exp(-cfg.nu * k2 * dt) + np.zeros_like(uh, dtype=np.float64)  # dt instead of dt/2
    u = uh * sp.dealias_mask(cfg)
    return sp._lawson_step(u, E, lambda v: sp._nonviscous(v, cfg, forcing, nonlinear_on), dt, cfg.rk_order)


def _halfwidth_floor(n, dealias):
    return n // 2 - 1 if dealias == sp.NONE else n // 3  # floor(n/3) aliases when 3 divides n


def _weight_two_everywhere(cfg):
    return np.full((1, 1, cfg.nh), 2.0)


def _wavenumbers_swapped_boxes(cfg):
    kx, ky, kz = _orig_wavenumbers(cfg)
    return kx, ky * (cfg.ly / cfg.lx), kz  # ky scaled with Lx


def _rhs_viscous_sign(uh, cfg, forcing=None, nonlinear_on=True):
    kx, ky, kz = sp.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    return sp._nonviscous(uh, cfg, forcing, nonlinear_on) + cfg.nu * k2 * (uh * sp.dealias_mask(cfg))


def _nonlinear_with_mistake(kind):
    def f(uh, cfg):
        D = sp.dealias_mask(cfg)
        u_hat = uh if kind == "input mask dropped" else uh * D
        u = sp.inverse(u_hat, cfg)
        om = sp.inverse(sp.curl_hat(u_hat, cfg), cfg)
        n = sp.forward(np.cross(u, om, axis=0))
        return n if kind == "output mask dropped" else n * D

    return f


_orig_nonviscous = sp._nonviscous


def _nonviscous_output_unmasked(uh, cfg, forcing, nonlinear_on):
    # both output masks (of the nonlinear term and after the projection) dropped;
    # either one alone is redundant with the other
    v = sp._forcing_or_zero(forcing, cfg, uh)
    if nonlinear_on:
        v = v + _nonlinear_with_mistake("output mask dropped")(uh, cfg)
    return sp.project(v, cfg)


def _nonviscous_forcing_sign(uh, cfg, forcing, nonlinear_on):
    neg = None if forcing is None else -np.asarray(forcing)
    return _orig_nonviscous(uh, cfg, neg, nonlinear_on)


def _diagnostics_with_mistake(kind):
    def f(uh, cfg, cfl=0.5):
        D = sp.dealias_mask(cfg)
        u = uh * D
        om = sp.curl_hat(u, cfg)
        w = sp.hermitian_weight(cfg)
        kx, ky, kz = sp.wavenumbers(cfg)
        kmag = np.sqrt(kx * kx + ky * ky + kz * kz) + 0.0 * D
        e_mode = 0.5 * w * np.sum(np.abs(u) ** 2, axis=0)
        half = 1.0 if kind == "enstrophy without 1/2" else 0.5
        enstrophy = float(np.sum(half * w * np.sum(np.abs(om) ** 2, axis=0)))
        helicity = float(np.sum(w * np.real(np.sum(np.conj(u) * om, axis=0))))
        max_div = float(np.max(np.abs(kx * u[0] + ky * u[1] + kz * u[2])))
        shell = np.floor(kmag if kind == "shell by floor(|k|)" else kmag + 0.5).astype(np.int64)
        spectrum = np.bincount(shell[D], weights=e_mode[D], minlength=int(shell[D].max()) + 1)
        uphys = sp.inverse(u, cfg)
        if kind == "max|u| of one component":
            max_u = float(np.max(np.abs(uphys)))
        else:
            max_u = float(np.sqrt(np.max(np.sum(uphys * uphys, axis=0))))
        pick = max if kind == "CFL on the largest spacing" else min
        cfl_dt = cfl * pick(cfg.lx / cfg.nx, cfg.ly / cfg.ny, cfg.lz / cfg.nz) / max_u
        return dict(energy=float(np.sum(e_mode)), enstrophy=enstrophy, helicity=helicity, max_div=max_div,
                    max_u=max_u, cfl_dt=cfl_dt, spectrum=spectrum)

    return f


HD_MISTAKES = {
    "twiddle sign": ("_twiddles", _twiddles_conjugated, [offt]),
    "output index order": ("fft_first", _fft_first_output_transposed, [offt]),
    "hermitian fill without conjugate": ("irfft3", _irfft3_without_conj, [offt]),
    "forward normalisation dropped": ("rfft3", lambda u: _orig_rfft3(u) * np.prod(np.shape(u)[-3:]), [offt]),
    "curl sign": ("curl_hat", lambda uh, cfg: -_orig_curl(uh, cfg), [sp, oracle]),
    "cross product order": ("nonlinear", _nonlinear_omega_cross_u, [sp, oracle]),
    "projection term dropped": ("project", _project_drops_z, [sp, oracle]),
    "rk4 stage weight": ("_lawson_step", _lawson_rk4_weight_one, [sp]),
    "rk2 first-stage coefficient": ("_lawson_step", _lawson_rk2_full_first_stage, [sp]),
    "integrating factor over a full step": ("rk_step", _rk_step_full_step_factor, [sp, oracle]),
    "mask half-width floor(N/3)": ("retained_halfwidth", _halfwidth_floor, [sp, oracle]),
    "hermitian weight": ("hermitian_weight", _weight_two_everywhere, [sp, oracle]),
    "box lengths swapped": ("wavenumbers", _wavenumbers_swapped_boxes, [sp, oracle]),
    "viscous term sign": ("rhs", _rhs_viscous_sign, [sp, oracle]),
    "forcing sign": ("_nonviscous", _nonviscous_forcing_sign, [sp]),
    "output mask dropped": ("_nonviscous", _nonviscous_output_unmasked, [sp]),
    "input mask dropped": ("nonlinear", _nonlinear_with_mistake("input mask dropped"), [sp, oracle]),
}
HD_MISTAKES.update({k: ("diagnostics", _diagnostics_with_mistake(k), [sp, oracle])
                    for k in ("enstrophy without 1/2", "shell by floor(|k|)", "max|u| of one component",
                              "CFL on the largest spacing")})


@pytest.mark.parametrize("name", list(HD_MISTAKES))
def test_planted_hd_mistake_fails_a_pin(name, monkeypatch):
    fn_name, fn, mods = HD_MISTAKES[name]
    _patch(monkeypatch, fn_name, fn, mods)
    assert some_pin_fails(HD_PINS) is not None, f"no pin notices: {name}"


# ---------------------------------------------------------------------------
# the LES closure (oracle/les.py): every basis tensor, the invariants, the
# network gradient and the adjoint of the force loss
# ---------------------------------------------------------------------------

LES_PINS = [
    LP.test_invariants_closed_forms,
    LP.test_tensor_basis_closed_forms,
    LP.test_tensor_basis_gradient_model_identity_and_equivariance,
    LP.test_gelu_derivative_matches_finite_differences,
    LP.test_mlp_gradients_match_central_differences,
    LP.test_force_loss_is_the_grid_mean_of_the_residual,
    LP.test_force_loss_gradients_match_central_differences,
]


def _basis_with_mistake(which):
    """tensor_basis with tensor `which` (0-based) built by a mistaken formula."""

    def tb(A, s_A=1.0):
        At = np.swapaxes(A, 0, 1)
        S = 0.5 * (A + At) / s_A
        R = 0.5 * (A - At) / s_A

        def mm(X, Y):
            return np.einsum("ik...,kj...->ij...", X, Y)

        def tr(X):
            return np.einsum("ii...->...", X)

        eye = np.eye(3).reshape((3, 3) + (1,) * (A.ndim - 2))
        S2, R2 = mm(S, S), mm(R, R)
        T = [S, mm(S, R) - mm(R, S), S2 - tr(S2) * eye / 3.0, R2 - tr(R2) * eye / 3.0,
             mm(R, S2) - mm(S2, R), mm(R2, S) + mm(S, R2) - 2.0 * tr(mm(S, R2)) * eye / 3.0]
        wrong = [0.5 * (A - At) / s_A,                          # R in place of S
                 mm(R, S) - mm(S, R),                           # commutator sign
                 S2,                                            # trace not removed
                 R2 - tr(R2) * eye,                             # 1 instead of 1/3
                 mm(S2, R) - mm(R, S2),                         # order swapped
                 mm(R2, S) + mm(S, R2) - tr(mm(S, R2)) * eye / 3.0]  # 1/3 instead of 2/3
        T[which] = wrong[which]
        return np.stack([np.stack([t[i, j] for (i, j) in les.SYM]) for t in T])

    return tb


def _invariants_with_mistake(A):
    At = np.swapaxes(A, 0, 1)
    S, R = 0.5 * (A + At), 0.5 * (A - At)

    def mm(X, Y):
        return np.einsum("ik...,kj...->ij...", X, Y)

    def tr(X):
        return np.einsum("ii...->...", X)

    S2, R2 = mm(S, S), mm(R, R)
    return np.stack([tr(S2), tr(R2), tr(mm(S2, S)), tr(mm(S2, R)), tr(mm(S2, R2))])  # tr(S^2 R) for tr(S R^2)


def _gelu_grad_without_chain(x):
    t = np.tanh(les.C_GELU * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * les.C_GELU  # the 1 + 3 a x^2 factor is lost


def _force_loss_with_mistake(kind):
    """force_loss_and_grads with one mistake planted in its adjoint."""

    def f(uh, cfg, p, norm, f_hat, rnd=None):
        D = sp.dealias_mask(cfg)
        A = les.gradient(uh, cfg)
        lam = les.invariants(A)
        X = (lam.reshape(5, -1).T - norm["mean"]) / norm["std"]
        y, cache = les.mlp_forward(p, X, rnd)
        Tb = les.tensor_basis(A, norm["s_A"]).reshape(6, 6, -1)
        tau = norm["s_tau"] * np.einsum("nmp,pn->mp", Tb, y).reshape((6,) + lam.shape[1:])
        th = sp.forward(tau)
        k = sp.wavenumbers(cfg)
        full = {}
        for m, (i, j) in enumerate(les.SYM):
            full[(i, j)] = th[m]
            full[(j, i)] = th[m]
        div = np.stack([sum(1j * k[j] * full[(i, j)] for j in range(3)) for i in range(3)])
        r_hat = sp.project(-div * D, cfg) * D - np.asarray(f_hat) * D
        w = sp.hermitian_weight(cfg)
        L = float(np.sum(w * np.abs(r_hat) ** 2))
        G = np.stack([np.stack([sp.inverse((1j * k[j] * r_hat[i])[None], cfg)[0] for j in range(3)])
                      for i in range(3)])
        scale = (1.0 if kind == "scale" else 2.0) / (cfg.nx * cfg.ny * cfg.nz)
        if kind == "symmetric part":
            dtau = np.stack([scale * G[i, j] for (i, j) in les.SYM])
        elif kind == "sign":
            dtau = np.stack([-scale * (G[i, j] + G[j, i]) if i != j else -scale * G[i, i] for (i, j) in les.SYM])
        else:
            dtau = np.stack([scale * (G[i, j] + G[j, i]) if i != j else scale * G[i, i] for (i, j) in les.SYM])
        dy = norm["s_tau"] * np.einsum("nmp,mp->pn", Tb, dtau.reshape(6, -1))
        return L, les._backward(p, cache, dy, rnd)

    return f


LES_MISTAKES = {f"basis tensor T{n + 1}": ("tensor_basis", _basis_with_mistake(n)) for n in range(6)}
LES_MISTAKES.update({
    "invariant tr(S R^2)": ("invariants", _invariants_with_mistake),
    "gelu derivative": ("gelu_grad", _gelu_grad_without_chain),
    "adjoint scale": ("force_loss_and_grads", _force_loss_with_mistake("scale")),
    "adjoint symmetric part": ("force_loss_and_grads", _force_loss_with_mistake("symmetric part")),
    "adjoint sign": ("force_loss_and_grads", _force_loss_with_mistake("sign")),
})


@pytest.mark.parametrize("name", list(LES_MISTAKES))
def test_planted_les_mistake_fails_a_pin(name, monkeypatch):
    fn_name, fn = LES_MISTAKES[name]
    monkeypatch.setattr(les, fn_name, fn)
    assert some_pin_fails(LES_PINS) is not None, f"no pin notices: {name}"


# ---------------------------------------------------------------------------
# the MHD system (Eqs. uMHD, bMHD in oracle/spectral.py)
# ---------------------------------------------------------------------------

MHD_PINS = [
    MP.test_mhd_tendency_matches_exact_advective_form,
    MP.test_zero_magnetic_field_reduces_to_hydrodynamics,
    MP.test_ideal_invariants_are_not_transferred,
    lambda: MP.test_parallel_beltrami_fields_decay_exactly(4),
    lambda: MP.test_parallel_beltrami_fields_decay_exactly(2),
    MP.test_mhd_diagnostics_closed_forms,
    MP.test_magnetic_helicity_of_a_wavenumber_two_field,
]


def _mhd_fields(ub, cfg):
    D = sp.dealias_mask(cfg)
    u_hat, b_hat = ub[:3] * D, ub[3:] * D
    return (D, sp.inverse(u_hat, cfg), sp.inverse(sp.curl_hat(u_hat, cfg), cfg), sp.inverse(b_hat, cfg),
            sp.inverse(sp.curl_hat(b_hat, cfg), cfg))


def _mhd_nonlinear_with_mistake(kind):
    def f(ub, cfg):
        D, u, om, b, j = _mhd_fields(ub, cfg)
        lorentz = np.cross(j, b, axis=0)
        emf = np.cross(u, b, axis=0)
        if kind == "lorentz sign":
            lorentz = -lorentz
        elif kind == "lorentz dropped":
            lorentz = 0.0 * lorentz
        elif kind == "induction sign":
            emf = -emf
        elif kind == "induction field":
            emf = np.cross(u, j, axis=0)  # current in place of the field
        return sp.forward(np.cross(u, om, axis=0) + lorentz) * D, sp.curl_hat(sp.forward(emf), cfg) * D

    return f


_orig_mhd_nonviscous = sp._mhd_nonviscous
_orig_mhd_rk_step = sp.mhd_rk_step
_orig_mhd_rhs = sp.mhd_rhs


def _mhd_nonviscous_lorentz_unprojected(ub, cfg, forcing, nonlinear_on=True):
    if not nonlinear_on:
        return _orig_mhd_nonviscous(ub, cfg, forcing, nonlinear_on)
    D, u, om, b, j = _mhd_fields(ub, cfg)
    f = sp._forcing_or_zero(forcing, cfg, ub[:3])
    n_u = sp.project(sp.forward(np.cross(u, om, axis=0)) * D + f, cfg) * D
    n_u = n_u + sp.forward(np.cross(j, b, axis=0)) * D  # the Lorentz force skips the projection
    n_b = sp.curl_hat(sp.forward(np.cross(u, b, axis=0)), cfg) * D
    return np.concatenate([n_u, n_b])


def _mhd_rk_step_swapped_diffusivities(ub, dt, cfg, forcing=None):
    return _orig_mhd_rk_step(ub, dt, dataclasses.replace(cfg, nu=cfg.eta, eta=cfg.nu), forcing)


def _mhd_rhs_viscosity_on_b(ub, cfg, forcing=None):
    return _orig_mhd_rhs(ub, dataclasses.replace(cfg, eta=cfg.nu), forcing)


def _mhd_diagnostics_with_mistake(kind):
    def f(ub, cfg, cfl=0.5):
        d = sp.diagnostics(ub[:3], cfg, cfl)
        D = sp.dealias_mask(cfg)
        u, b = ub[:3] * D, ub[3:] * D
        w = sp.hermitian_weight(cfg)
        kx, ky, kz = sp.wavenumbers(cfg)
        k2 = kx * kx + ky * ky + kz * kz
        with np.errstate(divide="ignore", invalid="ignore"):
            a = np.where(k2 > 0, sp.curl_hat(b, cfg) / np.where(k2 > 0, k2, 1.0), 0.0)
        if kind == "potential without 1/|k|^2":
            a = sp.curl_hat(b, cfg)
        half = 1.0 if kind == "magnetic energy without 1/2" else 0.5
        ch = 0.5 if kind == "cross helicity halved" else 1.0
        d["magnetic_energy"] = float(np.sum(half * w * np.sum(np.abs(b) ** 2, axis=0)))
        d["cross_helicity"] = float(np.sum(ch * w * np.real(np.sum(np.conj(u) * b, axis=0))))
        d["magnetic_helicity"] = float(np.sum(w * np.real(np.sum(np.conj(a) * b, axis=0))))
        return d

    return f


MHD_MISTAKES = {k: ("mhd_nonlinear", _mhd_nonlinear_with_mistake(k), [sp, oracle])
                for k in ("lorentz sign", "lorentz dropped", "induction sign", "induction field")}
MHD_MISTAKES.update({
    "lorentz force not projected": ("_mhd_nonviscous", _mhd_nonviscous_lorentz_unprojected, [sp]),
    "diffusivities swapped in the step": ("mhd_rk_step", _mhd_rk_step_swapped_diffusivities, [sp, oracle]),
    "viscosity on B in the right-hand side": ("mhd_rhs", _mhd_rhs_viscosity_on_b, [sp, oracle]),
})
MHD_MISTAKES.update({k: ("mhd_diagnostics", _mhd_diagnostics_with_mistake(k), [sp, oracle])
                     for k in ("potential without 1/|k|^2", "magnetic energy without 1/2",
                               "cross helicity halved")})


@pytest.mark.parametrize("name", list(MHD_MISTAKES))
def test_planted_mhd_mistake_fails_a_pin(name, monkeypatch):
    fn_name, fn, mods = MHD_MISTAKES[name]
    _patch(monkeypatch, fn_name, fn, mods)
    assert some_pin_fails(MHD_PINS) is not None, f"no pin notices: {name}"


# ---------------------------------------------------------------------------
# the Boussinesq system (Eqs. mom, temp, divv in oracle/spectral.py)
# ---------------------------------------------------------------------------

BQ_PINS = [
    BP.test_tendency_matches_exact_advective_form,
    BP.test_scalar_advection_matches_brute_force_convolution,
    BP.test_ideal_total_energy_and_scalar_variance_are_conserved,
    BP.test_internal_gravity_wave_tendency_and_frequency,
    BP.test_zero_scalar_reduces_to_hydrodynamics,
    BP.test_passive_scalar_diffusion_is_exact,
    BP.test_velocity_tendency_is_solenoidal_and_potential_energy_diagnostic,
    BP.test_linear_terms_carry_their_own_diffusivities,
]

_orig_bq_nonviscous = sp._bq_nonviscous
_orig_bq_rk_step = sp.boussinesq_rk_step
_orig_bq_rhs = sp.boussinesq_rhs


def _bq_nonviscous_with_mistake(kind):
    def f(ut, cfg, forcing, nonlinear_on=True):
        D = sp.dealias_mask(cfg)
        u_hat, th_hat = ut[:3] * D, ut[3] * D
        v = sp._forcing_or_zero(forcing, cfg, u_hat)
        buoy = np.zeros_like(v)
        buoy[0 if kind == "buoyancy on x" else 2] = -cfg.n_bv * th_hat
        if kind == "buoyancy sign":
            buoy = -buoy
        r_th = cfg.n_bv * (u_hat[0] if kind == "source from u_x" else u_hat[2])
        if kind == "source N w dropped":
            r_th = 0.0 * r_th
        if nonlinear_on:
            n_u, n_th = sp.boussinesq_nonlinear(ut, cfg)
            v = v + n_u
            r_th = r_th + n_th
        if kind == "buoyancy not projected":
            vel = sp.project(v, cfg) * D + buoy * D
        else:
            vel = sp.project(v + buoy, cfg) * D
        return np.concatenate([vel, (r_th * D)[None]])

    return f


def _bq_nonlinear_with_mistake(kind):
    def f(ut, cfg):
        D = sp.dealias_mask(cfg)
        u_hat, th_hat = ut[:3] * D, ut[3] * D
        u = sp.inverse(u_hat, cfg)
        om = sp.inverse(sp.curl_hat(u_hat, cfg), cfg)
        th = sp.inverse(th_hat, cfg)
        g = sp.forward((om if kind == "scalar advected by the vorticity" else u) * th)
        kx, ky, kz = sp.wavenumbers(cfg)
        sign = +1j if kind == "scalar advection sign" else -1j
        return sp.forward(np.cross(u, om, axis=0)) * D, sign * (kx * g[0] + ky * g[1] + kz * g[2]) * D

    return f


def _bq_rk_step_swapped_diffusivities(ut, dt, cfg, forcing=None, nonlinear_on=True):
    return _orig_bq_rk_step(ut, dt, dataclasses.replace(cfg, nu=cfg.kappa, kappa=cfg.nu), forcing, nonlinear_on)


def _bq_rhs_viscosity_on_theta(ut, cfg, forcing=None, nonlinear_on=True):
    return _orig_bq_rhs(ut, dataclasses.replace(cfg, kappa=cfg.nu), forcing, nonlinear_on)


def _bq_diagnostics_potential_energy_doubled(ut, cfg, cfl=0.5):
    d = sp.diagnostics(ut[:3], cfg, cfl)
    th = ut[3] * sp.dealias_mask(cfg)
    d["potential_energy"] = float(np.sum(sp.hermitian_weight(cfg) * np.abs(th) ** 2))  # 1/2 dropped
    return d


BQ_MISTAKES = {k: ("_bq_nonviscous", _bq_nonviscous_with_mistake(k), [sp])
               for k in ("buoyancy sign", "buoyancy on x", "source N w dropped", "source from u_x",
                         "buoyancy not projected")}
BQ_MISTAKES.update({k: ("boussinesq_nonlinear", _bq_nonlinear_with_mistake(k), [sp, oracle])
                    for k in ("scalar advection sign", "scalar advected by the vorticity")})
BQ_MISTAKES.update({
    "diffusivities swapped in the step": ("boussinesq_rk_step", _bq_rk_step_swapped_diffusivities, [sp, oracle]),
    "viscosity on theta in the right-hand side": ("boussinesq_rhs", _bq_rhs_viscosity_on_theta, [sp, oracle]),
    "potential energy without 1/2": ("boussinesq_diagnostics", _bq_diagnostics_potential_energy_doubled,
                                     [sp, oracle]),
})


@pytest.mark.parametrize("name", list(BQ_MISTAKES))
def test_planted_boussinesq_mistake_fails_a_pin(name, monkeypatch):
    fn_name, fn, mods = BQ_MISTAKES[name]
    _patch(monkeypatch, fn_name, fn, mods)
    assert some_pin_fails(BQ_PINS) is not None, f"no pin notices: {name}"


def test_unmodified_oracle_passes_every_listed_pin():
    """Control: with nothing planted, none of the pins used above fails."""
    assert some_pin_fails(HD_PINS) is None
    assert some_pin_fails(LES_PINS) is None
    assert some_pin_fails(MHD_PINS) is None
    assert some_pin_fails(BQ_PINS) is None


@pytest.mark.parametrize("fn_name,factory,mods,pins", [
    ("nonlinear", _nonlinear_with_mistake, [sp, oracle], HD_PINS),
    ("diagnostics", _diagnostics_with_mistake, [sp, oracle], HD_PINS),
    ("mhd_nonlinear", _mhd_nonlinear_with_mistake, [sp, oracle], MHD_PINS),
    ("mhd_diagnostics", _mhd_diagnostics_with_mistake, [sp, oracle], MHD_PINS),
    ("_bq_nonviscous", _bq_nonviscous_with_mistake, [sp], BQ_PINS),
    ("boussinesq_nonlinear", _bq_nonlinear_with_mistake, [sp, oracle], BQ_PINS),
])
def test_rewritten_copies_without_a_mistake_pass(fn_name, factory, mods, pins, monkeypatch):
    """Control for the rewritten copies above: with no mistake selected each
    one passes every pin, so a failing case comes from its planted mistake."""
    _patch(monkeypatch, fn_name, factory("none"), mods)
    assert some_pin_fails(pins) is None
    assert math.isfinite(float(np.sum(oracle.hermitian_weight(sp.Config(8, 8, 8)))))
