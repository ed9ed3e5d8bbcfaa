"""FP64 oracle of the learned large-eddy-simulation (LES) closure.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The closure models the subgrid stress of a filtered velocity field with a
pointwise multilayer perceptron of the resolved velocity-gradient invariants
(5 -> 64 -> 64 -> 6, GELU) whose outputs weight a tensor basis.  Readings
(the paper has no LES; these follow the workload statement):

  L1 filter: the sharp spectral box |p|, |q|, |r| <= kc; with kc equal to the
     2/3-rule half-width of the LES grid the filtered field is exactly an LES
     state (kc = 21 for a 64^3 LES).
  L2 subgrid stress: tau_ij = F[u_i u_j] - F[ubar_i ubar_j] (F the filter,
     ubar = F[u]), the products u_i u_j formed on the DNS grid, the result
     sampled on the LES grid.  The LES forms its own nonlinear term from ubar
     and truncates it at kc, so this is exactly the part of the filtered
     momentum flux that it misses (for the sharp filter, F[ubar ubar] differs
     from ubar ubar only above kc, where the closure term is discarded).
  L3 inputs: with A_ij = d u_i / d x_j, S = (A + A^T)/2, R = (A - A^T)/2, the
     invariants tr(S^2), tr(R^2), tr(S^3), tr(S R^2), tr(S^2 R^2) (the basis of
     Pope 1975 for a traceless gradient), standardised by fixed per-input
     scales: x_n = (lambda_n - mean_n) / std_n.
  L4 outputs: coefficients g_1..g_6 of the first six tensors of the same
     integrity basis (Pope 1975), built from the scaled S' = S / s_A,
     R' = R / s_A:
        T1 = S', T2 = S'R' - R'S', T3 = S'^2 - tr(S'^2) I/3,
        T4 = R'^2 - tr(R'^2) I/3, T5 = R'S'^2 - S'^2R',
        T6 = R'^2 S' + S'R'^2 - 2 tr(S'R'^2) I/3,
     tau = s_tau sum_n g_n T_n, components ordered 11, 22, 33, 12, 13, 23.
     Every T_n is symmetric, traceless and rotates with the flow, so the
     model stress does too.  (Taking the six stress components directly as
     outputs of rotation-invariant inputs is not equivariant: for isotropic
     data the mean-square-optimal such map is isotropic, a pure pressure that
     the projection removes.)
  L5 GELU: the tanh form 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))
     (Hendrycks and Gimpel 2016).
  L6 closure term of the momentum equation: -div tau, i.e. -i k_j tau_hat_ij,
     added to the nonlinear term before the Leray projection.
  L7 loss: mean over samples and the six components of (y - t)^2, where y is
     the network output (plain fit) or the model stress in units of s_tau,
     sum_n g_n T_n (tensor-basis fit).
  L8 force loss: L = sum over the half spectrum of w |r_hat|^2 (w = 1 on the
     kx = 0 plane, 2 elsewhere; by Parseval the grid mean of |r|^2), with
     r_hat = D P(closure term) - f_hat the residual against a given projected,
     band-limited subgrid force f_hat (the filtered DNS right-hand side minus
     the LES right-hand side of the filtered state).
  L9 transfer loss: L = sum over shells K of (T_model(K) - T_exact(K))^2 with
     T(K) = sum over the modes of shell K (K = floor(|k| + 1/2)) of
     w Re(u_hat* . f_hat), f_hat the projected closure term (model) or the
     subgrid force (exact): the energy the closure moves into or out of each
     shell.
"""

from __future__ import annotations

import math

import numpy as np

from . import spectral as sp

C_GELU = math.sqrt(2.0 / math.pi)
SYM = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))  # tau component order (L4)


# --------------------------------------------------------------------------
# Filter and subgrid stress (L1, L2)
# --------------------------------------------------------------------------

def box_filter(uh: np.ndarray, n_dns: int, n_les: int, kc: int) -> np.ndarray:
    """Keep |p|, |q|, |r| <= kc of a DNS spectral field (n_dns^3) and return it
    in the layout of an n_les^3 grid (Fourier coefficients are per unit
    volume, so they carry over unchanged)."""
    nh = n_les // 2 + 1
    out = np.zeros(uh.shape[:-3] + (n_les, n_les, nh), dtype=np.complex128)
    idx = np.concatenate([np.arange(0, kc + 1), np.arange(-kc, 0)])
    src = np.where(idx >= 0, idx, idx + n_dns)
    dst = np.where(idx >= 0, idx, idx + n_les)
    sel_src = np.ix_(src, src, np.arange(kc + 1))
    sel_dst = np.ix_(dst, dst, np.arange(kc + 1))
    for c in range(uh.shape[0]):
        out[c][sel_dst] = uh[c][sel_src]
    return out


def sgs_stress_true(uh_dns: np.ndarray, n_dns: int, n_les: int, kc: int) -> np.ndarray:
    """tau_ij = F[u_i u_j] - F[ubar_i ubar_j] on the n_les^3 grid, shape
    (6, n_les, n_les, n_les) in the order of SYM (reading L2).  Both products
    are formed on the DNS grid, where neither aliases."""
    cd = sp.Config(n_dns, n_dns, n_dns)
    cl = sp.Config(n_les, n_les, n_les)
    u = sp.inverse(uh_dns, cd)
    # ubar on the DNS grid: the filtered field, zero-padded
    ubar = sp.inverse(box_filter(uh_dns, n_dns, n_dns, kc), cd)
    out = np.empty((6, n_les, n_les, n_les))
    for m, (i, j) in enumerate(SYM):
        full = sp.forward(u[i] * u[j]) - sp.forward(ubar[i] * ubar[j])
        out[m] = sp.inverse(box_filter(full[None], n_dns, n_les, kc), cl)[0]
    return out


# --------------------------------------------------------------------------
# Gradient invariants (L3)
# --------------------------------------------------------------------------

def gradient(uh: np.ndarray, cfg: sp.Config) -> np.ndarray:
    """A_ij = d u_i/d x_j on the grid, shape (3, 3, nz, ny, nx)."""
    k = sp.wavenumbers(cfg)
    D = sp.dealias_mask(cfg)
    return np.stack([np.stack([sp.inverse((1j * k[j] * uh[i] * D)[None], cfg)[0] for j in range(3)])
                     for i in range(3)])


def invariants(A: np.ndarray) -> np.ndarray:
    """The five invariants of reading L3, shape (5,) + A.shape[2:]."""
    At = np.swapaxes(A, 0, 1)
    S = 0.5 * (A + At)
    R = 0.5 * (A - At)

    def mm(X, Y):
        return np.einsum("ik...,kj...->ij...", X, Y)

    def tr(X):
        return np.einsum("ii...->...", X)

    S2, R2 = mm(S, S), mm(R, R)
    return np.stack([tr(S2), tr(R2), tr(mm(S2, S)), tr(mm(S, R2)), tr(mm(S2, R2))])


def tensor_basis(A: np.ndarray, s_A: float = 1.0) -> np.ndarray:
    """T_1..T_6 of reading L4 for the gradient A (3, 3, ...), shape
    (6 tensors, 6 components) + A.shape[2:]."""
    At = np.swapaxes(A, 0, 1)
    S = 0.5 * (A + At) / s_A
    R = 0.5 * (A - At) / s_A

    def mm(X, Y):
        return np.einsum("ik...,kj...->ij...", X, Y)

    def tr(X):
        return np.einsum("ii...->...", X)

    eye = np.eye(3).reshape((3, 3) + (1,) * (A.ndim - 2))
    S2, R2 = mm(S, S), mm(R, R)
    T = [S,
         mm(S, R) - mm(R, S),
         S2 - tr(S2) * eye / 3.0,
         R2 - tr(R2) * eye / 3.0,
         mm(R, S2) - mm(S2, R),
         mm(R2, S) + mm(S, R2) - 2.0 * tr(mm(S, R2)) * eye / 3.0]
    return np.stack([np.stack([t[i, j] for (i, j) in SYM]) for t in T])


# --------------------------------------------------------------------------
# The network (L4, L5, L7)
# --------------------------------------------------------------------------

def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(C_GELU * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    t = np.tanh(C_GELU * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * C_GELU * (1.0 + 3.0 * 0.044715 * x * x)


def init_params(seed: int = 0, width: int = 64):
    """W1 (5 x w), b1, W2 (w x w), b2, W3 (w x 6), b3; scaled normal init."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((5, width)) / math.sqrt(5.0), "b1": np.zeros(width),
        "W2": rng.standard_normal((width, width)) / math.sqrt(width), "b2": np.zeros(width),
        "W3": rng.standard_normal((width, 6)) / math.sqrt(width) * 0.1, "b3": np.zeros(6),
    }


def mlp_forward(p, X, rnd=None):
    """y = (GELU(GELU(X W1 + b1) W2 + b2)) W3 + b3 for rows of X (B x 5).
    rnd, if given, rounds the operands of every product the way a BF16
    tensor-core kernel sees them (inputs, weights, hidden activations)."""
    r = rnd or (lambda a: a)
    z1 = r(X) @ r(p["W1"]) + p["b1"]
    h1 = gelu(z1)
    z2 = r(h1) @ r(p["W2"]) + p["b2"]
    h2 = gelu(z2)
    y = r(h2) @ r(p["W3"]) + p["b3"]
    return y, (X, z1, h1, z2, h2)


def mse_and_grads(p, X, T, rnd=None):
    """Loss L = mean((y - T)^2) (reading L7) and its gradients with respect to
    every parameter, by the chain rule written out."""
    y, cache = mlp_forward(p, X, rnd)
    B = X.shape[0]
    dy = 2.0 * (y - T) / (B * T.shape[1])
    return float(np.mean((y - T) ** 2)), _backward(p, cache, dy, rnd)


def mse_and_grads_tb(p, X, Bas, T, rnd=None):
    """Tensor-basis fit (readings L4, L7): model stress m = Bas y per sample
    (Bas of shape (B, 6 components, 6 tensors)), L = mean((m - T)^2) with T
    in units of s_tau; returns L and the parameter gradients."""
    y, cache = mlp_forward(p, X, rnd)
    m = np.einsum("bmn,bn->bm", Bas, y)
    e = m - T
    B = X.shape[0]
    dy = np.einsum("bmn,bm->bn", Bas, e) * (2.0 / (B * T.shape[1]))
    return float(np.mean(e ** 2)), _backward(p, cache, dy, rnd)


def _backward(p, cache, dy, rnd):
    """Parameter gradients given the output delta dy = dL/dy."""
    r = rnd or (lambda a: a)
    X_, z1, h1, z2, h2 = cache
    g = {}
    g["W3"] = r(h2).T @ r(dy)
    g["b3"] = r(dy).sum(0)
    dh2 = r(dy) @ r(p["W3"]).T
    dz2 = dh2 * gelu_grad(z2)
    g["W2"] = r(h1).T @ r(dz2)
    g["b2"] = r(dz2).sum(0)
    dh1 = r(dz2) @ r(p["W2"]).T
    dz1 = dh1 * gelu_grad(z1)
    g["W1"] = r(X_).T @ r(dz1)
    g["b1"] = r(dz1).sum(0)
    return g


def bf16_round(a):
    """Round float values to bfloat16 (8-bit mantissa, round to nearest even),
    returned as float64; used to feed the oracle the operands a BF16 kernel
    multiplies."""
    f = np.asarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# Closure term and LES right-hand side (L6)
# --------------------------------------------------------------------------

def model_stress(uh, cfg: sp.Config, p, norm, rnd=None):
    """Model stress tau (6, nz, ny, nx) of the state: invariants of its
    gradient, standardised (norm = dict(mean, std, s_tau, s_A)), through the
    MLP (rnd as in mlp_forward), weighting the tensor basis (reading L4)."""
    A = gradient(uh, cfg)
    lam = invariants(A)
    X = ((lam.reshape(5, -1).T - norm["mean"]) / norm["std"])
    y, _ = mlp_forward(p, X, rnd)
    Tb = tensor_basis(A, norm["s_A"]).reshape(6, 6, -1)
    tau = np.einsum("nmp,pn->mp", Tb, y)
    return (tau * norm["s_tau"]).reshape((6,) + lam.shape[1:])


def closure_term(uh, cfg: sp.Config, p, norm, rnd=None):
    """-i k_j tau_hat_ij, masked (reading L6)."""
    tau = model_stress(uh, cfg, p, norm, rnd)
    th = sp.forward(tau)
    k = sp.wavenumbers(cfg)
    full = {}
    for m, (i, j) in enumerate(SYM):
        full[(i, j)] = th[m]
        full[(j, i)] = th[m]
    div = np.stack([sum(1j * k[j] * full[(i, j)] for j in range(3)) for i in range(3)])
    return -div * sp.dealias_mask(cfg)


def force_loss_and_grads(uh, cfg: sp.Config, p, norm, f_hat, rnd=None):
    """Force loss of reading L8 and its parameter gradients by the adjoint:
    r(x) is linear in tau through tau -> D P(-div tau), so
    dL/dtau_ij(x) = (2 / (Nx Ny Nz)) d r_i / d x_j (r already projected and
    masked), summed over (i, j) and (j, i) for a stored off-diagonal
    component; dL/dg_n = s_tau sum_m T_n,m dL/dtau_m per point; the network
    part is the chain rule of mse_and_grads."""
    D = sp.dealias_mask(cfg)
    A = gradient(uh, cfg)
    lam = invariants(A)
    X = (lam.reshape(5, -1).T - norm["mean"]) / norm["std"]
    y, cache = mlp_forward(p, X, rnd)
    Tb = tensor_basis(A, norm["s_A"]).reshape(6, 6, -1)
    tau = norm["s_tau"] * np.einsum("nmp,pn->mp", Tb, y).reshape((6,) + lam.shape[1:])
    th = sp.forward(tau)
    k = sp.wavenumbers(cfg)
    full = {}
    for m, (i, j) in enumerate(SYM):
        full[(i, j)] = th[m]
        full[(j, i)] = th[m]
    div = np.stack([sum(1j * k[j] * full[(i, j)] for j in range(3)) for i in range(3)])
    r_hat = sp.project(-div * D, cfg) * D - np.asarray(f_hat) * D
    w = sp.hermitian_weight(cfg)
    L = float(np.sum(w * np.abs(r_hat) ** 2))
    # d r_i / d x_j on the grid
    G = np.stack([np.stack([sp.inverse((1j * k[j] * r_hat[i])[None], cfg)[0] for j in range(3)])
                  for i in range(3)])
    scale = 2.0 / (cfg.nx * cfg.ny * cfg.nz)
    dtau = np.stack([scale * (G[i, j] + G[j, i]) if i != j else scale * G[i, i] for (i, j) in SYM])
    dy = norm["s_tau"] * np.einsum("nmp,mp->pn", Tb, dtau.reshape(6, -1))
    return L, _backward(p, cache, dy, rnd)


def shell_index(cfg: sp.Config) -> np.ndarray:
    """K = floor(|k| + 1/2) of every stored mode (reading R9)."""
    kx, ky, kz = sp.wavenumbers(cfg)
    return np.floor(np.sqrt(kx * kx + ky * ky + kz * kz) + 0.5).astype(int)


def transfer_spectrum(uh, f_hat, cfg: sp.Config, nshells: int) -> np.ndarray:
    """T(K) = sum_{shell K} w Re(u_hat* . f_hat), K = 0..nshells-1 (reading L9)."""
    w = sp.hermitian_weight(cfg) * sp.dealias_mask(cfg)
    e = (w * np.real(np.conj(uh) * f_hat).sum(0))
    return np.bincount(shell_index(cfg).ravel(), weights=e.ravel(), minlength=nshells)[:nshells]


def transfer_loss_and_grads(uh, cfg: sp.Config, p, norm, T_exact, rnd=None):
    """Transfer loss of reading L9 and its parameter gradients.  dL/df_hat
    has the form of the force-loss gradient with the residual replaced by
    dT(K(k)) u_hat(k), dT = T_model - T_exact, so the adjoint of
    force_loss_and_grads applies to that field unchanged."""
    nsh = len(T_exact)
    D = sp.dealias_mask(cfg)
    A = gradient(uh, cfg)
    lam = invariants(A)
    X = (lam.reshape(5, -1).T - norm["mean"]) / norm["std"]
    y, cache = mlp_forward(p, X, rnd)
    Tb = tensor_basis(A, norm["s_A"]).reshape(6, 6, -1)
    tau = norm["s_tau"] * np.einsum("nmp,pn->mp", Tb, y).reshape((6,) + lam.shape[1:])
    th = sp.forward(tau)
    k = sp.wavenumbers(cfg)
    full = {}
    for m, (i, j) in enumerate(SYM):
        full[(i, j)] = th[m]
        full[(j, i)] = th[m]
    div = np.stack([sum(1j * k[j] * full[(i, j)] for j in range(3)) for i in range(3)])
    f_model = sp.project(-div * D, cfg) * D
    dT = transfer_spectrum(uh * D, f_model, cfg, nsh) - np.asarray(T_exact)
    L = float(np.sum(dT * dT))
    K = shell_index(cfg)
    dTk = np.where(K < nsh, dT[np.minimum(K, nsh - 1)], 0.0)
    r_hat = dTk * uh * D
    G = np.stack([np.stack([sp.inverse((1j * k[j] * r_hat[i])[None], cfg)[0] for j in range(3)])
                  for i in range(3)])
    scale = 2.0 / (cfg.nx * cfg.ny * cfg.nz)
    dtau = np.stack([scale * (G[i, j] + G[j, i]) if i != j else scale * G[i, i] for (i, j) in SYM])
    dy = norm["s_tau"] * np.einsum("nmp,mp->pn", Tb, dtau.reshape(6, -1))
    return L, _backward(p, cache, dy, rnd)


def _les_nonviscous(uh, cfg: sp.Config, p, norm, forcing, rnd):
    """D P(N + f - div tau): the LES right-hand side without the viscous term."""
    D = sp.dealias_mask(cfg)
    v = sp.nonlinear(uh, cfg) + closure_term(uh, cfg, p, norm, rnd)
    if forcing is not None:
        v = v + np.asarray(forcing) * D
    return sp.project(v, cfg) * D


def les_rhs(uh, cfg: sp.Config, p, norm, forcing=None, rnd=None):
    """RHS of the LES: D P(N + f - div tau) - nu |k|^2 D u."""
    kx, ky, kz = sp.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    D = sp.dealias_mask(cfg)
    return _les_nonviscous(uh, cfg, p, norm, forcing, rnd) - cfg.nu * k2 * uh * D


def les_rk_step(uh, dt: float, cfg: sp.Config, p, norm, forcing=None, rnd=None):
    """One IF-RK step of the LES: the scheme of the HD step (Sec. 2) with the
    closure term inside every stage's nonlinear term."""
    kx, ky, kz = sp.wavenumbers(cfg)
    k2 = kx * kx + ky * ky + kz * kz
    E = np.exp(-cfg.nu * k2 * dt / 2.0) + np.zeros_like(uh, dtype=np.float64)
    u = uh * sp.dealias_mask(cfg)
    return sp._lawson_step(u, E, lambda v: _les_nonviscous(v, cfg, p, norm, forcing, rnd), dt, cfg.rk_order)
