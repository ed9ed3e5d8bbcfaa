"""Learned LES closure workflow on the CUDA path.

Everything numerical runs in the library's kernels (include/ps.h): the DNS
and LES time steps, the training pairs (ps_les_training_sample), the box
filter (ps_les_filter), the tensor-basis fit and Adam (ps_mlp_grad_tb,
ps_mlp_adam) and the spectra (ps_diagnostics).  This module only sequences
the calls and keeps a few host-side statistics (normalisation constants,
time averages of spectra).

Workflow (``experiment``):
  1. a forced DNS on n_dns^3 from the seeded field, run past its transient;
  2. training pairs from snapshots of a training window: standardised
     gradient invariants X, gradients A and subgrid stresses T of the field
     box-filtered at kc and sampled on the n_les^3 grid;
  3. full-batch Adam on the tensor-basis loss;
  4. the DNS continues over an evaluation window; the LES (with the trained
     closure, and without any closure) starts from the filtered DNS state at
     the window's start and runs over the same window with a larger step;
  5. time-averaged shell spectra 1 <= K <= kc of LES and DNS are compared
     (the shells K <= kc of the DNS contain only modes inside the filter box,
     so they are the filtered DNS spectrum), and the cost per unit of
     simulated time is compared.
"""

from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs
from . import ps

H, NI, NO = 64, 5, 6
SHAPES = (("W1", (NI, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, NO)), ("b3", (NO,)))


def init_params(seed: int = 0, out_scale: float = 0.1) -> np.ndarray:
    """FP32 parameter vector (layout of ps_mlp_forward): weights normal with
    variance 1/fan_in (the output layer further scaled by out_scale), biases 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in SHAPES:
        if name.startswith("b"):
            parts.append(np.zeros(shape))
        else:
            w = rng.standard_normal(shape) / math.sqrt(shape[0])
            parts.append(w * (out_scale if name == "W3" else 1.0))
    v = np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)
    assert v.size == ps.MLP_NPARAM
    return v


def _torch():
    import torch
    return torch


def training_pairs(uhat_dns, n_dns: int, n_les: int, kc: int, norm=None):
    """(X, A, T) device tensors of one DNS state (see ps_les_training_sample)."""
    torch = _torch()
    P = n_les ** 3
    X = torch.empty((P, NI), device=uhat_dns.device, dtype=torch.float32)
    A = torch.empty((P, 9), device=uhat_dns.device, dtype=torch.float32)
    T = torch.empty((P, NO), device=uhat_dns.device, dtype=torch.float32)
    ps.ps_les_training_sample(n_dns, uhat_dns, n_les, kc, norm, X, A, T)
    return X, A, T


def calibrate(X_raw, A, T) -> dict:
    """Normalisation constants from one sample (host statistics): mean and
    std of the raw invariants, s_A = rms |A|, s_tau = rms of the stress
    components."""
    x = X_raw.double().cpu().numpy()
    a = A.double().cpu().numpy()
    t = T.double().cpu().numpy()
    std = x.std(0)
    std[std == 0] = 1.0
    return dict(mean=x.mean(0), std=std, s_A=float(math.sqrt(np.mean(np.sum(a * a, axis=1)))),
                s_tau=float(math.sqrt(np.mean(t * t))))


def train(params, X, A, T, norm: dict, iters: int = 2000, lr: float = 2e-3, log_every: int = 100):
    """Full-batch Adam on the tensor-basis loss (ps_mlp_grad_tb); cosine decay
    of the learning rate to lr/20.  Returns the logged (iteration, loss)."""
    torch = _torch()
    grad = torch.empty_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.empty(1, device=params.device, dtype=torch.float64)
    log = []
    n = X.shape[0]
    for it in range(1, iters + 1):
        ps.ps_mlp_grad_tb(params, X, A, T, n, norm["s_A"], norm["s_tau"], grad, loss)
        if it == 1 or it % log_every == 0 or it == iters:
            log.append((it, float(loss.item())))
        rate = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * (it - 1) / max(iters - 1, 1))))
        ps.ps_mlp_adam(params, grad, m, v, it, rate)
    return log


def train_force(plan, params, norm: dict, snaps, iters: int = 1000, lr: float = 1e-3, log_every: int = 100):
    """Full-batch Adam on the force loss (ps_plan_closure_grad) summed over
    the snapshots (ubar, exact force); logs the loss relative to the exact
    forces' own mean square (Parseval on the LES grid)."""
    torch = _torch()
    plan.set_closure(params, norm)
    grad = torch.empty_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.empty(1, device=params.device, dtype=torch.float64)
    zero = torch.zeros(ps.MLP_NPARAM, device=params.device, dtype=torch.float32)
    # the exact forces' mean square: the loss of the zero network
    z = torch.empty_like(loss)
    for k, (ub, f) in enumerate(snaps):
        plan.closure_grad(zero, ub, f, grad, z, accumulate=k > 0)
    ref = float(z.item())
    log = []
    for it in range(1, iters + 1):
        for k, (ub, f) in enumerate(snaps):
            plan.closure_grad(params, ub, f, grad, loss, accumulate=k > 0)
        if it == 1 or it % log_every == 0 or it == iters:
            log.append((it, float(loss.item()) / ref))
        rate = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * (it - 1) / max(iters - 1, 1))))
        ps.ps_mlp_adam(params, grad, m, v, it, rate)
    plan.set_closure(None)
    return log


def train_transfer(plan, params, norm: dict, snaps, iters: int = 500, lr: float = 1e-3, log_every: int = 50):
    """Full-batch Adam on the energy-transfer loss (ps_plan_closure_grad_transfer)
    summed over the snapshots (ubar, exact transfer T(K)); logs the loss
    relative to that of the zero network."""
    torch = _torch()
    plan.set_closure(params, norm)
    grad = torch.empty_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.empty(1, device=params.device, dtype=torch.float64)
    ref = sum(float(np.sum(np.asarray(te) ** 2)) for _, te in snaps)
    log = []
    for it in range(1, iters + 1):
        for k, (ub, te) in enumerate(snaps):
            plan.closure_grad_transfer(params, ub, te, grad, loss, accumulate=k > 0)
        if it == 1 or it % log_every == 0 or it == iters:
            log.append((it, float(loss.item()) / ref))
        rate = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * (it - 1) / max(iters - 1, 1))))
        ps.ps_mlp_adam(params, grad, m, v, it, rate)
    plan.set_closure(None)
    return log


def shell_transfer(uhat, force, kc: int) -> np.ndarray:
    """Energy transfer spectrum T(K) = sum over shell K of w Re(conj(u) . f)
    (w = 1 on the kx = 0 plane and, for an even grid, the kx = n/2 plane,
    2 elsewhere) for K = 0..kc; host analysis of small LES-grid fields."""
    u = uhat.cpu().numpy().astype(np.complex128)
    f = force.cpu().numpy().astype(np.complex128)
    n = u.shape[1]
    q = np.fft.fftfreq(n, 1.0 / n)
    kz, ky, kx = np.meshgrid(q, q, np.arange(u.shape[3]), indexing="ij")
    shell = np.floor(np.sqrt(kx * kx + ky * ky + kz * kz) + 0.5).astype(int)
    w = np.where((kx == 0) | ((n % 2 == 0) & (kx == n // 2)), 1.0, 2.0)
    e = (w * np.real(np.conj(u) * f).sum(0)).ravel()
    return np.bincount(shell.ravel(), weights=e, minlength=kc + 1)[:kc + 1]


def sgs_force(dns_plan, les_plan, uhat_dns, n_dns: int, n_les: int, kc: int, closure=None):
    """Exact subgrid force of the filtered state, F[rhs_DNS(u)] - rhs_LES(ubar),
    and (if a closure (params, norm) is given) the model's force; both are
    projected and band-limited.  Returns (ubar, exact, model or None)."""
    torch = _torch()
    shape = (3, n_les, n_les, n_les // 2 + 1)
    ubar = torch.zeros(shape, device=uhat_dns.device, dtype=torch.complex64)
    ps.ps_les_filter(n_dns, uhat_dns, n_les, kc, ubar)
    r_dns = dns_plan.rhs(uhat_dns)
    exact = torch.zeros(shape, device=uhat_dns.device, dtype=torch.complex64)
    ps.ps_les_filter(n_dns, r_dns, n_les, kc, exact)
    del r_dns
    les_plan.set_closure(None)
    r0 = les_plan.rhs(ubar)
    exact -= r0
    model = None
    if closure is not None:
        les_plan.set_closure(*closure)
        model = les_plan.rhs(ubar) - r0
        les_plan.set_closure(None)
    return ubar, exact, model


def _spectrum(plan, u, kc: int):
    d = plan.diagnostics(u)
    return np.asarray(d["spectrum"][:kc + 1]), d


def _timed_steps(plan, u, dt: float, nsteps: int, t0: float) -> float:
    """Wall time of nsteps steps (replayed as one captured graph, see
    ps_rk_steps; the first call of a given length includes its capture)."""
    torch = _torch()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    plan.rk_steps(u, dt, nsteps, t=t0)
    torch.cuda.synchronize()
    return time.perf_counter() - w0


def experiment(n_dns=512, n_les=64, kc=21, nu=2e-3, dt_dns=1e-3, dt_les=5e-3, t_spin=8.0, t_train=2.0,
               n_snap=8, t_eval=5.0, n_eval=10, iters=2000, lr=2e-3, fit="both", force_iters=1000,
               force_lr=1e-3, drain_only=False, seed=1, verbose=True, points_per_snap=0) -> dict:
    """Runs the workflow of the module docstring; fit = "stress" (tensor-basis
    stress loss), "force" (stress fit refined on the force loss), "transfer"
    (stress fit refined on the shell energy-transfer loss) or "both" (all
    three models evaluated).  points_per_snap > 0 keeps that many LES grid
    points of every snapshot for the stress fit (the same seeded subset each
    time; 0 keeps all n_les^3)."""
    torch = _torch()
    dev = "cuda"
    say = print if verbose else (lambda *a, **k: None)
    t_wall = time.perf_counter()
    f_dns = torch.from_numpy(inputs.forcing_field(n_dns, n_dns, n_dns, seed=2)).to(dev, torch.complex64)
    u = torch.from_numpy(inputs.random_solenoidal_field(n_dns, n_dns, n_dns, seed=seed)).to(dev, torch.complex64)
    dns = ps.Plan(n_dns, prec=ps.Precision.FP32, nu=nu, rk_order=4, forcing=f_dns)
    t = 0.0
    out = dict(n_dns=n_dns, n_les=n_les, kc=kc, nu=nu, dt_dns=dt_dns, dt_les=dt_les, t_spin=t_spin, points_per_snap=points_per_snap,
               t_train=t_train, n_snap=n_snap, t_eval=t_eval, n_eval=n_eval, iters=iters, lr=lr)
    # 1. spin-up (energy recorded every half time unit)
    n_spin = int(round(t_spin / dt_dns))
    chunk = max(1, int(round(0.5 / dt_dns)))
    series = [(t, dns.diagnostics(u)["energy"])]
    done = 0
    while done < n_spin:
        k = min(chunk, n_spin - done)
        _timed_steps(dns, u, dt_dns, k, t)
        t += k * dt_dns
        done += k
        series.append((t, dns.diagnostics(u)["energy"]))
    out["dns_energy_series"] = series
    d0 = dns.diagnostics(u)
    say(f"spin-up to t={t:.2f}: E={d0['energy']:.4f} Omega={d0['enstrophy']:.2f} max|u|={d0['max_u']:.3f}")
    out["dns_after_spinup"] = dict(energy=d0["energy"], enstrophy=d0["enstrophy"], max_u=d0["max_u"])
    # 2. training data over the training window: stress pairs (X, A, T) and,
    #    for the force fit, the filtered state with its exact subgrid force
    f_les = torch.from_numpy(inputs.forcing_field(n_les, n_les, n_les, seed=2)).to(dev, torch.complex64)
    les_plan = ps.Plan(n_les, prec=ps.Precision.FP32, nu=nu, rk_order=4, forcing=f_les)
    gap = int(round(t_train / n_snap / dt_dns))
    Xr, A, T = training_pairs(u, n_dns, n_les, kc)
    norm = calibrate(Xr, A, T)
    del Xr
    Xs, As, Ts, snaps = [], [], [], []
    keep = None
    if 0 < points_per_snap < n_les ** 3:
        g = torch.Generator(device="cpu").manual_seed(seed)
        keep = torch.randperm(n_les ** 3, generator=g)[:points_per_snap].to(dev)
    for k in range(n_snap):
        X, A, T = training_pairs(u, n_dns, n_les, kc, norm)
        if keep is not None:
            X, A, T = X[keep], A[keep], T[keep]
        Xs.append(X)
        As.append(A)
        Ts.append(T)
        if fit in ("force", "transfer", "both"):
            ubar, exact, _ = sgs_force(dns, les_plan, u, n_dns, n_les, kc)
            snaps.append((ubar, exact))
        _timed_steps(dns, u, dt_dns, gap, t)
        t += gap * dt_dns
    X, A, T = torch.cat(Xs), torch.cat(As), torch.cat(Ts)
    del Xs, As, Ts
    say(f"training pairs: {X.shape[0]} points from {n_snap} snapshots; s_A={norm['s_A']:.3f} s_tau={norm['s_tau']:.4g}")
    # 3. fit: stress (tensor-basis MSE), then optionally the force loss
    params = torch.from_numpy(init_params(seed)).to(dev)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    log = train(params, X, A, T, norm, iters=iters, lr=lr)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - w0
    # the target's own mean square in units of s_tau^2 (1 by construction
    # of s_tau on the calibration sample)
    tt = (T.double() / norm["s_tau"]).pow(2).mean().item()
    out["fit"] = dict(loss_log=log, target_mean_square=tt, explained=1.0 - log[-1][1] / tt, seconds=t_fit,
                      samples=int(X.shape[0]))
    say(f"stress fit: loss {log[0][1]:.4f} -> {log[-1][1]:.4f} (target mean square {tt:.4f}) in {t_fit:.1f} s")
    del X, A, T
    out["norm"] = {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in norm.items()}
    models = {"learned_stress": params}
    if fit in ("force", "both"):
        pf = params.clone()
        w0 = time.perf_counter()
        flog = train_force(les_plan, pf, norm, snaps, iters=force_iters, lr=force_lr)
        torch.cuda.synchronize()
        out["force_fit"] = dict(loss_log=flog, seconds=time.perf_counter() - w0)
        say(f"force fit: relative loss {flog[0][1]:.4f} -> {flog[-1][1]:.4f}")
        models = {"learned_force": pf} if fit == "force" else {"learned_stress": params, "learned_force": pf}
    if fit in ("transfer", "both"):
        pt = params.clone()
        nsh = int(math.ceil(math.sqrt(3.0) * kc)) + 1  # every shell of the retained cube
        tsnaps = [(ub, shell_transfer(ub, ex, nsh)) for ub, ex in snaps]
        if drain_only:  # target the drain alone: min(T_exact, 0) per shell
            tsnaps = [(ub, np.minimum(te, 0.0)) for ub, te in tsnaps]
        w0 = time.perf_counter()
        tlog = train_transfer(les_plan, pt, norm, tsnaps, iters=force_iters, lr=force_lr)
        torch.cuda.synchronize()
        out["transfer_fit"] = dict(loss_log=tlog, seconds=time.perf_counter() - w0)
        say(f"transfer fit: relative loss {tlog[0][1]:.4f} -> {tlog[-1][1]:.4f}")
        if fit == "transfer":
            models = {"learned_transfer": pt}
        else:
            models["learned_transfer"] = pt
    del snaps
    # 4. evaluation window: LES initial state, a-priori energy transfer of
    #    the exact and the modelled subgrid force, DNS spectra
    les0, exact, _ = sgs_force(dns, les_plan, u, n_dns, n_les, kc)
    out["transfer"] = dict(exact=shell_transfer(les0, exact, kc).tolist())
    say("SGS transfer exact: " + " ".join(f"{x:+.2e}" for x in out["transfer"]["exact"][1:]))
    for name, pm in models.items():
        _, _, model = sgs_force(dns, les_plan, u, n_dns, n_les, kc, closure=(pm, norm))
        out["transfer"][name] = shell_transfer(les0, model, kc).tolist()
        say(f"SGS transfer {name}: " + " ".join(f"{x:+.2e}" for x in out["transfer"][name][1:]))
    les_plan.close()
    del exact
    t_eval0 = t
    n_dns_eval = int(round(t_eval / dt_dns))
    per = n_dns_eval // n_eval
    spec_dns = []
    secs_dns = 0.0
    e_dns, eps_dns = [], []
    for k in range(n_eval):
        secs_dns += _timed_steps(dns, u, dt_dns, per, t)
        t += per * dt_dns
        s, d = _spectrum(dns, u, kc)
        spec_dns.append(s)
        e_dns.append(d["energy"])
        eps_dns.append(2.0 * nu * d["enstrophy"])  # dissipation rate of the DNS
    dns.close()
    del u, f_dns
    torch.cuda.empty_cache()
    dns_ms = 1e3 * secs_dns / (per * n_eval)
    les_per = int(round(per * dt_dns / dt_les))
    runs = {}
    for name, closure in list(models.items()) + [("no_model", None)]:
        plan = ps.Plan(n_les, prec=ps.Precision.FP32, nu=nu, rk_order=4, forcing=f_les)
        if closure is not None:
            plan.set_closure(closure, norm)
        ul = les0.clone()
        spec, en, eps, secs, tl, ok = [], [], [], 0.0, t_eval0, True
        for k in range(n_eval):
            dts = _timed_steps(plan, ul, dt_les, les_per, tl)
            if k > 0:  # the first chunk includes the graph capture
                secs += dts
            tl += les_per * dt_les
            s, d = _spectrum(plan, ul, kc)
            if d["status"] != ps.PS_OK or not np.all(np.isfinite(s)):
                ok = False
                break
            spec.append(s)
            en.append(d["energy"])
            # dissipation: resolved 2 nu Omega plus the energy the closure
            # removes, -sum_k w Re(u* . f_closure)
            drain = 0.0
            if closure is not None:
                plan.set_closure(None)
                r0 = plan.rhs(ul)
                plan.set_closure(closure, norm)
                drain = -float(shell_transfer(ul, plan.rhs(ul) - r0, ul.shape[1]).sum())
            eps.append(2.0 * nu * d["enstrophy"] + drain)
        plan.close()
        r = dict(finite=ok, ms_per_step=1e3 * secs / max(les_per * (len(spec) - 1), 1), steps=les_per * n_eval,
                 energy=en, dissipation=eps)
        if ok:
            r["dissipation_rel_err"] = float(abs(np.mean(eps) - np.mean(eps_dns)) / np.mean(eps_dns))
        if ok:
            E_les = np.mean(spec, axis=0)[1:]
            E_dns = np.mean(spec_dns, axis=0)[1:]
            rel = np.abs(E_les - E_dns) / E_dns
            r.update(spectrum=E_les.tolist(), rel_err=rel.tolist(), max_rel_err=float(rel.max()),
                     mean_rel_err=float(rel.mean()))
            say(f"LES {name}: max rel. spectrum error {rel.max():.3f} (mean {rel.mean():.3f}), "
                f"dissipation {np.mean(eps):.4f} vs DNS {np.mean(eps_dns):.4f}, {r['ms_per_step']:.3f} ms/step")
        else:
            say(f"LES {name}: non-finite state")
        runs[name] = r
    les_ms = runs[next(iter(models))]["ms_per_step"]
    # sampling uncertainty of the DNS time mean per shell: the standard error
    # of the mean of the n_eval samples, and the difference of the means of
    # the two halves of the window (both relative to the mean)
    sd = np.asarray(spec_dns)[:, 1:]
    mean_d = sd.mean(axis=0)
    stat = sd.std(axis=0, ddof=1) / np.sqrt(sd.shape[0]) / mean_d
    half = np.abs(sd[: sd.shape[0] // 2].mean(axis=0) - sd[sd.shape[0] // 2:].mean(axis=0)) / mean_d
    out["dns"] = dict(ms_per_step=dns_ms, spectrum=mean_d.tolist(), steps=per * n_eval,
                      energy=e_dns, dissipation=eps_dns, stat_rel_err=stat.tolist(),
                      max_stat_rel_err=float(stat.max()), half_window_rel_diff=half.tolist(),
                      max_half_window_rel_diff=float(half.max()))
    say(f"DNS time-mean spectrum: standard error up to {stat.max():.3f} (mean {stat.mean():.3f}), "
        f"half-window difference up to {half.max():.3f}")
    out["les"] = runs
    out["cost_ratio"] = (dns_ms / dt_dns) / (les_ms / dt_les) if les_ms > 0 else None
    out["wall_seconds"] = time.perf_counter() - t_wall
    say(f"cost per unit time: DNS/LES = {out['cost_ratio']:.1f}")
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="Learned LES closure: DNS data, fit, a posteriori LES")
    ap.add_argument("--n-dns", type=int, default=512)
    ap.add_argument("--n-les", type=int, default=64)
    ap.add_argument("--kc", type=int, default=21)
    ap.add_argument("--nu", type=float, default=2e-3)
    ap.add_argument("--dt-dns", type=float, default=1e-3)
    ap.add_argument("--dt-les", type=float, default=5e-3)
    ap.add_argument("--t-spin", type=float, default=8.0)
    ap.add_argument("--t-train", type=float, default=2.0)
    ap.add_argument("--n-snap", type=int, default=8)
    ap.add_argument("--t-eval", type=float, default=5.0)
    ap.add_argument("--n-eval", type=int, default=10)
    ap.add_argument("--iters", type=int, default=2000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--fit", choices=("stress", "force", "transfer", "both"), default="both")
    ap.add_argument("--force-iters", type=int, default=1000)
    ap.add_argument("--force-lr", type=float, default=1e-3)
    ap.add_argument("--drain-only", action="store_true", help="transfer fit: target min(T_exact, 0) per shell")
    ap.add_argument("--points-per-snap", type=int, default=0,
                    help="stress fit: LES grid points kept per snapshot (0 = all)")
    ap.add_argument("--out", default=None, help="write the result as JSON here")
    a = ap.parse_args(argv)
    r = experiment(n_dns=a.n_dns, n_les=a.n_les, kc=a.kc, nu=a.nu, dt_dns=a.dt_dns, dt_les=a.dt_les,
                   t_spin=a.t_spin, t_train=a.t_train, n_snap=a.n_snap, t_eval=a.t_eval, n_eval=a.n_eval,
                   iters=a.iters, lr=a.lr, fit=a.fit, force_iters=a.force_iters, force_lr=a.force_lr,
                   drain_only=a.drain_only, points_per_snap=a.points_per_snap)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(r, fh, indent=1)
    return r


if __name__ == "__main__":
    main()
