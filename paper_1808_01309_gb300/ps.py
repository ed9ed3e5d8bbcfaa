"""ctypes binding of libps.so (include/ps.h): argument marshalling only.

Every step of the right-hand side and of the Runge-Kutta step runs in the
library's CUDA kernels; torch is used for device buffers and streams.  If the
library is missing the import fails: there is no fallback.
"""

from __future__ import annotations

import ctypes
import enum
import math
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libps.so")


class PsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class Precision(enum.IntEnum):
    FP32 = 0
    FP64 = 1


class Equations(enum.IntEnum):
    HD = 0
    MHD = 1
    BOUSSINESQ = 2


class Dealias(enum.IntEnum):
    CUBIC = 0
    SPHERICAL = 1
    NONE = 2


PS_OK, PS_ERR_INVALID_ARG, PS_ERR_UNSUPPORTED, PS_ERR_OOM, PS_ERR_CUDA, PS_ERR_NONFINITE, PS_ERR_TIMEOUT = range(7)
_STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "out of memory", 4: "CUDA error",
           5: "non-finite", 6: "timeout"}
PS_NKINDS = 7

# Exported symbols and their signatures (kept in step with include/ps.h).
SYMBOLS = (
    "ps_plan_create", "ps_plan_destroy", "ps_plan_workspace_bytes", "ps_rhs", "ps_rk_step",
    "ps_rk_step_host", "ps_step_stats", "ps_diagnostics", "ps_plan_set_timing",
    "ps_plan_get_timing", "ps_plan_launch_count", "ps_kind_name", "ps_status_string",
    "ps_last_error", "ps_rhs_noalloc", "ps_ensemble_create", "ps_ensemble_destroy",
    "ps_ensemble_rk_steps", "ps_ensemble_tune", "ps_mlp_forward", "ps_mlp_grad", "ps_mlp_adam",
    "ps_plan_set_closure", "ps_les_training_sample", "ps_mlp_grad_tb",
    "ps_les_filter", "ps_mlp_backward", "ps_plan_closure_grad", "ps_plan_set_host_mode", "ps_rk_steps",
    "ps_plan_closure_grad_transfer", "ps_checkpoint_save", "ps_checkpoint_load", "ps_checkpoint_info",
    "ps_fft_r2c", "ps_fft_c2r", "ps_probe_fma_tflops", "ps_plan_set_wait_test",
    "ps_slab_create", "ps_slab_destroy", "ps_slab_info_get", "ps_slab_inverse", "ps_slab_xpass",
    "ps_slab_forward", "ps_slab_check", "ps_ensemble_check", "ps_ensemble_set_wait_test",
    "ps_plan_set_pass_shape",
)
HOST_AUTO, HOST_COPY, HOST_MAPPED, HOST_SMCOPY, HOST_CUBE_CE = 0, 1, 2, 3, 4
MLP_NPARAM = 4934
ENS_SEQUENTIAL, ENS_GRAPH, ENS_PERSISTENT, ENS_AUTO, ENS_BATCHED = 0, 1, 2, 3, 4
ENS_PASSES = ("z_inverse", "y_inverse", "x_fused", "y_forward", "z_forward", "update")
ENS_MAX_SIZES = 8
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


class PsConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("prec", ctypes.c_int), ("eq", ctypes.c_int), ("dealias", ctypes.c_int),
        ("rk_order", ctypes.c_int),
        ("nu", ctypes.c_double), ("eta", ctypes.c_double),
        ("forcing", ctypes.c_void_p),
        ("n_bv", ctypes.c_double), ("kappa", ctypes.c_double),
    ]


class PsDiag(ctypes.Structure):
    _fields_ = [
        ("energy", ctypes.c_double), ("enstrophy", ctypes.c_double), ("helicity", ctypes.c_double),
        ("max_div", ctypes.c_double), ("max_u", ctypes.c_double), ("cfl_dt", ctypes.c_double),
        ("time", ctypes.c_double),
        ("spectrum", ctypes.POINTER(ctypes.c_double)), ("nshells", ctypes.c_int),
        ("magnetic_energy", ctypes.c_double), ("cross_helicity", ctypes.c_double),
        ("magnetic_helicity", ctypes.c_double),
        ("potential_energy", ctypes.c_double),
    ]


class PsEnsTuning(ctypes.Structure):
    _fields_ = [("branches", ctypes.c_int), ("nsizes", ctypes.c_int), ("n", ctypes.c_int * 8),
                ("xrpc", ctypes.c_int * 8), ("step_ms", ctypes.c_double),
                ("pass_cols", (ctypes.c_int * 3) * 8), ("pass_points", (ctypes.c_int * 3) * 8),
                ("persistent_step_ms", ctypes.c_double),
                ("persistent_ctas_per_sm", ctypes.c_int), ("persistent_order", ctypes.c_int),
                ("persistent_tiles_per_item", ctypes.c_int * 6), ("batched_step_ms", ctypes.c_double),
                ("batched_members_per_launch", ctypes.c_int), ("best_mode", ctypes.c_int)]


class PsSlabInfo(ctypes.Structure):
    _fields_ = [("ncx", ctypes.c_int), ("kxp", ctypes.c_int), ("cxp", ctypes.c_int), ("rows", ctypes.c_int)]


class PsTiming(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * PS_NKINDS), ("launches", ctypes.c_longlong * PS_NKINDS)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libps.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(the CUDA path has no fallback)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.ps_plan_create.argtypes = [ctypes.POINTER(PsConfig), P, ctypes.POINTER(P)]
    lib.ps_plan_destroy.argtypes = [P]
    lib.ps_plan_workspace_bytes.argtypes = [ctypes.POINTER(PsConfig), ctypes.POINTER(ctypes.c_size_t)]
    lib.ps_rhs.argtypes = [P, P, P, ctypes.c_double]
    lib.ps_rk_step.argtypes = [P, P, ctypes.c_double, ctypes.c_double]
    lib.ps_rk_step_host.argtypes = [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.ps_step_stats.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.ps_diagnostics.argtypes = [P, P, ctypes.c_double, ctypes.POINTER(PsDiag)]
    lib.ps_plan_set_timing.argtypes = [P, ctypes.c_int]
    lib.ps_plan_get_timing.argtypes = [P, ctypes.POINTER(PsTiming)]
    lib.ps_plan_launch_count.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    lib.ps_rhs_noalloc.argtypes = [ctypes.POINTER(PsConfig), P, P, P, ctypes.c_double]
    lib.ps_ensemble_create.argtypes = [ctypes.POINTER(PsConfig), ctypes.c_int, P, ctypes.POINTER(P)]
    lib.ps_ensemble_destroy.argtypes = [P]
    lib.ps_ensemble_rk_steps.argtypes = [P, ctypes.POINTER(P), ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int]
    lib.ps_ensemble_tune.argtypes = [P, ctypes.POINTER(P), ctypes.c_double, ctypes.POINTER(PsEnsTuning)]
    lib.ps_ensemble_check.argtypes = [P]
    lib.ps_plan_set_pass_shape.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]
    lib.ps_ensemble_set_wait_test.argtypes = [P, ctypes.c_uint]
    lib.ps_mlp_forward.argtypes = [P, P, P, ctypes.c_longlong, P]
    lib.ps_mlp_grad.argtypes = [P, P, P, ctypes.c_longlong, P, P, P]
    lib.ps_mlp_adam.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, P]
    lib.ps_plan_set_closure.argtypes = [P, P, ctypes.POINTER(ctypes.c_double)]
    lib.ps_les_training_sample.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double), P, P, P, P]
    lib.ps_plan_set_host_mode.argtypes = [P, ctypes.c_int]
    lib.ps_plan_closure_grad_transfer.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_double), ctypes.c_int, P, P,
                                                  ctypes.c_int]
    lib.ps_rk_steps.argtypes = [P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.ps_checkpoint_save.argtypes = [P, P, ctypes.c_double, ctypes.c_longlong, ctypes.c_char_p]
    lib.ps_fft_r2c.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
    lib.ps_fft_c2r.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
    lib.ps_checkpoint_load.argtypes = [P, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.c_char_p]
    lib.ps_checkpoint_info.argtypes = [ctypes.c_char_p, ctypes.POINTER(PsConfig), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_longlong)]
    lib.ps_mlp_backward.argtypes = [P, P, P, ctypes.c_longlong, P, P]
    lib.ps_plan_closure_grad.argtypes = [P, P, P, P, P, P, ctypes.c_int]
    lib.ps_les_filter.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, P]
    lib.ps_mlp_grad_tb.argtypes = [P, P, P, P, ctypes.c_longlong, ctypes.c_double, ctypes.c_double, P, P, P]
    lib.ps_probe_fma_tflops.argtypes = [ctypes.c_int, P, ctypes.POINTER(ctypes.c_double)]
    lib.ps_plan_set_wait_test.argtypes = [P, ctypes.c_int]
    lib.ps_slab_create.argtypes = [ctypes.POINTER(PsConfig), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   P, ctypes.POINTER(P)]
    lib.ps_slab_destroy.argtypes = [P]
    lib.ps_slab_info_get.argtypes = [P, ctypes.POINTER(PsSlabInfo)]
    lib.ps_slab_inverse.argtypes = [P, P, P]
    lib.ps_slab_xpass.argtypes = [P, P, P]
    lib.ps_slab_forward.argtypes = [P, P, P, P]
    lib.ps_slab_check.argtypes = [P]
    for name in SYMBOLS:
        fn = getattr(lib, name)
        if name in ("ps_kind_name", "ps_status_string", "ps_last_error"):
            fn.restype = ctypes.c_char_p
        else:
            fn.restype = ctypes.c_int
    lib.ps_kind_name.argtypes = [ctypes.c_int]
    lib.ps_status_string.argtypes = [ctypes.c_int]
    lib.ps_last_error.argtypes = []
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != PS_OK:
        msg = load().ps_last_error().decode(errors="replace")
        raise PsError(status, msg)


def make_config(nx, ny=None, nz=None, *, lx=2 * math.pi, ly=2 * math.pi, lz=2 * math.pi,
                prec=Precision.FP32, eq=Equations.HD, dealias=Dealias.CUBIC, rk_order=4,
                nu=0.0, eta=0.0, forcing=None, n_bv=0.0, kappa=0.0) -> PsConfig:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    fptr = None
    if forcing is not None:
        fptr = forcing.data_ptr() if hasattr(forcing, "data_ptr") else int(forcing)
    return PsConfig(int(nx), int(ny), int(nz), float(lx), float(ly), float(lz), int(prec), int(eq),
                    int(dealias), int(rk_order), float(nu), float(eta), fptr, float(n_bv), float(kappa))


def _ptr(t) -> int:
    return t.data_ptr() if hasattr(t, "data_ptr") else int(t)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---- functions with the C names -------------------------------------------------

def ps_plan_create(cfg: PsConfig, stream=None) -> ctypes.c_void_p:
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.ps_plan_create(ctypes.byref(cfg), _stream_handle(stream), ctypes.byref(h)))
    return h


def ps_plan_destroy(plan) -> None:
    _check(load().ps_plan_destroy(plan))


def ps_plan_workspace_bytes(cfg: PsConfig) -> int:
    n = ctypes.c_size_t()
    _check(load().ps_plan_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def ps_rhs(plan, uhat, rhs_out, t: float = 0.0) -> None:
    _check(load().ps_rhs(plan, _ptr(uhat), _ptr(rhs_out), float(t)))


def ps_rhs_noalloc(cfg: PsConfig, uhat, rhs_out, t: float = 0.0, stream=None) -> None:
    """Right-hand side without a plan and without allocating (static scratch)."""
    _check(load().ps_rhs_noalloc(ctypes.byref(cfg), _stream_handle(stream), _ptr(uhat), _ptr(rhs_out), float(t)))


def ps_rk_step(plan, uhat, dt: float, t: float = 0.0) -> None:
    _check(load().ps_rk_step(plan, _ptr(uhat), float(dt), float(t)))


def ps_rk_steps(plan, uhat, dt: float, t: float = 0.0, nsteps: int = 1) -> None:
    _check(load().ps_rk_steps(plan, _ptr(uhat), float(dt), float(t), int(nsteps)))


def ps_rk_step_host(plan, uhat_host, dt: float, t: float = 0.0, nsteps: int = 1) -> None:
    _check(load().ps_rk_step_host(plan, _ptr(uhat_host), float(dt), float(t), int(nsteps)))


def ps_slab_create(cfg: PsConfig, kx_lo: int, kx_hi: int, z_lo: int, z_hi: int, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().ps_slab_create(ctypes.byref(cfg), int(kx_lo), int(kx_hi), int(z_lo), int(z_hi),
                                 _stream_handle(stream), ctypes.byref(h)))
    return h


def ps_slab_destroy(slab) -> None:
    _check(load().ps_slab_destroy(slab))


def ps_slab_info_get(slab) -> PsSlabInfo:
    info = PsSlabInfo()
    _check(load().ps_slab_info_get(slab, ctypes.byref(info)))
    return info


def ps_slab_inverse(slab, uhat_local, out6) -> None:
    _check(load().ps_slab_inverse(slab, _ptr(uhat_local), _ptr(out6)))


def ps_slab_xpass(slab, xin, xout) -> None:
    _check(load().ps_slab_xpass(slab, _ptr(xin), _ptr(xout)))


def ps_slab_forward(slab, yin, uhat_local, rhs_local) -> None:
    _check(load().ps_slab_forward(slab, _ptr(yin), _ptr(uhat_local), _ptr(rhs_local)))


def ps_slab_check(slab) -> None:
    _check(load().ps_slab_check(slab))


def ps_plan_set_wait_test(plan, polls: int) -> None:
    """Test hook: the x pass waits for a copy that never comes and gives up
    after `polls` polls (0 turns the hook off)."""
    _check(load().ps_plan_set_wait_test(plan, int(polls)))


def ps_plan_set_pass_shape(plan, pass_: int, variant: int) -> tuple[int, int]:
    """Tile shape variant of a column pass (0 z-inverse, 1 y passes, 2 z-forward);
    returns (kx columns per CTA, points per thread)."""
    c, e = ctypes.c_int(), ctypes.c_int()
    _check(load().ps_plan_set_pass_shape(plan, int(pass_), int(variant), ctypes.byref(c), ctypes.byref(e)))
    return c.value, e.value


def ps_probe_fma_tflops(prec: int, stream=None) -> float:
    """Measured FMA rate of the device in TFLOP/s (FP32 or FP64)."""
    out = ctypes.c_double()
    _check(load().ps_probe_fma_tflops(int(prec), _stream_handle(stream), ctypes.byref(out)))
    return out.value


def ps_fft_r2c(n: int, nfields: int, phys, spec, stream=None) -> None:
    _check(load().ps_fft_r2c(int(n), int(nfields), _ptr(phys), _ptr(spec), _stream_handle(stream)))


def ps_fft_c2r(n: int, nfields: int, spec, phys, stream=None) -> None:
    _check(load().ps_fft_c2r(int(n), int(nfields), _ptr(spec), _ptr(phys), _stream_handle(stream)))


def ps_checkpoint_save(plan, uhat, t: float, step: int, path: str) -> None:
    _check(load().ps_checkpoint_save(plan, _ptr(uhat), float(t), int(step), os.fsencode(path)))


def ps_checkpoint_load(plan, uhat, path: str) -> tuple[float, int]:
    t, step = ctypes.c_double(), ctypes.c_longlong()
    _check(load().ps_checkpoint_load(plan, _ptr(uhat), ctypes.byref(t), ctypes.byref(step), os.fsencode(path)))
    return t.value, step.value


def ps_checkpoint_info(path: str) -> tuple[PsConfig, float, int]:
    cfg, t, step = PsConfig(), ctypes.c_double(), ctypes.c_longlong()
    _check(load().ps_checkpoint_info(os.fsencode(path), ctypes.byref(cfg), ctypes.byref(t), ctypes.byref(step)))
    return cfg, t.value, step.value


def ps_plan_set_host_mode(plan, mode: int) -> None:
    _check(load().ps_plan_set_host_mode(plan, int(mode)))


def ps_step_stats(plan) -> tuple[float, float]:
    e, m = ctypes.c_double(), ctypes.c_double()
    _check(load().ps_step_stats(plan, ctypes.byref(e), ctypes.byref(m)))
    return e.value, m.value


def ps_diagnostics(plan, uhat, cfl: float = 0.5, nshells: int = 4096) -> dict:
    spec = (ctypes.c_double * max(nshells, 1))()
    d = PsDiag()
    d.spectrum = ctypes.cast(spec, ctypes.POINTER(ctypes.c_double))
    d.nshells = nshells
    st = load().ps_diagnostics(plan, _ptr(uhat), float(cfl), ctypes.byref(d))
    out = dict(energy=d.energy, enstrophy=d.enstrophy, helicity=d.helicity, max_div=d.max_div,
               max_u=d.max_u, cfl_dt=d.cfl_dt, time=d.time, magnetic_energy=d.magnetic_energy,
               cross_helicity=d.cross_helicity, magnetic_helicity=d.magnetic_helicity,
               potential_energy=d.potential_energy,
               spectrum=[spec[i] for i in range(min(d.nshells, nshells))], status=st)
    if st not in (PS_OK, PS_ERR_NONFINITE):
        _check(st)
    return out


def ps_plan_set_timing(plan, enable: bool) -> None:
    _check(load().ps_plan_set_timing(plan, 1 if enable else 0))


def ps_plan_get_timing(plan) -> dict:
    t = PsTiming()
    _check(load().ps_plan_get_timing(plan, ctypes.byref(t)))
    lib = load()
    return {lib.ps_kind_name(k).decode(): (t.ms[k], t.launches[k]) for k in range(PS_NKINDS)}


def ps_plan_launch_count(plan) -> int:
    n = ctypes.c_longlong()
    _check(load().ps_plan_launch_count(plan, ctypes.byref(n)))
    return n.value


def ps_ensemble_create(cfgs, stream=None) -> ctypes.c_void_p:
    arr = (PsConfig * len(cfgs))(*cfgs)
    h = ctypes.c_void_p()
    _check(load().ps_ensemble_create(arr, len(cfgs), _stream_handle(stream), ctypes.byref(h)))
    return h


def ps_ensemble_destroy(ens) -> None:
    _check(load().ps_ensemble_destroy(ens))


def _ptr_array(states):
    return (ctypes.c_void_p * len(states))(*[_ptr(s) for s in states])


def ps_ensemble_rk_steps(ens, states, dt: float, t: float = 0.0, nsteps: int = 1, mode: int = ENS_GRAPH) -> None:
    _check(load().ps_ensemble_rk_steps(ens, _ptr_array(states), float(dt), float(t), int(nsteps), int(mode)))


def ps_ensemble_tune(ens, states, dt: float) -> dict:
    t = PsEnsTuning()
    _check(load().ps_ensemble_tune(ens, _ptr_array(states), float(dt), ctypes.byref(t)))
    return {"branches": t.branches, "step_ms": t.step_ms,
            "xrpc": {int(t.n[i]): int(t.xrpc[i]) for i in range(t.nsizes)},
            "pass_shapes": {int(t.n[i]): {p: (int(t.pass_cols[i][k]), int(t.pass_points[i][k]))
                                          for k, p in enumerate(("z_inverse", "y_passes", "z_forward"))}
                            for i in range(t.nsizes)},
            "persistent_step_ms": t.persistent_step_ms,
            "persistent_ctas_per_sm": t.persistent_ctas_per_sm, "persistent_order": t.persistent_order,
            "persistent_tiles_per_item": {ENS_PASSES[k]: int(t.persistent_tiles_per_item[k]) for k in range(6)},
            "batched_step_ms": t.batched_step_ms,
            "batched_members_per_launch": t.batched_members_per_launch,
            "best_mode": {ENS_GRAPH: "graph", ENS_PERSISTENT: "persistent",
                          ENS_BATCHED: "batched"}.get(t.best_mode, str(t.best_mode))}


def ps_ensemble_check(ens) -> None:
    """Raises PsError (PS_ERR_TIMEOUT) if a bounded wait of a persistent launch gave up."""
    _check(load().ps_ensemble_check(ens))


def ps_ensemble_set_wait_test(ens, polls: int) -> None:
    _check(load().ps_ensemble_set_wait_test(ens, int(polls)))


def ps_mlp_forward(params, X, Y, count: int, stream=None) -> None:
    _check(load().ps_mlp_forward(_ptr(params), _ptr(X), _ptr(Y), int(count), _stream_handle(stream)))


def ps_mlp_grad(params, X, T, count: int, grad, loss, stream=None) -> None:
    _check(load().ps_mlp_grad(_ptr(params), _ptr(X), _ptr(T), int(count), _ptr(grad), _ptr(loss),
                              _stream_handle(stream)))


def ps_mlp_adam(params, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    _check(load().ps_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), float(beta1),
                              float(beta2), float(eps), _stream_handle(stream)))


def _norm12(norm):
    """(mean[5], std[5], s_tau, s_A) as a ctypes double[12], or None."""
    if norm is None:
        return None
    if isinstance(norm, dict):
        vals = list(norm["mean"]) + list(norm["std"]) + [norm.get("s_tau", 1.0), norm.get("s_A", 1.0)]
    else:
        vals = list(norm)
    if len(vals) != 12:
        raise ValueError("normalisation needs mean[5], std[5], s_tau and s_A")
    return (ctypes.c_double * 12)(*[float(v) for v in vals])


def ps_plan_set_closure(plan, params, norm) -> None:
    """Attach the closure (params: device FP32 vector; norm: mean, std, s_tau,
    s_A); params None detaches it."""
    if params is None:
        _check(load().ps_plan_set_closure(plan, None, None))
        return
    _check(load().ps_plan_set_closure(plan, _ptr(params), _norm12(norm)))


def ps_les_training_sample(n_dns: int, uhat_dns, n_les: int, kc: int, norm, X, A, T, stream=None) -> None:
    _check(load().ps_les_training_sample(int(n_dns), _ptr(uhat_dns), int(n_les), int(kc), _norm12(norm),
                                         _ptr(X), None if A is None else _ptr(A), _ptr(T), _stream_handle(stream)))


def ps_mlp_backward(params, X, dY, count: int, grad, stream=None) -> None:
    _check(load().ps_mlp_backward(_ptr(params), _ptr(X), _ptr(dY), int(count), _ptr(grad), _stream_handle(stream)))


def ps_plan_closure_grad(plan, params, ubar, force, grad, loss, accumulate: bool = False) -> None:
    _check(load().ps_plan_closure_grad(plan, _ptr(params), _ptr(ubar), _ptr(force), _ptr(grad), _ptr(loss),
                                       1 if accumulate else 0))


def ps_plan_closure_grad_transfer(plan, params, ubar, t_exact, grad, loss, accumulate: bool = False) -> None:
    te = [float(x) for x in t_exact]
    arr = (ctypes.c_double * len(te))(*te)
    _check(load().ps_plan_closure_grad_transfer(plan, _ptr(params), _ptr(ubar), arr, len(te), _ptr(grad), _ptr(loss),
                                                1 if accumulate else 0))


def ps_les_filter(n_dns: int, uhat_dns, n_les: int, kc: int, uhat_les, stream=None) -> None:
    _check(load().ps_les_filter(int(n_dns), _ptr(uhat_dns), int(n_les), int(kc), _ptr(uhat_les),
                                _stream_handle(stream)))


def ps_mlp_grad_tb(params, X, A, T, count: int, s_A: float, s_tau: float, grad, loss, stream=None) -> None:
    _check(load().ps_mlp_grad_tb(_ptr(params), _ptr(X), _ptr(A), _ptr(T), int(count), float(s_A), float(s_tau),
                                 _ptr(grad), _ptr(loss), _stream_handle(stream)))


# ---- convenience wrapper ------------------------------------------------------------

class Plan:
    """Owns one ps_plan; fields are torch tensors of shape (ncomp, nz, ny,
    nx//2+1) with ncomp = 3 (HD), 6 (MHD) or 4 (Boussinesq), complex64 (FP32)
    or complex128 (FP64), contiguous, on the plan's device."""

    def __init__(self, nx, ny=None, nz=None, *, stream=None, **kw):
        self.cfg = make_config(nx, ny, nz, **kw)
        self._forcing = kw.get("forcing")  # keep alive until creation copied it
        self.stream = stream
        self.handle = ps_plan_create(self.cfg, stream)

    @property
    def shape(self):
        c = self.cfg
        nc = {Equations.MHD: 6, Equations.BOUSSINESQ: 4}.get(Equations(c.eq), 3)
        return (nc, c.nz, c.ny, c.nx // 2 + 1)

    def _check_field(self, t):
        import torch
        want = torch.complex64 if self.cfg.prec == Precision.FP32 else torch.complex128
        if tuple(t.shape) != self.shape or t.dtype != want or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"field must be a contiguous CUDA {want} tensor of shape {self.shape}")

    def rhs(self, uhat, out=None, t=0.0):
        import torch
        self._check_field(uhat)
        if out is None:
            out = torch.empty_like(uhat)
        self._check_field(out)
        ps_rhs(self.handle, uhat, out, t)
        return out

    def rk_step(self, uhat, dt, t=0.0):
        self._check_field(uhat)
        ps_rk_step(self.handle, uhat, dt, t)
        return uhat

    def rk_steps(self, uhat, dt, nsteps, t=0.0):
        """nsteps steps replayed as one captured CUDA graph (ps_rk_steps)."""
        self._check_field(uhat)
        ps_rk_steps(self.handle, uhat, dt, t, nsteps)
        return uhat

    def diagnostics(self, uhat, cfl=0.5):
        self._check_field(uhat)
        return ps_diagnostics(self.handle, uhat, cfl)

    def step_stats(self):
        return ps_step_stats(self.handle)

    def set_pass_shape(self, pass_, variant):
        return ps_plan_set_pass_shape(self.handle, pass_, variant)

    def set_closure(self, params, norm=None):
        """Attach a trained LES closure (see ps_plan_set_closure); None detaches."""
        ps_plan_set_closure(self.handle, params, norm)

    def closure_grad(self, params, ubar, force, grad, loss, accumulate=False):
        """Force-matched loss and gradient of the attached closure (see
        ps_plan_closure_grad)."""
        self._check_field(ubar)
        self._check_field(force)
        ps_plan_closure_grad(self.handle, params, ubar, force, grad, loss, accumulate)

    def closure_grad_transfer(self, params, ubar, t_exact, grad, loss, accumulate=False):
        """Energy-transfer loss and gradient of the attached closure (see
        ps_plan_closure_grad_transfer)."""
        self._check_field(ubar)
        ps_plan_closure_grad_transfer(self.handle, params, ubar, t_exact, grad, loss, accumulate)

    def close(self):
        if self.handle:
            ps_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
