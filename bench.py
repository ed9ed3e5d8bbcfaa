#!/usr/bin/env python3
"""Benchmark of the pseudospectral Navier-Stokes hot path on GB300.

One step = one integrating-factor RK4 step (ps_rk_step): four right-hand-side
evaluations (curl, backward transforms, u x omega, forward transforms, 2/3
dealiasing, Leray projection, forcing) with the stage updates and the FP64
energy / max|u| reductions fused in.  Workload: 512^3 forced hydrodynamics,
seeded solenoidal field with E(K) ~ K^4 exp(-2 (K/4)^2) normalised to 0.5,
forcing on shells 2 <= |k| <= 3, nu = 2e-3, dt = 1e-3, FP32 bulk with FP64
reductions.  The state (1.6 GB) is larger than L2, so no flush is needed.

Metric: RHS Gpoints/s = 4 N^3 / (time per RK4 step) over all ranks, and ms per
RK step.  The FP64 path and the FP32/FP64 speed ratio are reported alongside.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The headline steps run with per-kernel timing off; a separate pass with the
plan's per-kernel events gives the kernel split and the roofline of the
dominant kernel.  The FP64 oracle (oracle/) is timed as the CPU baseline in
child processes (one BLAS thread, and all cores) and, in the background while
the GPU legs run, gives the per-output FP32 error table at 256^3.

Multi-GPU (torchrun): every rank runs an independent replica of the workload
(the single-field solve is not sharded); value sums the ranks' points.
"""

from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS Gpoints/s and time/RK step at 512^3, FP32 vs FP64 on GPU, % HBM roofline"
UNIT = "Gpoints/s"
FALLBACK_HBM_GBS = 6800.0
_COMMON = ["ps_passes.cuh", "ps_fft.cuh", "ps_async.cuh", "ps_kernels.h"]
KIND_FILES = {
    "z_inverse": _COMMON + ["k_zinv_f32.cu"],
    "y_inverse": _COMMON + ["k_yinv_f32.cu"],
    "x_fused": _COMMON + ["k_xpass_f32.cu"],
    "y_forward": _COMMON + ["k_yfwd_f32.cu"],
    "z_forward": _COMMON + ["k_zfwd_f32.cu"],
    "update": _COMMON + ["k_zfwd_f32.cu"],
}
CPU_N = 256       # grid of the oracle's CPU-baseline sample (one RHS: ~15-20 s)
REF_N = 128       # grid of the reference arm's per-step sample (one RHS: ~2 s)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-table", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--mhd-steps", type=int, default=5)
    ap.add_argument("--boussinesq-steps", type=int, default=5)
    ap.add_argument("--fp32-error-steps", type=int, default=100)
    ap.add_argument("--ensemble-steps", type=int, default=50)
    ap.add_argument("--les-steps", type=int, default=200)
    ap.add_argument("--oracle-job", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--kernel-case", default=None,
                    help="small profiling case 'nx,ny,nz[,fp64]': run --reps right-hand sides of the seeded "
                         "random field on that grid and exit (for ncu captures of one kernel)")
    ap.add_argument("--reps", type=int, default=3)
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int) -> float:
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def source_hash(files) -> str:
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(ROOT, "paper_1808_01309_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(kind: str, n: int):
    """DRAM bytes per launch of `kind` at n^3 FP32 from a committed ncu summary
    under profiles/ (a line "traffic <kind> n=<n> fp32 src=<hash>
    bytes_per_launch=<B>"), or None if absent or taken on other kernel
    sources."""
    paths = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    if not paths:
        return None
    want = source_hash(KIND_FILES[kind])
    pat = re.compile(r"^traffic\s+(\S+)\s+n=(\d+)\s+fp32\s+src=(\w+)\s+bytes_per_launch=([0-9.eE+]+)")
    for path in paths:
        for line in open(path):
            m = pat.match(line.strip())
            if m and m.group(1) == kind and int(m.group(2)) == n and m.group(3) == want:
                return float(m.group(4))
    return None


def ncu_smem_wavefronts(kind: str, n: int):
    """Shared-memory wavefronts per launch of `kind` at n^3 FP32 from a
    committed ncu summary under profiles/ (a line "smem <kind> n=<n> fp32
    src=<hash> wavefronts_per_launch=<W>"), or None if absent or taken on
    other kernel sources."""
    want = source_hash(KIND_FILES[kind])
    pat = re.compile(r"^smem\s+(\S+)\s+n=(\d+)\s+fp32\s+src=(\w+)\s+wavefronts_per_launch=([0-9.eE+]+)")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            m = pat.match(line.strip())
            if m and m.group(1) == kind and int(m.group(2)) == n and m.group(3) == want:
                return float(m.group(4))
    return None


SMEM_BYTES_PER_CLK = 128  # shared-memory bandwidth of one SM: one 128-byte wavefront per clock


def onchip_roofline(kind: str, n: int, avg_ms: float):
    """The dominant kernel against its shared-memory bandwidth: ncu wavefronts
    per launch x 128 B over the launch's CUDA-event time, against 128 B per
    clock per SM at the maximum SM clock (nominal, from the unit counts)."""
    wf = ncu_smem_wavefronts(kind, n)
    if wf is None:
        return None
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    peak = SMEM_BYTES_PER_CLK * nsm * mhz * 1e6 / 1e9  # GB/s
    achieved = wf * SMEM_BYTES_PER_CLK / (avg_ms * 1e-3) / 1e9
    return {"bound": "shared memory", "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "GB/s",
            "frac": round(achieved / peak, 4), "wavefronts_per_launch": wf,
            "peak_source": f"nominal: {SMEM_BYTES_PER_CLK} B/clk/SM x {nsm} SMs x {mhz:.0f} MHz",
            "source": "ncu l1tex__data_pipe_lsu_wavefronts_mem_shared.sum of a committed capture (profiles/)"}


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


BAD_CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(c: dict) -> bool:
    """True when a timed region's clock record cannot stand: a hardware or
    thermal slowdown was active, or the median SM clock sat well below the
    maximum with no reason reported (a clock lock).  sw_power_cap is kept."""
    if any(r in c.get("reasons", []) for r in BAD_CLOCK_REASONS):
        return True
    sm, mx = c.get("sm_mhz"), c.get("sm_max_mhz")
    return bool(sm and mx and not c.get("reasons") and sm < 0.85 * mx)


# ---------------------------------------------------------------------------
# Roofline models
# ---------------------------------------------------------------------------

def retained(n: int):
    """K = ceil(n/3) - 1 (cubic 2/3 rule), cx = K + 1, c2 = 2K + 1, modes = c2^2 cx."""
    K = (n + 2) // 3 - 1
    cx, c2 = K + 1, 2 * K + 1
    return K, cx, c2, c2 * c2 * cx


def algorithmic_bytes(n: int, vb: int):
    """Compulsory HBM bytes per launch of each kernel kind for one RHS stage of
    an IF-RK4 step on an n^3 grid with the cubic 2/3 rule (vb bytes per complex
    value): every pass reads its input and writes its output once, for the
    retained modes and lines only."""
    K, cx, c2, modes = retained(n)
    b = {
        "z_inverse": (3 * modes + 6 * n * c2 * cx) * vb,
        "y_inverse": (6 * n * c2 * cx + 6 * n * n * cx) * vb,
        "x_fused": (6 * n * n * cx + 3 * n * n * cx) * vb,
        "y_forward": (3 * n * n * cx + 3 * n * c2 * cx) * vb,
        "z_forward": (3 * n * c2 * cx + 3 * modes) * vb,
    }
    # per-mode update of an RK4 step, averaged over its four stages: reads the
    # transformed nonlinear term and the state; stages 1-3 write stage input and
    # accumulator (2-3 also read the accumulator), stage 4 reads the
    # accumulator and writes the full state
    nh = n // 2 + 1
    up = [3 * modes + 3 * modes + 2 * 3 * modes,
          3 * modes + 3 * modes + 3 * 3 * modes,
          3 * modes + 3 * modes + 3 * 3 * modes,
          3 * modes + 3 * modes + 3 * modes + 3 * n * n * nh]
    b["update"] = sum(up) / 4 * vb
    return b


def dense_model_bytes(n: int, vb: int):
    """Bytes per launch in the roofline model of an unpruned fused
    three-passes-per-direction schedule: with S = n^2 (n/2+1) vb one complex
    field, an HD RHS reads 3+6+6+3+3 S and writes 6+6+3+3+3 S (42 S), an
    IF-RK4 step moves 4 x 42 S + 30 S = 198 S.  Reported for context only: the
    pruned design never moves the masked part of these bytes."""
    S = n * n * (n // 2 + 1) * vb
    return {"z_inverse": 9 * S, "y_inverse": 12 * S, "x_fused": 9 * S, "y_forward": 6 * S,
            "z_forward": 6 * S, "update": 30 * S / 4}, 198 * S


# Radix schedules of the line transforms (the Sched table of csrc/ps_fft.cuh):
# (points per thread E, line length N) -> stage radices.
SCHED = {
    (8, 8): [8], (16, 16): [16], (8, 16): [8, 2], (8, 32): [8, 4], (8, 64): [8, 8], (16, 128): [16, 8],
    (8, 128): [8, 8, 2], (16, 256): [16, 16], (8, 256): [8, 8, 4], (8, 512): [8, 8, 8],
    (16, 1024): [16, 8, 8], (8, 1024): [8, 8, 8, 2], (12, 48): [6, 4, 2], (12, 96): [6, 4, 4],
    (12, 192): [6, 4, 4, 2],
}


def points_per_thread(fp64: bool, n: int) -> int:
    if n % 3 == 0:
        return 12
    return 16 if (not fp64 and n in (16, 128, 256, 1024)) else 8


def dft_flops(r: int) -> int:
    """Real flops of the in-register DFT of radix r: the radix-2 network for
    powers of two (4 per butterfly, plus 6 for a general twiddle, 4 for one on
    the diagonal, 0 for +-i), 16 for the 3-point DFT, two of those plus two
    twiddles and six adds for r = 6."""
    if r == 3:
        return 16
    if r == 6:
        return 2 * 16 + 2 * 6 + 6 * 2
    total, length = 0, 2
    while length <= r:
        for _ in range(r // length):
            for j in range(length // 2):
                s = (32 // length) * j  # twiddle exp(2 pi i s/32)
                total += 4 + (0 if s in (0, 8) else 4 if s in (4, 12) else 6)
        length *= 2
    return total


def line_flops(n: int, fp64: bool) -> int:
    """Real flops of one length-n line transform of the kernels' schedule:
    the stage DFTs and, after the first stage, (r - 1) complex twiddle
    multiplications (6 flops) per butterfly."""
    radices = SCHED[(points_per_thread(fp64, n), n)]
    f = 0
    for s, r in enumerate(radices):
        f += (n // r) * (dft_flops(r) + (6 * (r - 1) if s > 0 else 0))
    return f


def flops_per_rhs(n: int, fp64: bool):
    """Algorithmic flops of each pass of one HD right-hand side on the
    retained lines (cubic 2/3 rule), and their total: line transforms from
    the schedule plus the pointwise work (curl 18 and energy 12 flops per
    retained mode, packing 6 and the product and max|u| 14 per grid point,
    the split 16 per retained output mode of the x pass, 1/N^3 2 per mode
    and the projection and stage update about 60 per mode)."""
    K, cx, c2, modes = retained(n)
    L = line_flops(n, fp64)
    rows = n * n
    f = {
        "z_inverse": 6 * c2 * cx * L + 30 * modes,
        "y_inverse": 6 * n * cx * L,
        "x_fused": rows * 5 * L + rows * n * 20 + rows * cx * 16,
        "y_forward": 3 * n * cx * L,
        "z_forward": 3 * c2 * cx * L + 6 * modes,
        "update": 60 * modes,
    }
    return f, sum(f.values())


# ---------------------------------------------------------------------------
# The GPU arm
# ---------------------------------------------------------------------------

def make_inputs(n: int):
    """Initial state and forcing of the forced n^3 workload (workloads.forced)."""
    from paper_1808_01309_gb300 import workloads
    w = workloads.forced(n)
    return w.initial_state(), w.forcing()


def time_steps(plan, ud, dt, steps, warmup, stream, world, ps):
    """Device time (ms, CUDA events on the plan stream) of `steps` RK4 steps
    after `warmup` untimed ones, bracketed by a barrier and a synchronisation
    on both sides; returns (ms, kernel launches in the timed region)."""
    import torch
    for i in range(warmup):
        plan.rk_step(ud, dt, t=i * dt)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    l0 = ps.ps_plan_launch_count(plan.handle)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        plan.rk_step(ud, dt, t=(warmup + i) * dt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    barrier(world)
    torch.cuda.synchronize()
    return ms, ps.ps_plan_launch_count(plan.handle) - l0


def start_oracle_job(job: dict, threads):
    """Runs `python bench.py --oracle-job <json>` in a child process (numpy
    only, no GPU) with the BLAS pool set to `threads` (None = all cores)."""
    env = dict(os.environ)
    if threads is not None:
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
    env.pop("WORLD_SIZE", None)
    return subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-job", json.dumps(job)],
                            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)


def finish_oracle_job(proc, timeout=1800):
    out, err = proc.communicate(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError(f"oracle job failed ({proc.returncode}): {err[-2000:]}")
    return json.loads(out.strip().splitlines()[-1])


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps

    # the FP32 error table against the oracle: the GPU side here, the oracle
    # side in the cpu_baseline leg (the oracle runs nowhere else)
    want_table = rank == 0 and world == 1 and not args.no_oracle_table and not args.no_cpu_baseline

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, nu, dt = args.n, 2e-3, 1e-3
    u, f = make_inputs(n)
    stream = torch.cuda.current_stream(dev)
    out = {}

    # ---- FP32 (headline): per-kernel timing off ----------------------------
    ud = torch.from_numpy(u).to(dev, torch.complex64)
    fd = torch.from_numpy(f).to(dev, torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=nu, rk_order=4, forcing=fd, stream=stream)
    ps.ps_plan_set_timing(plan.handle, False)
    for i in range(args.warmup):
        plan.rk_step(ud, dt)
    torch.cuda.synchronize()

    def timed_region():
        with ClockSampler(local) as clk:
            ms, launches = time_steps(plan, ud, dt, args.steps, 0, stream, world, ps)
        return ms, launches, clk.summary()

    ms, launches, clocks = timed_region()
    # a throttled or clock-locked region is taken once more (every rank agrees)
    if reduce_max(1.0 if clocks_rejected(clocks) else 0.0, world) > 0:
        first = clocks
        ms, launches, clocks = timed_region()
        clocks["remeasured"] = {"first_attempt": first, "rejected_again": clocks_rejected(clocks)}
    ms_max = reduce_max(ms, world)
    ms_step = ms_max / args.steps
    e_step, umax_step = plan.step_stats()

    # ---- per-kernel split: a separate pass with the plan's events -----------
    ksplit = max(4, args.steps // 2)
    ps.ps_plan_set_timing(plan.handle, True)
    ms_split, _ = time_steps(plan, ud, dt, ksplit, 0, stream, world, ps)
    kt = ps.ps_plan_get_timing(plan.handle)
    ps.ps_plan_set_timing(plan.handle, False)
    plan.close()

    hbm, peak_src = measured_peaks()
    alg = algorithmic_bytes(n, 8)
    dense, step_dense = dense_model_bytes(n, 8)
    kinds = {k: v for k, v in kt.items() if k in alg and v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    avg_ms = kinds[dom][0] / kinds[dom][1]
    kernel_ms = {k: round(v[0] / v[1], 4) for k, v in kinds.items()}
    kernel_share = {k: round(v[0] / sum(x[0] for x in kinds.values()), 4) for k, v in kinds.items()}
    kernel_gbs = {k: round(alg[k] / (v[0] / v[1] * 1e-3) / 1e9, 1) for k, v in kinds.items()}
    kernel_frac = {k: round(kernel_gbs[k] / hbm, 3) for k in kernel_gbs}
    step_bytes = sum(alg[k] * kinds[k][1] for k in kinds) / ksplit
    roof = {"dom": dom, "avg_ms": avg_ms, "achieved": alg[dom] / (avg_ms * 1e-3) / 1e9, "alg": alg[dom],
            "dense": dense[dom], "dense_achieved": dense[dom] / (avg_ms * 1e-3) / 1e9, "step_dense": step_dense,
            "kernel_ms": kernel_ms, "kernel_share": kernel_share, "kernel_gbs": kernel_gbs,
            "kernel_frac": kernel_frac, "step_bytes": step_bytes, "split_ms_per_step": ms_split / ksplit,
            "split_steps": ksplit, "traffic": ncu_traffic(dom, n), "hbm": hbm, "peak_src": peak_src,
            "onchip": onchip_roofline(dom, n, avg_ms)}

    # ---- end to end: host buffers through the C ABI -------------------------
    e2e = None
    if not args.no_e2e:
        host = torch.from_numpy(u.astype(np.complex64)).pin_memory()
        plan = ps.Plan(n, prec=ps.Precision.FP32, nu=nu, rk_order=4, forcing=fd, stream=stream)
        ksteps = max(3, args.steps // 2)

        def host_steps(mode):
            ps.ps_plan_set_host_mode(plan.handle, mode)
            for _ in range(max(1, args.warmup // 2)):
                ps.ps_rk_step_host(plan.handle, host, dt, 0.0, 1)
            barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(ksteps):
                ps.ps_rk_step_host(plan.handle, host, dt, i * dt, 1)
            t1 = time.perf_counter()
            return reduce_max((t1 - t0) * 1e3, world) / ksteps

        copy_ms = host_steps(ps.HOST_COPY)
        mapped_ms = host_steps(ps.HOST_MAPPED)
        ce_ms = host_steps(ps.HOST_CUBE_CE)
        e2e_ms = host_steps(ps.HOST_AUTO)
        nbytes = host.numel() * host.element_size()
        _, cx, c2, _ = retained(n)
        ret_bytes = 3 * cx * c2 * c2 * host.element_size()

        def gpts(ms):
            return round(world * 4 * n ** 3 / (ms * 1e-3) / 1e9, 3)

        e2e = {"value": gpts(e2e_ms), "unit": UNIT, "ms_per_step": round(e2e_ms, 3),
               # default mode: the retained modes cross the host link each way;
               # host threads write the masked modes' zeros during the step
               "h2d_bytes_per_step": ret_bytes, "d2h_bytes_per_step": ret_bytes, "steps": ksteps,
               "api": "ps_rk_step_host (pinned host state, 1 step per call; default mode: retained modes "
                      "gathered/scattered by kernels through the device mapping, masked modes zeroed by host "
                      "threads during the step)",
               "cube_copy_engine_zeros": {"ms_per_step": round(ce_ms, 3), "value": gpts(ce_ms),
                                          "h2d_bytes_per_step": ret_bytes, "d2h_bytes_per_step": nbytes},
               "copy_engines_whole_state": {"ms_per_step": round(copy_ms, 3), "value": gpts(copy_ms),
                                            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
               # in place: the passes read the retained modes 5 times and write the state once
               "in_place": {"ms_per_step": round(mapped_ms, 3), "value": gpts(mapped_ms),
                            "h2d_bytes_per_step": 5 * ret_bytes, "d2h_bytes_per_step": nbytes}}
        plan.close()
        del host
    del ud, fd
    torch.cuda.empty_cache()

    # ---- FP64: bound by the FP64 pipe (flops against the probed FMA rate) ----
    fp64 = None
    if args.fp64_steps > 0:
        ud = torch.from_numpy(u).to(dev, torch.complex128)
        fd = torch.from_numpy(f).to(dev, torch.complex128)
        plan = ps.Plan(n, prec=ps.Precision.FP64, nu=nu, rk_order=4, forcing=fd, stream=stream)
        ms64, _ = time_steps(plan, ud, dt, args.fp64_steps, 3, stream, world, ps)
        ms64 = reduce_max(ms64, world) / args.fp64_steps
        ps.ps_plan_set_timing(plan.handle, True)
        time_steps(plan, ud, dt, 1, 0, stream, world, ps)
        kt64 = ps.ps_plan_get_timing(plan.handle)
        ps.ps_plan_set_timing(plan.handle, False)
        plan.close()
        del ud, fd
        torch.cuda.empty_cache()
        peak64 = ps.ps_probe_fma_tflops(ps.Precision.FP64, stream)
        peak32 = ps.ps_probe_fma_tflops(ps.Precision.FP32, stream)
        fl, fl_rhs = flops_per_rhs(n, True)
        flops_step = 4 * fl_rhs
        achieved = flops_step / (ms64 * 1e-3) / 1e12
        alg64 = algorithmic_bytes(n, 16)
        bytes64 = sum(alg64[k] * kt64[k][1] for k in alg64 if k in kt64)
        per_kernel = {}
        for k in fl:
            if k in kt64 and kt64[k][1] > 0:
                t = kt64[k][0] / kt64[k][1] * 1e-3
                per_kernel[k] = {"ms": round(t * 1e3, 3), "tflops": round(fl[k] / t / 1e12, 3),
                                 "frac_fp64": round(fl[k] / t / 1e12 / peak64, 3),
                                 "frac_hbm": round(alg64[k] / t / 1e9 / hbm, 3)}
        fp64 = {"ms_per_step": round(ms64, 3), "value": round(world * 4 * n ** 3 / (ms64 * 1e-3) / 1e9, 3),
                "unit": UNIT, "steps": args.fp64_steps, "fp32_speedup": round(ms64 / ms_step, 2),
                "roofline": {"bound": "alu", "flops_per_step": flops_step, "achieved": round(achieved, 3),
                             "peak": round(peak64, 3), "unit": "TFLOP/s", "frac": round(achieved / peak64, 3),
                             "peak_source": "measured live: ps_probe_fma_tflops(FP64), FMA chains, CUDA events",
                             "flop_model": "line transforms of the kernels' radix schedules on the retained "
                                           "lines + pointwise work (bench.flops_per_rhs)",
                             "hbm_frac": round(bytes64 / (ms64 * 1e-3) / 1e9 / hbm, 3),
                             "per_kernel": per_kernel},
                "fp32_fma_peak_tflops": round(peak32, 2)}

    # ---- MHD variant (u and B, twice the transforms per RHS) -----------------
    mhd = None
    if args.mhd_steps > 0:
        from paper_1808_01309_gb300 import inputs
        b = inputs.random_solenoidal_field(n, n, n, seed=51)
        ub = torch.from_numpy(np.concatenate([u, b])).to(dev, torch.complex64)
        del b
        fd = torch.from_numpy(f).to(dev, torch.complex64)
        plan = ps.Plan(n, prec=ps.Precision.FP32, eq=ps.Equations.MHD, nu=nu, eta=nu, rk_order=4,
                       forcing=fd, stream=stream)
        msm, _ = time_steps(plan, ub, dt, args.mhd_steps, 3, stream, world, ps)
        msm = reduce_max(msm, world) / args.mhd_steps
        mhd = {"ms_per_step": round(msm, 3), "value": round(world * 4 * n ** 3 / (msm * 1e-3) / 1e9, 3),
               "unit": UNIT, "steps": args.mhd_steps, "prec": "fp32",
               "workload": f"{n}^3 MHD, u and B seeded with the same spectrum (seeds 1, 51), eta = nu",
               "vs_hd_step": round(msm / ms_step, 2)}
        plan.close()
        del ub, fd
        torch.cuda.empty_cache()

    # ---- Boussinesq variant (u and theta: one more field each way) -----------
    bq = None
    if args.boussinesq_steps > 0:
        from paper_1808_01309_gb300 import inputs
        th = inputs.random_scalar_field(n, n, n, seed=61)
        ut = torch.from_numpy(np.concatenate([u, th])).to(dev, torch.complex64)
        del th
        fd = torch.from_numpy(f).to(dev, torch.complex64)
        plan = ps.Plan(n, prec=ps.Precision.FP32, eq=ps.Equations.BOUSSINESQ, nu=nu, kappa=nu, n_bv=1.0,
                       rk_order=4, forcing=fd, stream=stream)
        msb, _ = time_steps(plan, ut, dt, args.boussinesq_steps, 3, stream, world, ps)
        msb = reduce_max(msb, world) / args.boussinesq_steps
        bq = {"ms_per_step": round(msb, 3), "value": round(world * 4 * n ** 3 / (msb * 1e-3) / 1e9, 3),
              "unit": UNIT, "steps": args.boussinesq_steps, "prec": "fp32",
              "workload": f"{n}^3 Boussinesq, u seeded as above, theta with the same spectrum shape "
                          "(seed 61, variance 0.5), N = 1, kappa = nu",
              "vs_hd_step": round(msb / ms_step, 2)}
        plan.close()
        del ut, fd
        torch.cuda.empty_cache()

    # ---- FP32 error per step against FP64 at 256^3 (the 256^3 workload) ------
    err = None
    if args.fp32_error_steps > 0:
        err = fp32_error_per_step(args.fp32_error_steps, dev, stream)

    # ---- FP32 outputs on the cpu_baseline grid for the table against the oracle
    gpu_table = fp32_outputs(min(n, CPU_N), dev, stream) if want_table else None

    ens = None
    if not args.no_ensemble:
        ens = run_ensemble(args, dev, stream)
        torch.cuda.empty_cache()

    les = run_les_cost(args, dev, stream, ms_step) if args.les_steps > 0 else None

    out.update(mhd=mhd, bq=bq, err=err, ens=ens, gpu_table=gpu_table, les=les, ms_step=ms_step, launches=launches,
               clocks=clocks, roof=roof, e2e=e2e, fp64=fp64, energy=e_step, max_u=umax_step)
    return out


def _ensemble_sizes():
    from paper_1808_01309_gb300 import workloads
    return workloads.ENSEMBLE_SIZES


ENSEMBLE_SIZES = _ensemble_sizes()


def fp32_error_per_step(steps, dev, stream):
    """The forced 256^3 workload stepped in FP32 and in FP64 side by side:
    relative L2 distance of the FP32 state from the FP64 one after every step
    and the relative energy difference at the end.  The FP64 CUDA path stands
    in for the FP64 oracle over the 100 steps (each of its right-hand sides
    is held to 1e-12 of the oracle by the parity tests); the first step is
    compared with the oracle itself by the error table."""
    import torch
    from paper_1808_01309_gb300 import ps, workloads
    w = workloads.forced(256, steps=steps)
    u0, f = w.initial_state(), w.forcing()
    plans, states = [], []
    for prec, dt in ((ps.Precision.FP32, torch.complex64), (ps.Precision.FP64, torch.complex128)):
        fd = torch.from_numpy(f).to(dev, dt)
        plans.append(ps.Plan(256, prec=prec, nu=w.nu, rk_order=4, forcing=fd, stream=stream))
        states.append(torch.from_numpy(u0).to(dev, dt))
    errs = []
    for i in range(steps):
        for p, s in zip(plans, states):
            p.rk_step(s, w.dt, t=i * w.dt)
        d = states[0].to(torch.complex128) - states[1]
        errs.append(float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(states[1])))
    e32 = plans[0].diagnostics(states[0])["energy"]
    e64 = plans[1].diagnostics(states[1])["energy"]
    for p in plans:
        p.close()
    del states
    torch.cuda.empty_cache()
    return {"workload": "forced 256^3, nu = 2e-3, dt = 1e-3, IF-RK4", "steps": steps,
            "rel_l2_after_step": {str(i + 1): float(f"{errs[i]:.3e}")
                                  for i in sorted(set(range(0, steps, max(1, steps // 10))) | {steps - 1})},
            "max_rel_l2": float(f"{max(errs):.3e}"), "energy_rel_diff": float(f"{abs(e32 - e64) / e64:.3e}"),
            "reference": "FP64 CUDA path (per-RHS parity with the FP64 oracle 1e-12)"}


def fp32_outputs(n, dev, stream):
    """FP32 CUDA outputs of the forced n^3 workload from its initial state:
    the right-hand side, the state after one IF-RK4 step and the diagnostics
    of both states (numpy, on the host)."""
    import numpy as np
    import torch
    from paper_1808_01309_gb300 import ps, workloads
    w = workloads.forced(n)
    u0, f = w.initial_state(), w.forcing()
    fd = torch.from_numpy(f).to(dev, torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=w.nu, rk_order=4, forcing=fd, stream=stream)
    ud = torch.from_numpy(u0).to(dev, torch.complex64)
    rhs = plan.rhs(ud).cpu().numpy().astype(np.complex128)
    d0 = plan.diagnostics(ud)
    plan.rk_step(ud, w.dt)
    u1 = ud.cpu().numpy().astype(np.complex128)
    d1 = plan.diagnostics(ud)
    plan.close()
    del ud, fd
    torch.cuda.empty_cache()
    return {"rhs": rhs, "u1": u1, "d0": d0, "d1": d1}


def _diag_errors(g, r):
    """Relative error of each diagnostic of the CUDA path (g) against the
    oracle's (r); helicity relative to its Schwarz bound 2 sqrt(E Omega)."""
    out = {}
    for k in ("energy", "enstrophy", "max_u", "cfl_dt"):
        out[k] = float(f"{abs(g[k] - r[k]) / abs(r[k]):.3e}")
    out["helicity"] = float(f"{abs(g['helicity'] - r['helicity']) / (2 * math.sqrt(r['energy'] * r['enstrophy'])):.3e}")
    spec_r = r["spectrum"]
    spec_g = g["spectrum"][:len(spec_r)]
    rel = [abs(a - b) / b for a, b in zip(spec_g, spec_r) if b > 1e-12 * max(spec_r)]
    out["spectrum_max_rel"] = float(f"{max(rel):.3e}")
    out["max_div_gpu"] = float(f"{g['max_div']:.3e}")
    return out


def fp32_error_table(g, ref_dir, n):
    """Per-output error of the FP32 CUDA path against the FP64 oracle on the
    forced n^3 workload (right-hand side, state after one RK4 step,
    diagnostics of the initial and the stepped state); the oracle side comes
    from the cpu_baseline leg's run."""
    import numpy as np
    ref = np.load(os.path.join(ref_dir, "table.npz"))
    with open(os.path.join(ref_dir, "diag.json")) as fh:
        rd = json.load(fh)

    def field(a, b):
        d = a - b
        return {"rel_l2": float(f"{np.linalg.norm(d) / np.linalg.norm(b):.3e}"),
                "max_mode_rel": float(f"{np.max(np.abs(d)) / np.max(np.abs(b)):.3e}")}

    return {"workload": f"forced {n}^3 (seeded field + forcing, nu = 2e-3, dt = 1e-3), FP32 CUDA path "
                        "against the FP64 oracle (oracle side from the cpu_baseline leg's run)",
            "rhs": field(g["rhs"], ref["rhs"]), "state_after_rk4_step": field(g["u1"], ref["u1"]),
            "diagnostics_initial": _diag_errors(g["d0"], rd["d0"]),
            "diagnostics_after_step": _diag_errors(g["d1"], rd["d1"]),
            "tolerances": {"rhs_rel_l2": 2e-6, "energy_after_100_steps": 1e-4}}


def run_ensemble(args, dev, stream):
    """48 independent unforced solves (16 each at 64^3, 96^3, 128^3), seeds
    1000+i, nu_i = 1e-3 + 4e-3 U(seed 2000+i), FP32, IF-RK4, dt = 1e-3:
    member-by-member launches vs one CUDA graph of the members' launch chains
    vs one persistent kernel over a (member, pass, tile) work queue vs batched
    launches (one per pass for the members of a grid size; all autotuned);
    the largest relative difference of the persistent and graph final states
    is reported."""
    import torch
    from paper_1808_01309_gb300 import inputs, ps
    cfgs, host = [], []
    for i, n in enumerate(ENSEMBLE_SIZES):
        cfgs.append(ps.make_config(n, prec=ps.Precision.FP32, nu=inputs.ensemble_viscosity(i), rk_order=4))
        host.append(torch.from_numpy(inputs.random_solenoidal_field(n, n, n, seed=1000 + i)).to(dev, torch.complex64))
    ens = ps.ps_ensemble_create(cfgs, stream)
    K, dt = args.ensemble_steps, 1e-3
    points = 4 * sum(n ** 3 for n in ENSEMBLE_SIZES) * K
    t0 = time.perf_counter()
    tuning = ps.ps_ensemble_tune(ens, host, dt)
    tune_s = time.perf_counter() - t0
    out = {"members": len(cfgs), "sizes": "16x64^3 + 16x96^3 + 16x128^3", "steps": K, "prec": "fp32",
           "tuning": tuning, "tune_s": round(tune_s, 2)}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    finals = {}
    for mode, name in ((ps.ENS_SEQUENTIAL, "sequential"), (ps.ENS_GRAPH, "graph"), (ps.ENS_PERSISTENT, "persistent"),
                       (ps.ENS_BATCHED, "batched")):
        states = [h.clone() for h in host]
        # warm-up (for the graph: captures and instantiates the K-step graph)
        t1 = time.perf_counter()
        ps.ps_ensemble_rk_steps(ens, states, dt, 0.0, K, mode)
        torch.cuda.synchronize()
        first = time.perf_counter() - t1
        e0.record(stream)
        ps.ps_ensemble_rk_steps(ens, states, dt, 0.0, K, mode)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ps.ps_ensemble_check(ens)
        out[name] = {"ms": round(ms, 3), "ms_per_step": round(ms / K, 4),
                     "gpoints_s": round(points / (ms * 1e-3) / 1e9, 3), "first_call_s": round(first, 3)}
        finals[name] = states
    out["graph_speedup"] = round(out["sequential"]["ms"] / out["graph"]["ms"], 3)
    out["persistent_speedup"] = round(out["sequential"]["ms"] / out["persistent"]["ms"], 3)
    out["persistent_vs_graph"] = round(out["graph"]["ms"] / out["persistent"]["ms"], 3)
    out["batched_speedup"] = round(out["sequential"]["ms"] / out["batched"]["ms"], 3)
    out["batched_vs_graph"] = round(out["graph"]["ms"] / out["batched"]["ms"], 3)
    # the graph runs the tuned tile shapes, the persistent launch the default
    # ones: equal to rounding (bitwise with equal shapes, see the GPU tests)
    out["persistent_vs_graph_max_rel"] = float(max(
        ((a - b).abs().max() / b.abs().max()).item() for a, b in zip(finals["persistent"], finals["graph"])))
    out["default_mode"] = tuning["best_mode"]
    ps.ps_ensemble_destroy(ens)
    return out


def run_les_cost(args, dev, stream, ms_dns):
    """Cost of the learned LES closure against the DNS it replaces: the 64^3
    FP32 LES step with the closure attached (MLP 5-64-64-6 on the BF16
    tensor cores inside every RK4 stage, graph-replayed through
    ps_rk_steps, dt = 5e-3) against the headline 512^3 DNS step (dt =
    1e-3), per unit of simulated time.  The network weights here are the
    initial ones (the cost does not depend on them); the accuracy of the
    trained closure comes from the LES workflow (paper_1808_01309_gb300.les)."""
    import torch
    from paper_1808_01309_gb300 import inputs, les, ps
    n, dt_les, dt_dns, K = 64, 5e-3, 1e-3, args.les_steps
    f = torch.from_numpy(inputs.forcing_field(n, n, n, seed=2)).to(dev, torch.complex64)
    u = torch.from_numpy(inputs.random_solenoidal_field(n, n, n, seed=1)).to(dev, torch.complex64)
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=2e-3, rk_order=4, forcing=f, stream=stream)
    out = {"workload": f"{n}^3 FP32 LES, IF-RK4, dt = {dt_les}, kc = 21, forcing as the DNS; steps "
                       f"graph-replayed (ps_rk_steps)", "steps": K}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for name, params in (("no_closure", None), ("closure", torch.from_numpy(les.init_params(1)).to(dev))):
        if params is not None:
            plan.set_closure(params, {"mean": [0.0] * 5, "std": [1.0] * 5, "s_tau": 1e-6, "s_A": 1.0})
        plan.rk_steps(u, dt_les, K)  # capture and warm-up
        torch.cuda.synchronize()
        e0.record(stream)
        plan.rk_steps(u, dt_les, K)
        e1.record(stream)
        torch.cuda.synchronize()
        out[f"ms_les_{name}"] = round(e0.elapsed_time(e1) / K, 4)
    plan.close()
    ms_les = out["ms_les_closure"]
    out.update({"ms_les": ms_les, "ms_dns": round(ms_dns, 3), "dt_les": dt_les, "dt_dns": dt_dns,
                "dns": "512^3 FP32 headline step", "cost_ratio": round((ms_dns / dt_dns) / (ms_les / dt_les), 1),
                "target": ">= 10x lower cost per simulated time"})
    return out


# ---------------------------------------------------------------------------
# The FP64 oracle on the host cores (child processes; numpy only)
# ---------------------------------------------------------------------------

def oracle_job(job: dict) -> dict:
    """Work of one oracle child process of the cpu_baseline leg (see
    start_oracle_job): times one oracle RHS of the forced n^3 workload; with
    job["table_dir"] it then (untimed) also takes one IF-RK4 step and the
    diagnostics of both states and writes them with that RHS to the
    directory, the oracle side of the FP32 error table."""
    import numpy as np

    import oracle
    from paper_1808_01309_gb300 import workloads
    n = int(job["n"])
    w = workloads.forced(n)
    u, f = w.initial_state(), w.forcing()
    cfg = oracle.Config(n, n, n, nu=w.nu, rk_order=4)
    if job["kind"] != "rhs_time":
        raise ValueError(f"unknown oracle job {job['kind']!r}")
    t0 = time.perf_counter()
    rhs = oracle.rhs(u, cfg, forcing=f)
    secs = time.perf_counter() - t0
    if job.get("table_dir"):
        u1 = oracle.rk_step(u, w.dt, cfg, forcing=f)
        d0, d1 = oracle.diagnostics(u, cfg), oracle.diagnostics(u1, cfg)
        np.savez(os.path.join(job["table_dir"], "table.npz"), rhs=rhs, u1=u1)
        js = {k: {kk: (vv.tolist() if hasattr(vv, "tolist") else vv) for kk, vv in d.items()}
              for k, d in (("d0", d0), ("d1", d1))}
        with open(os.path.join(job["table_dir"], "diag.json"), "w") as fh:
            json.dump(js, fh)
    return {"seconds": secs, "n": n}


def cpu_cores() -> int:
    return os.cpu_count() or 1


def cpu_baseline_rows(n: int, table_dir=None):
    """One oracle RHS of the forced n^3 workload timed in a child process with
    one BLAS thread and with all cores; Gpoints/s per grid point.  With
    table_dir the all-cores run also writes the oracle side of the FP32 error
    table there."""
    rows = {}
    for name, threads in (("single_core", 1), ("all_cores", None)):
        job = {"kind": "rhs_time", "n": n}
        if threads is None and table_dir:
            job["table_dir"] = table_dir
        r = finish_oracle_job(start_oracle_job(job, threads))
        rows[name] = {"value": round(n ** 3 / r["seconds"] / 1e9, 6), "unit": UNIT, "seconds": round(r["seconds"], 2),
                      "cores": 1 if threads == 1 else cpu_cores()}
    return rows


def cpu_sample_desc(n_cpu, n, secs, cores):
    return (f"one FP64 oracle RHS of the same recipe (seeded field + forcing, nu = 2e-3) on a {n_cpu}^3 grid "
            f"instead of {n}^3 ({secs:.1f} s; numpy, the oracle's own mixed-radix FFT, BLAS pool of {cores} "
            f"thread{'s' if cores > 1 else ''}; elementwise steps single-threaded), throughput per grid point")


def config_of(n: int, world: int) -> dict:
    return {"workload": f"{n}^3 forced HD: seeded E(K)~K^4 exp(-2(K/4)^2) field (E=0.5), forcing on "
                        f"2<=|k|<=3, nu=2e-3, dt=1e-3, IF-RK4, cubic 2/3 dealias, FP32 bulk + FP64 "
                        f"reductions; step = one RK4 step = 4 RHS", "n": n, "rk_order": 4,
            "l2": f"inputs larger than L2 (state {3 * n * n * (n // 2 + 1) * 8 / 1e9:.2f} GB, 129 MB L2), no flush",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The oracle as it stands, timed on the host cores (all of them): each
    step is one FP64 oracle RHS of the same recipe at REF_N^3, a bounded
    sample of the workload, so that the whole run ends within minutes."""
    import oracle
    nc = min(args.n, REF_N)
    u, f = make_inputs(nc)
    cfg = oracle.Config(nc, nc, nc, nu=2e-3, rk_order=4)
    for _ in range(args.warmup):
        oracle.rhs(u, cfg, forcing=f)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.rhs(u, cfg, forcing=f)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = nc ** 3 / t / 1e9
    desc = ("each step: " + cpu_sample_desc(nc, args.n, t, cpu_cores())
            + "; ms_per_step is the time of that sample, the work each timed step did")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args.n, args.gpus),
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_case(spec: str, reps: int) -> None:
    """Small cases for ncu captures of one kernel family, run one after the
    other on the default stream.  spec = "nx,ny,nz[,fp64][,mhd|boussinesq]"
    runs `reps` right-hand sides of the seeded random field with forcing on
    that grid (e.g. 512,512,128 for the x and y passes with 512-point lines,
    256,128,512 for the z passes); "les" runs `reps` 64^3 RK4 steps with the
    learned closure attached; "mlp" runs `reps` MLP forward evaluations of
    64^3 samples; "ensemble_persistent" / "ensemble_batched" run `reps`
    one-step calls of a six-member FP32 ensemble (64^3, 96^3, 128^3, twice
    each) in that mode; "aux" runs once each the kernels the other cases
    miss (diagnostics, a host-buffer step and a small right-hand side
    without a plan, MLP gradient and Adam step, LES training sample, filter
    and closure gradients)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import inputs, les, ps
    parts = spec.split(",")
    if parts[0] in ("ensemble_persistent", "ensemble_batched"):
        sizes = [64, 96, 128, 64, 96, 128]
        cfgs = [ps.make_config(n, prec=ps.Precision.FP32, nu=inputs.ensemble_viscosity(i), rk_order=4)
                for i, n in enumerate(sizes)]
        st = [torch.from_numpy(inputs.random_solenoidal_field(n, n, n, seed=1000 + i)).to("cuda", torch.complex64)
              for i, n in enumerate(sizes)]
        ens = ps.ps_ensemble_create(cfgs)
        mode = ps.ENS_PERSISTENT if parts[0] == "ensemble_persistent" else ps.ENS_BATCHED
        for _ in range(reps):
            ps.ps_ensemble_rk_steps(ens, st, 1e-3, 0.0, 1, mode)
        ps.ps_ensemble_check(ens)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": spec, "reps": reps, "u_norm": float(sum(torch.linalg.vector_norm(u) for u in st))}))
        ps.ps_ensemble_destroy(ens)
        return
    if parts[0] == "aux":
        c64 = torch.complex64
        u = inputs.random_solenoidal_field(64, 64, 64, seed=1)
        plan = ps.Plan(64, prec=ps.Precision.FP32, nu=2e-3, rk_order=4)
        plan.diagnostics(torch.from_numpy(u).to("cuda", c64))
        ps.ps_rk_step_host(plan.handle, torch.from_numpy(u.astype(np.complex64)).pin_memory(), 1e-3)
        plan.close()
        u32 = torch.from_numpy(inputs.random_solenoidal_field(32, 32, 32, seed=2)).to("cuda", c64)
        ps.ps_rhs_noalloc(ps.make_config(32, prec=ps.Precision.FP32, nu=2e-3), u32, torch.empty_like(u32))
        params = torch.from_numpy(les.init_params(1)).to("cuda")
        B = 1 << 16
        X, T = torch.randn((B, 5), device="cuda"), torch.randn((B, 6), device="cuda")
        G = torch.empty(ps.MLP_NPARAM, device="cuda")
        L = torch.empty(1, device="cuda", dtype=torch.float64)
        ps.ps_mlp_grad(params, X, T, B, G, L)
        ps.ps_mlp_adam(params, G, torch.zeros_like(params), torch.zeros_like(params), 1, 1e-3)
        ud64 = torch.from_numpy(inputs.random_solenoidal_field(64, 64, 64, seed=13)).to("cuda", c64)
        Xs, As, Ts = (torch.empty((32 ** 3, k), device="cuda") for k in (5, 9, 6))
        ps.ps_les_training_sample(64, ud64, 32, 10, None, Xs, As, Ts)
        ubar = torch.empty((3, 32, 32, 17), device="cuda", dtype=c64)
        ps.ps_les_filter(64, ud64, 32, 10, ubar)
        norm = {"mean": Xs.mean(0).double().tolist(), "std": Xs.std(0).double().tolist(), "s_tau": 0.05,
                "s_A": float(As.square().sum(1).mean().sqrt())}
        plan = ps.Plan(32, prec=ps.Precision.FP32, nu=1e-3)
        plan.set_closure(params, norm)
        force = torch.from_numpy(inputs.forcing_field(32, 32, 32, seed=3)).to("cuda", c64)
        plan.closure_grad(params, ubar, force, G, L)
        plan.closure_grad_transfer(params, ubar, np.zeros(16), G, L)
        plan.rk_step(ubar, 1e-3)
        plan.close()
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": spec, "loss": float(L.item())}))
        return
    if parts[0] == "mlp":
        P = 64 ** 3
        params = torch.from_numpy(les.init_params(1)).to("cuda")
        X = torch.randn((P, 5), device="cuda")
        Y = torch.empty((P, 6), device="cuda")
        for _ in range(reps):
            ps.ps_mlp_forward(params, X, Y, P)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": spec, "reps": reps, "y_norm": float(Y.norm())}))
        return
    if parts[0] == "les":
        n = 64
        f = torch.from_numpy(inputs.forcing_field(n, n, n, seed=2)).to("cuda", torch.complex64)
        u = torch.from_numpy(inputs.random_solenoidal_field(n, n, n, seed=1)).to("cuda", torch.complex64)
        plan = ps.Plan(n, prec=ps.Precision.FP32, nu=2e-3, rk_order=4, forcing=f)
        plan.set_closure(torch.from_numpy(les.init_params(1)).to("cuda"),
                         {"mean": [0.0] * 5, "std": [1.0] * 5, "s_tau": 1e-6, "s_A": 1.0})
        for _ in range(reps):
            plan.rk_step(u, 5e-3)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": spec, "reps": reps, "u_norm": float(torch.linalg.vector_norm(u))}))
        plan.close()
        return
    nx, ny, nz = (int(v) for v in parts[:3])
    fp64 = "fp64" in parts[3:]
    eq = ps.Equations.MHD if "mhd" in parts[3:] else ps.Equations.BOUSSINESQ if "boussinesq" in parts[3:] \
        else ps.Equations.HD
    P, dt = (ps.Precision.FP64, torch.complex128) if fp64 else (ps.Precision.FP32, torch.complex64)
    u = inputs.random_solenoidal_field(nx, ny, nz, seed=1)
    if eq == ps.Equations.MHD:
        u = np.concatenate([u, inputs.random_solenoidal_field(nx, ny, nz, seed=51)])
    elif eq == ps.Equations.BOUSSINESQ:
        u = np.concatenate([u, inputs.random_scalar_field(nx, ny, nz, seed=61)])
    ud = torch.from_numpy(u).to("cuda", dt)
    f = torch.from_numpy(inputs.forcing_field(nx, ny, nz, seed=2)).to("cuda", dt)
    plan = ps.Plan(nx, ny, nz, prec=P, eq=eq, nu=2e-3, eta=2e-3, kappa=2e-3, n_bv=1.0, rk_order=4, forcing=f)
    out = torch.empty_like(ud)
    for _ in range(reps):
        plan.rhs(ud, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": spec, "reps": reps, "rhs_norm": float(torch.linalg.vector_norm(out))}))
    plan.close()


def main():
    args = parse_args()
    if args.oracle_job is not None:
        print(json.dumps(oracle_job(json.loads(args.oracle_job))), flush=True)
        return
    if args.kernel_case is not None:
        kernel_case(args.kernel_case, args.reps)
        return
    world, rank, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    n = args.n

    if args.impl == "reference":
        # the oracle, timed as it stands on this host (rank 0 only)
        if rank == 0:
            run_reference(args)
        return

    res = run_ours(args, world, rank, local)
    if rank != 0:
        return
    cpu = None
    table = None
    if not args.no_cpu_baseline and world == 1:
        nc = min(n, CPU_N)
        table_dir = tempfile.mkdtemp(prefix="ps_oracle_") if res["gpu_table"] is not None else None
        rows = cpu_baseline_rows(nc, table_dir)
        if table_dir:
            table = fp32_error_table(res["gpu_table"], table_dir, nc)
            for name in os.listdir(table_dir):
                os.remove(os.path.join(table_dir, name))
            os.rmdir(table_dir)
        a = rows["all_cores"]
        cpu = {"value": a["value"], "unit": UNIT, "cores": a["cores"], "kind": "oracle",
               "sample": cpu_sample_desc(nc, n, a["seconds"], a["cores"]),
               "single_core": {"value": rows["single_core"]["value"], "cores": 1,
                               "seconds": rows["single_core"]["seconds"]}}
    ms = res["ms_step"]
    value = world * 4 * n ** 3 / (ms * 1e-3) / 1e9
    r = res["roof"]
    hbm = r["hbm"]
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_of(n, world),
        "roofline": {"bound": "hbm", "kernel": r["dom"], "achieved": round(r["achieved"], 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(r["achieved"] / hbm, 4),
                     "traffic": r["traffic"],
                     "onchip": r["onchip"],
                     "algorithmic_bytes": r["alg"],
                     "bytes_model": "compulsory bytes of the pruned passes: each pass reads its input and writes "
                                    "its output once, retained modes and lines only (bench.algorithmic_bytes)",
                     "peak_source": f"{r['peak_src']} (MEASURED_PEAKS.json hbm_gbs)" if r["peak_src"] == "measured"
                     else "fallback 6800 GB/s",
                     "avg_launch_ms": round(r["avg_ms"], 4),
                     "kernel_ms": r["kernel_ms"], "kernel_share": r["kernel_share"],
                     "kernel_alg_gbs": r["kernel_gbs"], "kernel_frac": r["kernel_frac"],
                     "step_alg_bytes": r["step_bytes"],
                     "step_frac": round(r["step_bytes"] / (ms * 1e-3) / 1e9 / hbm, 4),
                     "split_pass": {"steps": r["split_steps"], "ms_per_step": round(r["split_ms_per_step"], 3),
                                    "note": "per-kernel times from a separate pass with the plan's per-kernel "
                                            "events; the headline steps run without them"},
                     # the unpruned 42 S / 198 S model, for context only
                     "dense_model": {"algorithmic_bytes": r["dense"], "achieved": round(r["dense_achieved"], 1),
                                     "frac": round(r["dense_achieved"] / hbm, 4), "step_bytes": r["step_dense"],
                                     "step_frac": round(r["step_dense"] / (ms * 1e-3) / 1e9 / hbm, 4)}},
        "cpu_baseline": cpu,
        "e2e": res["e2e"],
        "fp64": res["fp64"],
        "mhd": res["mhd"],
        "boussinesq": res["bq"],
        "fp32_vs_oracle_256": table,
        "fp32_error_256": res["err"],
        "ensemble": res["ens"],
        "les": res["les"],
        "clocks": res["clocks"],
        "gpu_launches": res["launches"],
        "stats": {"energy_at_last_step_start": res["energy"], "max_u": res["max_u"]},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
