"""Host-side logic of bench.py, without a GPU: the max-over-ranks reduction
over two gloo ranks, the roofline byte model and the traffic lookup."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        v = bench.reduce_max(float(10 + 5 * rank), world)
        bench.barrier(world)
        q.put((rank, v))
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


def test_single_rank_reduction_is_identity():
    assert bench.reduce_max(3.5, 1) == 3.5


def test_algorithmic_bytes_model():
    b = bench.algorithmic_bytes(512, 8)
    K, cx, c2 = 170, 171, 341
    assert b["x_fused"] == 9 * 512 * 512 * cx * 8
    assert b["z_inverse"] == (3 * c2 * c2 * cx + 6 * 512 * c2 * cx) * 8
    # one RK4 step moves about 56.6 GB at 512^3 FP32 (the z-forward transform
    # hands the retained nonlinear term to the update kernel through HBM)
    step = 4 * sum(v for k, v in b.items())
    assert 54e9 < step < 59e9


def test_traffic_lookup_requires_matching_sources(tmp_path, monkeypatch):
    assert bench.ncu_traffic("x_fused", 999) is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("x_fused", 512) is None


def test_clock_summary_parses_nvidia_smi_lines():
    c = bench.ClockSampler(0)
    c.lines = ["1965, 2070, 900.1, Not Active, Not Active, Not Active, Active",
               "1980, 2070, 950.0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["sm_mhz"] == 1972.5 and s["sm_max_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"]


def test_clock_records_that_force_a_second_measurement():
    ok = {"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": []}
    assert not bench.clocks_rejected(ok)
    # the power cap is kept (noted), even with the clock pulled down
    assert not bench.clocks_rejected({"sm_mhz": 1500, "sm_max_mhz": 2070, "reasons": ["sw_power_cap"]})
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected({**ok, "reasons": [r]})
    # well below the maximum with no reason: a leftover clock lock
    assert bench.clocks_rejected({"sm_mhz": 1400, "sm_max_mhz": 2070, "reasons": []})
    assert not bench.clocks_rejected({"sm_mhz": 1900, "sm_max_mhz": 2070, "reasons": []})
    # no samples: nothing to reject on
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]})


def test_roofline_model_bytes_add_up_to_the_step_model():
    """Per-launch model bytes of the five passes (42 S per RHS plus the RK
    updates) sum to the 198 S of one IF-RK4 step; the pruned compulsory bytes
    of the retained modes are smaller."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    n = 512
    S = n * n * (n // 2 + 1) * 8
    model, step = b.dense_model_bytes(n, 8)
    assert step == 198 * S
    assert abs(4 * sum(model.values()) - step) < 1e-6 * step
    assert sum(model[k] for k in model if k != "update") == 42 * S
    pruned = b.algorithmic_bytes(n, 8)
    assert all(pruned[k] < model[k] for k in model)


def test_flop_model_of_the_line_transforms():
    """The in-register DFT counts follow the radix-2 network (R/2 log2 R
    butterflies of 4 flops plus the non-trivial twiddles), and a 512-point
    line of the radix-8 schedule costs 3 stages of 64 radix-8 DFTs plus two
    stages of 7 twiddle multiplications per butterfly."""
    assert bench.dft_flops(2) == 4
    assert bench.dft_flops(4) == 16
    assert bench.dft_flops(8) == 12 * 4 + 2 * 4
    assert bench.line_flops(512, True) == 3 * 64 * 56 + 2 * 64 * 7 * 6
    f, total = bench.flops_per_rhs(512, True)
    assert total == sum(f.values()) and 4.5e10 < total < 5.0e10
    # every kernel schedule in the table has radices multiplying to the length
    import math as m
    for (e, n), radices in bench.SCHED.items():
        assert m.prod(radices) == n and radices[0] <= e


def test_oracle_child_job_times_one_rhs():
    r = bench.finish_oracle_job(bench.start_oracle_job({"kind": "rhs_time", "n": 16}, 1), timeout=300)
    assert r["n"] == 16 and r["seconds"] > 0


def test_cpu_baseline_job_writes_the_oracle_side_of_the_error_table(tmp_path):
    """The FP32 error table's oracle side comes from the cpu_baseline leg's
    all-cores run; a CUDA side equal to it up to FP32 rounding gives errors at
    the FP32 level, one rounded to other values larger ones."""
    import numpy as np
    r = bench.finish_oracle_job(bench.start_oracle_job({"kind": "rhs_time", "n": 16, "table_dir": str(tmp_path)},
                                                       None), timeout=300)
    assert r["n"] == 16 and (tmp_path / "table.npz").exists() and (tmp_path / "diag.json").exists()
    ref = np.load(tmp_path / "table.npz")
    import json
    rd = json.loads((tmp_path / "diag.json").read_text())
    g = {"rhs": ref["rhs"].astype(np.complex64).astype(np.complex128),
         "u1": ref["u1"].astype(np.complex64).astype(np.complex128), "d0": rd["d0"], "d1": rd["d1"]}
    t = bench.fp32_error_table(g, str(tmp_path), 16)
    assert 0 < t["rhs"]["rel_l2"] < 1e-6 and 0 < t["state_after_rk4_step"]["rel_l2"] < 1e-6
    assert t["diagnostics_initial"]["energy"] == 0.0
    g["rhs"] = g["rhs"] * (1 + 1e-3)
    assert abs(bench.fp32_error_table(g, str(tmp_path), 16)["rhs"]["rel_l2"] - 1e-3) < 1e-5


def test_reference_arm_reports_our_config():
    """The reference arm runs the oracle as it stands on a bounded sample and
    reports it under the same config as the GPU arm."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--n", "32"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"] == bench.config_of(32, 1)
    assert line["cpu_baseline"]["cores"] >= 1 and line["value"] > 0
    assert abs(line["steps"] * line["ms_per_step"] - 1e3 * 32 ** 3 / line["value"] / 1e9) < 1.0


def test_committed_profiles_match_the_current_kernel_sources():
    """The bench line's `traffic` and `onchip` figures come from committed ncu
    summaries keyed by a hash of the kernel sources: a kernel change without a
    new capture would silently drop them, so the current sources must have
    both lines."""
    import bench
    assert bench.ncu_traffic("x_fused", 512) is not None
    assert bench.ncu_smem_wavefronts("x_fused", 512) is not None
