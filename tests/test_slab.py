"""Slab decomposition of the right-hand side (paper_1808_01309_gb300/slab.py),
on CPU: the partition, and the right-hand side assembled from P ranks' kx
slabs against the oracle's right-hand side of the whole field, with the two
all-to-all exchanges done by a loopback in one process and by
torch.distributed over gloo between 2 and 3 CPU processes.  The local passes
come from a test backend built on the oracle's transforms
(tests/slab_cpu_backend.py); the CUDA backend runs the same exchanges in
tests/test_gpu_slab.py."""

import math
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs, slab

from .parity import assert_parity

torch = pytest.importorskip("torch")


def test_split_covers_every_item_once_with_sizes_within_one():
    for n in (1, 5, 20, 171, 512):
        for parts in (1, 2, 3, 4, 7):
            spans = [slab.split(n, parts, i) for i in range(parts)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(parts - 1))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab.split(10, 0, 0)


def _case(nx=24, ny=12, nz=20):
    cfg = oracle.Config(nx, ny, nz, lx=2 * math.pi, ly=3.0, lz=5.0, nu=3e-3)
    u = inputs.random_solenoidal_field(nx, ny, nz, seed=7, ly=3.0, lz=5.0)
    f = inputs.forcing_field(nx, ny, nz, seed=2, ly=3.0, lz=5.0)
    return cfg, u, f


@pytest.mark.parametrize("P,shape", [(1, (24, 12, 20)), (2, (24, 12, 20)), (3, (24, 12, 20)), (4, (24, 12, 20)),
                                     (4, (8, 12, 6)), (5, (8, 8, 3))])
def test_loopback_slabs_match_the_oracle(P, shape):
    """Includes ranks that own no kx column (8 points along x keep 3 columns)
    and ranks that own no z plane (3 planes over 5 ranks)."""
    from .slab_cpu_backend import CpuBackend, assemble, local_columns
    cfg, u, f = _case(*shape)
    cx = slab.retained_columns(cfg.nx)
    lays = [slab.SlabLayout(cfg.nx, cfg.ny, cfg.nz, cx, P, r) for r in range(P)]
    backends = [CpuBackend(cfg, lay, local_columns(f, lay)) for lay in lays]
    parts = slab.rhs_loopback(backends, lays, [local_columns(u, lay) for lay in lays])
    got = assemble([p.numpy() for p in parts], lays, cfg.nx // 2 + 1)
    assert_parity(got, oracle.rhs(u, cfg, forcing=f), 1e-13, f"loopback P={P}")


def _rank(rank, world, port, q, shape):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from tests.slab_cpu_backend import CpuBackend, local_columns
        cfg, u, f = _case(*shape)
        lay = slab.SlabLayout(cfg.nx, cfg.ny, cfg.nz, slab.retained_columns(cfg.nx), world, rank)
        comm = slab.TorchDistributed()
        out = slab.rhs_local(CpuBackend(cfg, lay, local_columns(f, lay)), lay, local_columns(u, lay), comm)
        q.put((rank, out.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape", [(2, (24, 12, 20)), (3, (24, 12, 20)), (4, (8, 12, 6))])
def test_gloo_ranks_match_the_oracle(world, shape):
    import multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, shape)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    cfg, u, f = _case(*shape)
    lays = [slab.SlabLayout(cfg.nx, cfg.ny, cfg.nz, slab.retained_columns(cfg.nx), world, r) for r in range(world)]
    from .slab_cpu_backend import assemble
    full = assemble([got[r] for r in range(world)], lays, cfg.nx // 2 + 1)
    assert_parity(full, oracle.rhs(u, cfg, forcing=f), 1e-13, f"gloo world={world}")
    assert np.all(full[..., slab.retained_columns(cfg.nx):] == 0)


def _rank_with_a_lost_peer(rank, world, port, q):
    import datetime

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        q.put((rank, "left"))  # this rank fails before the exchanges and leaves
        return
    try:
        from tests.slab_cpu_backend import CpuBackend, local_columns
        cfg, u, f = _case()
        lay = slab.SlabLayout(cfg.nx, cfg.ny, cfg.nz, slab.retained_columns(cfg.nx), world, rank)
        slab.rhs_local(CpuBackend(cfg, lay, local_columns(f, lay)), lay, local_columns(u, lay),
                       slab.TorchDistributed())
        q.put((rank, "finished"))
    except RuntimeError as e:
        q.put((rank, "error: " + str(e).splitlines()[0][:80]))


def test_a_lost_rank_ends_the_exchange_with_an_error():
    """A rank that leaves before the exchanges (failure injected on the host):
    the surviving rank's all-to-all ends with an error (gloo reports the
    closed connection; the process group's 5 s timeout bounds the wait
    otherwise) instead of waiting for ever."""
    import multiprocessing as mp
    import time
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_with_a_lost_peer, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.monotonic()
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        if p.exitcode is None:
            p.kill()
    assert got[1] == "left"
    assert got[0].startswith("error"), got[0]
    assert time.monotonic() - t0 < 100
