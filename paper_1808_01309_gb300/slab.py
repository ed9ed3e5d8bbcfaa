"""Slab decomposition of the right-hand side over P ranks.

The paper distributes each 3D transform over MPI tasks as slabs and
exchanges the data once per transform with an all-to-all between the passes
along the local axes and the pass along the distributed axis (Sec. 2, the
slab decomposition in z; Sec. 3.3, the transpose and exchange).  Here the
same structure maps onto the five passes of one right-hand side:

  * spectral space is split into slabs of the retained kx columns: rank r
    owns columns [kx_lo(r), kx_hi(r)) of all (ky, kz);
  * physical space is split into z slabs: rank r owns planes
    [z_lo(r), z_hi(r)) of all (y, x);
  * rank r runs the backward z and y transforms (curl included) on its kx
    columns, then exchange A (6 fields) gives every rank complete x rows of
    its z planes; the x pass (backward x, u x omega, forward x) is local;
    exchange B (3 fields) returns the kx columns; the forward y and z
    transforms, the projection, forcing and viscous term are local again.

That is one all-to-all per 3D transform, of 6 and 3 fields.  The local
passes run in a backend (the CUDA path through the C ABI; tests plug in
others) and the exchanges in a communicator (torch.distributed all_to_all,
NCCL between GPUs or gloo between CPU processes; or a loopback that plays
all ranks in one process).  This module holds the partition and the
exchange bookkeeping only: it performs no step of the method itself.
"""

from __future__ import annotations

import dataclasses


def split(n: int, parts: int, index: int):
    """[lo, hi) of part `index` when n items are split into `parts` contiguous
    parts whose sizes differ by at most one (the first n % parts get one
    more)."""
    if parts < 1 or not 0 <= index < parts:
        raise ValueError("bad partition")
    base, extra = divmod(n, parts)
    lo = index * base + min(index, extra)
    return lo, lo + base + (1 if index < extra else 0)


@dataclasses.dataclass(frozen=True)
class SlabLayout:
    """Ownership of kx columns and z planes for rank `rank` of `nranks`.

    cx is the number of retained kx columns (kx = 0..Kx); kx columns beyond
    Kx are zero in every state and right-hand side and belong to no rank."""

    nx: int
    ny: int
    nz: int
    cx: int
    nranks: int
    rank: int

    def kx_range(self, r: int | None = None):
        return split(self.cx, self.nranks, self.rank if r is None else r)

    def z_range(self, r: int | None = None):
        return split(self.nz, self.nranks, self.rank if r is None else r)

    @property
    def nkx(self) -> int:
        lo, hi = self.kx_range()
        return hi - lo

    @property
    def nzl(self) -> int:
        lo, hi = self.z_range()
        return hi - lo


def retained_columns(nx: int, dealias: int = 0) -> int:
    """Retained kx count Kx + 1 (cubic or spherical 2/3 rule, or all but the
    Nyquist column)."""
    return nx // 2 if dealias == 2 else (nx + 2) // 3


def pack_a(lay: SlabLayout, a):
    """Exchange A, sender side: the backward-transformed fields [6, nz, ny,
    nkx] of this rank's kx columns, cut into the z planes of every rank."""
    return [a[:, slice(*lay.z_range(s))].contiguous() for s in range(lay.nranks)]


def recv_shapes_a(lay: SlabLayout):
    return [(6, lay.nzl, lay.ny, lay.kx_range(r)[1] - lay.kx_range(r)[0]) for r in range(lay.nranks)]


def unpack_a(lay: SlabLayout, blocks):
    """Exchange A, receiver side: the blocks of every rank's kx columns for
    this rank's z planes, joined into full x rows [6, rows, cx]."""
    import torch
    return torch.cat(blocks, dim=3).reshape(6, lay.nzl * lay.ny, lay.cx)


def pack_b(lay: SlabLayout, xo):
    """Exchange B, sender side: the x pass output [3, rows, cx] of this
    rank's z planes, cut into the kx columns of every rank."""
    xo = xo.reshape(3, lay.nzl, lay.ny, lay.cx)
    return [xo[..., slice(*lay.kx_range(r))].contiguous() for r in range(lay.nranks)]


def recv_shapes_b(lay: SlabLayout):
    return [(3, lay.z_range(s)[1] - lay.z_range(s)[0], lay.ny, lay.nkx) for s in range(lay.nranks)]


def unpack_b(lay: SlabLayout, blocks):
    """Exchange B, receiver side: the z planes of every rank for this rank's
    kx columns, joined into [3, nz, ny, nkx]."""
    import torch
    return torch.cat(blocks, dim=1)


class TorchDistributed:
    """One rank of a torch.distributed process group: the all-to-all of one
    list of contiguous tensors as one batch of point-to-point sends and
    receives (grouped send/recv under NCCL between GPUs; gloo between CPU
    ranks, whose backend has no all_to_all); the block a rank keeps is not
    sent."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.nranks = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def exchange(self, send, recv_shapes):
        import torch
        like = send[0]
        recv = [torch.empty(s, dtype=like.dtype, device=like.device) for s in recv_shapes]
        recv[self.rank].copy_(send[self.rank])
        ops = []
        for peer in range(self.nranks):
            if peer == self.rank:
                continue
            ops.append(self.dist.P2POp(self.dist.irecv, recv[peer], peer, self.group))
            ops.append(self.dist.P2POp(self.dist.isend, send[peer], peer, self.group))
        if ops:
            for w in self.dist.batch_isend_irecv(ops):
                w.wait()
        return recv


def rhs_local(backend, lay: SlabLayout, uhat_local, comm):
    """Right-hand side of this rank's kx slab, with the two exchanges done by
    `comm` (TorchDistributed).

    backend: inverse_yz(uhat_local) -> [6, nz, ny, nkx]: curl and backward
             z and y transforms of the local kx columns;
             x_pass(xin [6, rows, cx]) -> [3, rows, cx]: backward x
             transforms, u x omega and forward x transforms of full rows;
             forward_yz(yin [3, nz, ny, nkx], uhat_local) -> the right-hand
             side of the local columns (forward y and z transforms, 1/N^3,
             mask, forcing, projection, viscous term)."""
    a = backend.inverse_yz(uhat_local)
    xin = unpack_a(lay, comm.exchange(pack_a(lay, a), recv_shapes_a(lay)))
    xo = backend.x_pass(xin)
    yin = unpack_b(lay, comm.exchange(pack_b(lay, xo), recv_shapes_b(lay)))
    return backend.forward_yz(yin, uhat_local)


def rhs_loopback(backends, lays, uhats):
    """The same right-hand side with every rank played in this process, one
    pass at a time over all ranks, the exchanges by handing blocks over
    (backends, lays and uhats indexed by rank)."""
    P = len(lays)
    a = [backends[r].inverse_yz(uhats[r]) for r in range(P)]
    sends = [pack_a(lays[r], a[r]) for r in range(P)]
    xin = [unpack_a(lays[s], [sends[r][s] for r in range(P)]) for s in range(P)]
    xo = [backends[s].x_pass(xin[s]) for s in range(P)]
    sends = [pack_b(lays[s], xo[s]) for s in range(P)]
    yin = [unpack_b(lays[r], [sends[s][r] for s in range(P)]) for r in range(P)]
    return [backends[r].forward_yz(yin[r], uhats[r]) for r in range(P)]


class CudaSlab:
    """The CUDA backend of one rank: the ps_slab_* calls of the C ABI on
    device tensors (this class only allocates buffers, pads rows to the
    kernels' widths and passes pointers)."""

    def __init__(self, lay: SlabLayout, **plan_kwargs):
        import torch

        from . import ps
        self.ps = ps
        self.lay = lay
        self.forcing = plan_kwargs.get("forcing")
        cfg = ps.make_config(lay.nx, lay.ny, lay.nz, **plan_kwargs)
        self.dtype = torch.complex64 if cfg.prec == ps.Precision.FP32 else torch.complex128
        lo, hi = lay.kx_range()
        zlo, zhi = lay.z_range()
        self.handle = ps.ps_slab_create(cfg, lo, hi, zlo, zhi)
        self.info = ps.ps_slab_info_get(self.handle)

    def inverse_yz(self, uhat_local):
        import torch
        lay, i = self.lay, self.info
        out6 = torch.empty((6, lay.nz, lay.ny, i.kxp), dtype=self.dtype, device=uhat_local.device)
        self.ps.ps_slab_inverse(self.handle, uhat_local, out6)
        return out6[..., : i.ncx]

    def x_pass(self, xin):
        import torch
        i = self.info
        xp = torch.zeros((6, i.rows, i.cxp), dtype=self.dtype, device=xin.device)
        xp[..., : xin.shape[2]] = xin
        xo = torch.empty((3, i.rows, i.cxp), dtype=self.dtype, device=xin.device)
        self.ps.ps_slab_xpass(self.handle, xp, xo)
        return xo[..., : xin.shape[2]]

    def forward_yz(self, yin, uhat_local):
        import torch
        lay, i = self.lay, self.info
        yp = torch.zeros((3, lay.nz, lay.ny, i.kxp), dtype=self.dtype, device=yin.device)
        yp[..., : i.ncx] = yin
        out = torch.empty_like(uhat_local)
        self.ps.ps_slab_forward(self.handle, yp, uhat_local, out)
        self.ps.ps_slab_check(self.handle)
        return out

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.ps.ps_slab_destroy(self.handle)
            self.handle = None
