"""A CPU backend for the slab decomposition (paper_1808_01309_gb300/slab.py),
for tests only.

It computes the local passes of one rank with the oracle's transforms
(oracle/fft.py) and the oracle's readings of the method (curl, mask,
projection, forcing, viscous term), on torch tensors so that the slab
module's exchanges (torch.distributed with gloo, or the loopback) move them.
With it the partition and both exchanges are checked against the oracle's
right-hand side on CPU processes; the CUDA backend runs the same exchanges
on the GPU."""

from __future__ import annotations

import math

import numpy as np
import torch

import oracle
from oracle import fft as offt
from oracle.spectral import Config, retained_halfwidth


class CpuBackend:
    def __init__(self, cfg: Config, lay, forcing_local=None):
        self.cfg = cfg
        self.lay = lay
        self.lo, self.hi = lay.kx_range()
        self.f = forcing_local
        n = cfg
        self.p = np.arange(self.lo, self.hi).reshape(1, 1, -1)
        q = np.arange(n.ny)
        r = np.arange(n.nz)
        self.q = np.where(q < (n.ny + 1) // 2, q, q - n.ny).reshape(1, -1, 1)
        self.r = np.where(r < (n.nz + 1) // 2, r, r - n.nz).reshape(-1, 1, 1)
        self.kx = 2 * math.pi / n.lx * self.p
        self.ky = 2 * math.pi / n.ly * self.q
        self.kz = 2 * math.pi / n.lz * self.r
        Kx = retained_halfwidth(n.nx, n.dealias)
        Ky = retained_halfwidth(n.ny, n.dealias)
        Kz = retained_halfwidth(n.nz, n.dealias)
        self.D = (np.abs(self.p) <= Kx) & (np.abs(self.q) <= Ky) & (np.abs(self.r) <= Kz)

    def inverse_yz(self, uhat_local):
        u = uhat_local.numpy() * self.D
        om = 1j * np.stack([self.ky * u[2] - self.kz * u[1], self.kz * u[0] - self.kx * u[2],
                            self.kx * u[1] - self.ky * u[0]])
        a = np.concatenate([u, om])
        a = offt.fft_axis(a, 1, +1)
        a = offt.fft_axis(a, 2, +1)
        return torch.from_numpy(a)

    def x_pass(self, xin):
        c = self.cfg
        nh, cx = c.nx // 2 + 1, xin.shape[2]
        half = np.zeros((6, xin.shape[1], nh), dtype=np.complex128)
        half[:, :, :cx] = xin.numpy()
        full = np.empty((6, xin.shape[1], c.nx), dtype=np.complex128)
        full[..., :nh] = half
        full[..., nh:] = np.conj(half[..., c.nx - nh:0:-1])
        phys = offt.fft_axis(full, 2, +1).real
        n = np.cross(phys[:3], phys[3:], axis=0)
        return torch.from_numpy(offt.fft_axis(n.astype(np.complex128), 2, -1)[..., :cx])

    def forward_yz(self, yin, uhat_local):
        c = self.cfg
        v = offt.fft_axis(yin.numpy(), 2, -1)
        v = offt.fft_axis(v, 1, -1) / (c.nx * c.ny * c.nz)
        v = v * self.D
        if self.f is not None:
            v = v + self.f.numpy() * self.D
        k2 = self.kx ** 2 + self.ky ** 2 + self.kz ** 2
        kd = self.kx * v[0] + self.ky * v[1] + self.kz * v[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.where(k2 > 0, kd / np.where(k2 > 0, k2, 1.0), 0.0)
        proj = np.stack([v[0] - self.kx * s, v[1] - self.ky * s, v[2] - self.kz * s])
        proj = np.where(k2 > 0, proj, 0.0) * self.D
        out = proj - c.nu * k2 * uhat_local.numpy() * self.D
        return torch.from_numpy(out)


def local_columns(field, lay):
    """The kx columns of this rank from a global state [c, nz, ny, nh]."""
    lo, hi = lay.kx_range()
    return torch.from_numpy(np.ascontiguousarray(field[..., lo:hi]))


def assemble(parts, lays, nh):
    """Global [c, nz, ny, nh] from every rank's kx columns (zero beyond them)."""
    c, nz, ny = parts[0].shape[:3]
    out = np.zeros((c, nz, ny, nh), dtype=np.complex128)
    for part, lay in zip(parts, lays):
        lo, hi = lay.kx_range()
        out[..., lo:hi] = np.asarray(part)
    return out


def oracle_rhs(u, cfg, f):
    return oracle.rhs(u, cfg, forcing=f)
