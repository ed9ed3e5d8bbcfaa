"""The slab decomposition on the GPU: the CUDA passes of P ranks' kx and z
slabs (ps_slab_* through the C ABI), exchanged by the loopback of
paper_1808_01309_gb300/slab.py in one process, assemble to the oracle's
right-hand side mode by mode (FP64 1e-12, FP32 2e-6), uneven splits and an
anisotropic box included.  The gloo version of the same exchanges runs on
CPU processes in tests/test_slab.py."""

import math

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs, slab

from .parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n3,P,forced", [((32, 32, 32), 2, True), ((48, 32, 64), 3, True), ((64, 16, 32), 4, False),
                                         ((128, 64, 96), 2, True)])
def test_slab_ranks_assemble_the_oracle_rhs(ps, prec, n3, P, forced):
    nx, ny, nz = n3
    P_, dtype, tol = ((ps.Precision.FP64, torch.complex128, 1e-12) if prec == "fp64"
                      else (ps.Precision.FP32, torch.complex64, 2e-6))
    lx, ly, lz = 2 * math.pi, 3.0, 5.0
    u = inputs.random_solenoidal_field(nx, ny, nz, seed=11, ly=ly, lz=lz)
    f = inputs.forcing_field(nx, ny, nz, seed=2, ly=ly, lz=lz) if forced else None
    cfg = oracle.Config(nx, ny, nz, lx=lx, ly=ly, lz=lz, nu=2e-3)
    cx = slab.retained_columns(nx)
    lays = [slab.SlabLayout(nx, ny, nz, cx, P, r) for r in range(P)]

    def local(field, lay):
        lo, hi = lay.kx_range()
        return torch.from_numpy(np.ascontiguousarray(field[..., lo:hi])).to("cuda", dtype)

    backends = [slab.CudaSlab(lay, prec=P_, nu=2e-3, lx=lx, ly=ly, lz=lz,
                              forcing=local(f, lay) if forced else None) for lay in lays]
    parts = slab.rhs_loopback(backends, lays, [local(u, lay) for lay in lays])
    got = np.zeros((3, nz, ny, nx // 2 + 1), dtype=np.complex128)
    for part, lay in zip(parts, lays):
        lo, hi = lay.kx_range()
        got[..., lo:hi] = part.cpu().numpy()
    for b in backends:
        b.close()
    assert_parity(got, oracle.rhs(u, cfg, forcing=f), tol, f"{P} slabs {n3} {prec}")


def test_slab_rejects_bad_ranges(ps):
    cfg = ps.make_config(32, prec=ps.Precision.FP32)
    for args in ((0, 0, 0, 32), (5, 12, 0, 32), (0, 11, 0, 33), (3, 2, 0, 32), (0, 11, 16, 16)):
        with pytest.raises(ps.PsError) as e:
            ps.ps_slab_create(cfg, *args)
        assert e.value.status == ps.PS_ERR_INVALID_ARG
    with pytest.raises(ps.PsError) as e:
        ps.ps_slab_create(ps.make_config(32, eq=ps.Equations.MHD), 0, 11, 0, 32)
    assert e.value.status == ps.PS_ERR_UNSUPPORTED
