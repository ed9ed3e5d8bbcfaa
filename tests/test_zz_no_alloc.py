"""ps_rhs_noalloc: the right-hand side for callers that cannot allocate device
memory (a host program whose allocator owns the device, a plugin that must
keep the footprint fixed).  It must give the same result as the plan-based
ps_rhs and as the FP64 oracle, call after call, while using only its static
scratch array, for every dealiasing rule and at the largest documented size.

This file is named so that pytest collects it last."""

import math

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs

from .parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6}


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


def relerr(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,n3,forced,dealias", [
    ("fp64", (32, 32, 32), True, "cubic"), ("fp32", (64, 32, 16), True, "cubic"),
    ("fp32", (64, 64, 64), False, "cubic"), ("fp32", (32, 64, 16), True, "spherical"),
    ("fp64", (16, 32, 64), False, "spherical"), ("fp32", (32, 32, 32), True, "none"),
    # the largest documented case: 64^3 FP64, forced, no dealiasing (about
    # 31 MB of the 32 MiB array; the scratch offsets are tightest here)
    ("fp64", (64, 64, 64), True, "none")])
def test_noalloc_matches_plan_rhs_on_consecutive_calls(ps, prec, n3, forced, dealias):
    nx, ny, nz = n3
    P = ps.Precision.FP64 if prec == "fp64" else ps.Precision.FP32
    dtype = torch.complex128 if prec == "fp64" else torch.complex64
    D = {"cubic": ps.Dealias.CUBIC, "spherical": ps.Dealias.SPHERICAL, "none": ps.Dealias.NONE}[dealias]
    OD = {"cubic": oracle.spectral.CUBIC, "spherical": oracle.spectral.SPHERICAL,
          "none": oracle.spectral.NONE}[dealias]
    dev = torch.device("cuda:0")
    fh = inputs.forcing_field(nx, ny, nz, seed=2, ly=3.0) if forced else None
    f = torch.from_numpy(fh).to(dev, dtype) if forced else None
    kw = dict(prec=P, nu=2e-3, lx=2 * math.pi, ly=3.0, lz=2 * math.pi, forcing=f, dealias=D)
    plan = ps.Plan(nx, ny, nz, **kw)
    cfg = ps.make_config(nx, ny, nz, **kw)
    ocfg = oracle.Config(nx, ny, nz, ly=3.0, nu=2e-3, dealias=OD)
    for seed in (1, 7):  # two calls in a row, different inputs
        uh = inputs.random_solenoidal_field(nx, ny, nz, seed=seed, ly=3.0)
        u = torch.from_numpy(uh).to(dev, dtype)
        ref = plan.rhs(u)
        out = torch.full_like(u, float("nan"))
        ps.ps_rhs_noalloc(cfg, u, out)
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(out)).all()
        assert relerr(out, ref) < TOL[prec]
        # and against the oracle itself, mode by mode
        got = out.cpu().numpy().astype(np.complex128)
        assert_parity(got, oracle.rhs(uh, ocfg, forcing=fh), TOL[prec], f"noalloc {dealias} seed {seed}")
    plan.close()


def test_noalloc_rejects_grids_beyond_its_scratch(ps):
    # rejected on the host before any launch
    u = torch.zeros((3, 256, 256, 129), dtype=torch.complex64, device="cuda")
    out = torch.zeros_like(u)
    cfg = ps.make_config(256, prec=ps.Precision.FP32)
    with pytest.raises(ps.PsError) as e:
        ps.ps_rhs_noalloc(cfg, u, out)
    assert e.value.status == ps.PS_ERR_INVALID_ARG
    assert "static array" in str(e.value)
