"""The C-ABI library builds, loads and exports every symbol include/ps.h
declares; host-side argument checks return the documented status without
touching a GPU."""

import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


def header_functions():
    src = open(os.path.join(ROOT, "include", "ps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ps_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_path():
    names = header_functions()
    for n in ("ps_plan_create", "ps_plan_destroy", "ps_rhs", "ps_rk_step", "ps_diagnostics"):
        assert n in names


def test_library_exports_every_declared_symbol(ps):
    lib = ps.load()
    for name in header_functions():
        assert hasattr(lib, name), name
    assert set(header_functions()) <= set(ps.SYMBOLS)


def test_status_strings(ps):
    lib = ps.load()
    assert lib.ps_status_string(0) == b"ok"
    assert lib.ps_status_string(1) == b"invalid argument"
    assert lib.ps_kind_name(2) == b"x_fused"
    assert lib.ps_kind_name(99) == b"?"


@pytest.mark.parametrize("bad", [
    dict(nx=12), dict(nx=4), dict(ny=2048), dict(nz=0), dict(nx=24), dict(nx=384), dict(lx=0.0), dict(ly=-1.0),
    dict(lz=math.inf), dict(rk_order=3), dict(nu=-1e-3), dict(nu=math.nan),
    dict(dealias=7), dict(prec=5),
])
def test_invalid_configs_are_rejected_before_any_cuda_call(ps, bad):
    kw = dict(nx=32, ny=32, nz=32)
    kw.update(bad)
    nx, ny, nz = kw.pop("nx"), kw.pop("ny"), kw.pop("nz")
    cfg = ps.make_config(nx, ny, nz, **kw)
    with pytest.raises(ps.PsError) as e:
        ps.ps_plan_create(cfg)
    assert e.value.status == ps.PS_ERR_INVALID_ARG
    with pytest.raises(ps.PsError):
        ps.ps_plan_workspace_bytes(cfg)


def test_mhd_rejects_negative_diffusivity(ps):
    cfg = ps.make_config(32, eq=ps.Equations.MHD, eta=-1.0)
    with pytest.raises(ps.PsError) as e:
        ps.ps_plan_create(cfg)
    assert e.value.status == ps.PS_ERR_INVALID_ARG


@pytest.mark.parametrize("bad", [dict(kappa=-1.0), dict(kappa=math.nan), dict(n_bv=math.inf), dict(eq=3)])
def test_boussinesq_rejects_bad_parameters(ps, bad):
    kw = dict(eq=ps.Equations.BOUSSINESQ, kappa=1e-3, n_bv=1.0)
    kw.update(bad)
    cfg = ps.make_config(32, **kw)
    with pytest.raises(ps.PsError) as e:
        ps.ps_plan_create(cfg)
    assert e.value.status == ps.PS_ERR_INVALID_ARG


def test_boussinesq_workspace_holds_the_scalar_fields(ps):
    # 9 fields into the x pass instead of 6 (u, omega, grad theta), 4 out
    # instead of 3, 4-component stage buffers
    hd = ps.ps_plan_workspace_bytes(ps.make_config(128))
    bq = ps.ps_plan_workspace_bytes(ps.make_config(128, eq=ps.Equations.BOUSSINESQ, kappa=1e-3, n_bv=1.0))
    assert 1.35 < bq / hd < 1.55


def test_mhd_workspace_is_about_twice_hd(ps):
    hd = ps.ps_plan_workspace_bytes(ps.make_config(128))
    mhd = ps.ps_plan_workspace_bytes(ps.make_config(128, eq=ps.Equations.MHD))
    assert 1.9 < mhd / hd < 2.1


def test_null_arguments(ps):
    lib = ps.load()
    assert lib.ps_rhs(None, None, None, 0.0) == ps.PS_ERR_INVALID_ARG
    assert lib.ps_rk_step(None, None, 0.1, 0.0) == ps.PS_ERR_INVALID_ARG
    assert lib.ps_plan_destroy(None) == ps.PS_OK
    assert lib.ps_plan_create(None, None, None) == ps.PS_ERR_INVALID_ARG


def test_workspace_bytes_scale_with_the_retained_cube(ps):
    b32 = ps.ps_plan_workspace_bytes(ps.make_config(32))
    b64 = ps.ps_plan_workspace_bytes(ps.make_config(64))
    b64d = ps.ps_plan_workspace_bytes(ps.make_config(64, prec=ps.Precision.FP64))
    assert 6 < b64 / b32 < 10
    assert 1.9 < b64d / b64 < 2.1
    # 512^3 FP32: two 6-field intermediates and two compact 3-field stage buffers
    b512 = ps.ps_plan_workspace_bytes(ps.make_config(512))
    assert 4.0e9 < b512 < 5.5e9


@pytest.mark.parametrize("n,nf", [(8, 1), (1024, 1), (100, 1), (64, 0), (64, 17)])
def test_plain_transforms_check_their_arguments(ps, n, nf):
    lib = ps.load()
    assert lib.ps_fft_r2c(n, nf, 1, 2, None) == ps.PS_ERR_INVALID_ARG
    assert lib.ps_fft_c2r(n, nf, 1, 2, None) == ps.PS_ERR_INVALID_ARG
    assert lib.ps_fft_r2c(64, 1, None, None, None) == ps.PS_ERR_INVALID_ARG



def test_test_hook_and_probe_reject_bad_arguments_on_the_host(ps):
    lib = ps.load()
    assert lib.ps_plan_set_wait_test(None, 10) == ps.PS_ERR_INVALID_ARG
    assert lib.ps_probe_fma_tflops(1, None, None) == ps.PS_ERR_INVALID_ARG
    import ctypes
    out = ctypes.c_double()
    assert lib.ps_probe_fma_tflops(7, None, ctypes.byref(out)) == ps.PS_ERR_INVALID_ARG


@pytest.mark.parametrize("prec,addr", [(0, 0x1004), (1, 0x1008)])
def test_misaligned_forcing_is_rejected_before_any_cuda_call(ps, prec, addr):
    cfg = ps.make_config(32, prec=ps.Precision(prec), forcing=addr)
    with pytest.raises(ps.PsError) as e:
        ps.ps_plan_create(cfg)
    assert e.value.status == ps.PS_ERR_INVALID_ARG
    assert "aligned" in str(e.value)


def test_every_entry_point_rejects_null_arguments_on_the_host(ps):
    """Every call of the ABI, given NULL handles, NULL pointers and zero sizes,
    returns PS_ERR_INVALID_ARG with a message before any CUDA call (this runs
    without a GPU); the destroy calls accept NULL as a no-op."""
    import ctypes
    lib = ps.load()
    strings = ("ps_kind_name", "ps_status_string", "ps_last_error")
    for name in ps.SYMBOLS:
        if name in strings:
            continue
        fn = getattr(lib, name)
        args = []
        for t in fn.argtypes:
            if t in (ctypes.c_double, ctypes.c_float):
                args.append(0.0)
            elif t in (ctypes.c_int, ctypes.c_uint, ctypes.c_longlong):
                args.append(0)
            else:
                args.append(None)
        st = fn(*args)
        if name.endswith("_destroy"):
            assert st == ps.PS_OK, name
        else:
            assert st == ps.PS_ERR_INVALID_ARG, (name, st)
            assert lib.ps_last_error(), name
