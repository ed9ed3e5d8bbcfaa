"""Checkpoint header parsing (ps_checkpoint_info) on files written here from
the documented format with Python's struct module; no GPU needed."""

import math
import struct

import pytest


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


def fnv1a64(data: bytes) -> int:
    """FNV-1a, 64 bit, from its published definition."""
    h = 0xCBF29CE484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def write_file(path, nx=8, ny=8, nz=16, prec=0, eq=2, dealias=0, rk=4, ncomp=4, box=(1.0, 2.0, 3.0),
               coef=(1e-3, 2e-3, 1.5, 4e-3), t=0.25, step=17, payload=None, magic=b"PSCKPT\x00\x01",
               version=1, hbytes=136, checksum=None):
    vb = 8 if prec == 0 else 16
    n = ncomp * nz * ny * (nx // 2 + 1) * vb
    if payload is None:
        payload = bytes((i * 7) % 251 for i in range(n))
    hdr = magic + struct.pack("<II", version, hbytes)
    hdr += struct.pack("<8i", nx, ny, nz, prec, eq, dealias, rk, ncomp)
    hdr += struct.pack("<8d", *box, *coef, t)
    hdr += struct.pack("<qQQ", step, len(payload), fnv1a64(payload) if checksum is None else checksum)
    assert len(hdr) == 136
    with open(path, "wb") as f:
        f.write(hdr + payload)


def test_fnv1a_reference_values():
    # published test vectors of FNV-1a 64
    assert fnv1a64(b"") == 0xCBF29CE484222325
    assert fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert fnv1a64(b"foobar") == 0x85944171F73967E8


def test_info_reads_the_documented_header(ps, tmp_path):
    p = tmp_path / "a.ckpt"
    write_file(p)
    cfg, t, step = ps.ps_checkpoint_info(str(p))
    assert (cfg.nx, cfg.ny, cfg.nz) == (8, 8, 16)
    assert cfg.prec == ps.Precision.FP32 and cfg.eq == ps.Equations.BOUSSINESQ
    assert cfg.dealias == 0 and cfg.rk_order == 4
    assert (cfg.lx, cfg.ly, cfg.lz) == (1.0, 2.0, 3.0)
    assert (cfg.nu, cfg.eta, cfg.n_bv, cfg.kappa) == (1e-3, 2e-3, 1.5, 4e-3)
    assert t == 0.25 and step == 17
    assert not cfg.forcing


@pytest.mark.parametrize("bad", [dict(magic=b"PSCKPT\x00\x02"), dict(version=2), dict(hbytes=128),
                                 dict(ncomp=3), dict(payload=b"\x00" * 16), dict(prec=7)])
def test_info_rejects_inconsistent_headers(ps, tmp_path, bad):
    p = tmp_path / "b.ckpt"
    write_file(p, **bad)
    with pytest.raises(ps.PsError) as e:
        ps.ps_checkpoint_info(str(p))
    assert e.value.status == ps.PS_ERR_INVALID_ARG


def test_info_rejects_missing_and_truncated_files(ps, tmp_path):
    with pytest.raises(ps.PsError):
        ps.ps_checkpoint_info(str(tmp_path / "missing.ckpt"))
    p = tmp_path / "c.ckpt"
    write_file(p)
    data = p.read_bytes()
    p.write_bytes(data[:100])
    with pytest.raises(ps.PsError) as e:
        ps.ps_checkpoint_info(str(p))
    assert e.value.status == ps.PS_ERR_INVALID_ARG
