"""Checkpoint and resume through the C ABI: bitwise continuation, the file
payload and checksum, and rejection of corrupted or mismatched files."""

import numpy as np
import pytest

from paper_1808_01309_gb300 import inputs

from .test_checkpoint import fnv1a64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


@pytest.mark.parametrize("eq", ["hd", "boussinesq"])
def test_resume_continues_bit_for_bit(ps, tmp_path, eq):
    n, dt = 32, 2e-3
    u = inputs.random_solenoidal_field(n, n, n, seed=4)
    kw = dict(nu=3e-3, forcing=torch.from_numpy(inputs.forcing_field(n, n, n, seed=2)).to("cuda", torch.complex64))
    if eq == "boussinesq":
        u = np.concatenate([u, inputs.random_scalar_field(n, n, n, seed=64)])
        kw.update(eq=ps.Equations.BOUSSINESQ, kappa=5e-3, n_bv=2.0)
    plan = ps.Plan(n, prec=ps.Precision.FP32, **kw)
    a = torch.from_numpy(u.astype(np.complex64)).cuda()
    for i in range(3):
        plan.rk_step(a, dt, t=i * dt)
    path = str(tmp_path / "s.ckpt")
    ps.ps_checkpoint_save(plan.handle, a, 3 * dt, 3, path)
    raw = open(path, "rb").read()
    payload = raw[136:]
    assert payload == a.cpu().numpy().tobytes()
    assert int.from_bytes(raw[128:136], "little") == fnv1a64(payload)
    for i in range(3, 6):
        plan.rk_step(a, dt, t=i * dt)
    plan2 = ps.Plan(n, prec=ps.Precision.FP32, **kw)
    b = torch.zeros_like(a)
    t, step = ps.ps_checkpoint_load(plan2.handle, b, path)
    assert (t, step) == (3 * dt, 3)
    for i in range(step, 6):
        plan2.rk_step(b, dt, t=i * dt)
    assert torch.equal(a, b)
    plan.close()
    plan2.close()


def test_corrupted_or_mismatched_checkpoints_are_rejected(ps, tmp_path):
    n = 16
    u = torch.from_numpy(inputs.random_solenoidal_field(n, n, n, seed=5).astype(np.complex64)).cuda()
    plan = ps.Plan(n, prec=ps.Precision.FP32, nu=1e-3)
    path = tmp_path / "c.ckpt"
    ps.ps_checkpoint_save(plan.handle, u, 0.5, 7, str(path))
    data = bytearray(path.read_bytes())
    data[136 + 1000] ^= 0x40
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(data))
    target = torch.ones_like(u)
    with pytest.raises(ps.PsError) as e:
        ps.ps_checkpoint_load(plan.handle, target, str(bad))
    assert e.value.status == ps.PS_ERR_INVALID_ARG
    assert torch.equal(target, torch.ones_like(u))  # untouched: checksum checked first
    other = ps.Plan(32, prec=ps.Precision.FP32, nu=1e-3)
    with pytest.raises(ps.PsError) as e:
        ps.ps_checkpoint_load(other.handle, torch.zeros((3, 32, 32, 17), dtype=torch.complex64, device="cuda"),
                              str(path))
    assert e.value.status == ps.PS_ERR_INVALID_ARG
    t, step = ps.ps_checkpoint_load(plan.handle, target, str(path))
    assert (t, step) == (0.5, 7) and torch.equal(target, u)
    plan.close()
    other.close()
