"""Golden fixtures (tests/golden/*.txt): exact rational tendencies of
trigonometric flows, written by tests/golden/make_golden.py.  The oracle is
checked against them on the CPU, the CUDA path on the GPU."""

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs
from tests.golden.make_golden import FIELDS

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
N = 32  # every product mode (|k| <= 6 per axis) lies inside the 2/3 cube K = 10


def load(name):
    modes, inv = {}, {}
    for line in open(os.path.join(HERE, name + ".txt")):
        if line.startswith("# energy"):
            t = line.split()
            inv = {"energy": Fraction(t[2]), "enstrophy": Fraction(t[4])}
        if line.startswith("#") or not line.strip():
            continue
        p, q, r, c, re, im = line.split()
        modes[(int(p), int(q), int(r), int(c))] = complex(float(Fraction(re)), float(Fraction(im)))
    return modes, inv


def expected(modes, n):
    out = np.zeros((3, n, n, n // 2 + 1), dtype=np.complex128)
    for (p, q, r, c), v in modes.items():
        if p >= 0:
            out[c, r % n, q % n, p] = v
    return out


@pytest.mark.parametrize("name", sorted(FIELDS))
def test_fixture_is_current(name):
    """The stored file equals what the generator writes now."""
    import tempfile
    from tests.golden import make_golden as mg
    title, terms = FIELDS[name]
    with tempfile.TemporaryDirectory() as d:
        old = mg.HERE
        mg.HERE = d
        try:
            mg.write(name, title, terms)
        finally:
            mg.HERE = old
        assert open(os.path.join(d, name + ".txt")).read() == open(os.path.join(HERE, name + ".txt")).read()


@pytest.mark.parametrize("name", sorted(FIELDS))
def test_oracle_matches_golden(name):
    modes, inv = load(name)
    _, terms = FIELDS[name]
    u = inputs.trig_field(N, N, N, terms)
    cfg = oracle.Config(N, N, N, nu=0.0)
    got = oracle.rhs(u, cfg)
    exp = expected(modes, N)
    assert np.max(np.abs(exp)) > 0.01
    assert np.max(np.abs(got - exp)) < 1e-15
    d = oracle.diagnostics(u, cfg)
    assert abs(d["energy"] - float(inv["energy"])) < 1e-15
    assert abs(d["enstrophy"] - float(inv["enstrophy"])) < 1e-14


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(FIELDS))
def test_cuda_path_matches_golden(name, prec):
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps
    modes, _ = load(name)
    _, terms = FIELDS[name]
    u = inputs.trig_field(N, N, N, terms)
    P, dt = (ps.Precision.FP64, torch.complex128) if prec == "fp64" else (ps.Precision.FP32, torch.complex64)
    plan = ps.Plan(N, prec=P, nu=0.0)
    got = plan.rhs(torch.from_numpy(u).to("cuda", dt))
    torch.cuda.synchronize()
    got = got.cpu().numpy().astype(np.complex128)
    exp = expected(modes, N)
    rel = np.linalg.norm(got - exp) / np.linalg.norm(exp)
    assert rel < (1e-12 if prec == "fp64" else 2e-6)
    plan.close()
