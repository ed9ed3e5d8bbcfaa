"""Host-side parts of the LES workflow (paper_1808_01309_gb300/les.py) that
run without a GPU: the parameter layout of the network, the normalisation
statistics and the shell transfer spectrum used to evaluate the closures,
checked against the oracle's spectrum and weights; CPU only."""

import math

import numpy as np
import pytest

import oracle
from paper_1808_01309_gb300 import inputs, les, ps

torch = pytest.importorskip("torch")


def test_parameter_vector_layout():
    p = les.init_params(seed=3, out_scale=0.1)
    assert p.dtype == np.float32 and p.size == ps.MLP_NPARAM
    sizes = [int(np.prod(s)) for _, s in les.SHAPES]
    assert sum(sizes) == p.size == 5 * 64 + 64 + 64 * 64 + 64 + 64 * 6 + 6
    parts = np.split(p, np.cumsum(sizes)[:-1])
    named = dict(zip([n for n, _ in les.SHAPES], parts))
    for b in ("b1", "b2", "b3"):
        assert np.all(named[b] == 0)
    # weights with variance 1/fan_in, the output layer scaled down
    assert abs(np.std(named["W2"]) * math.sqrt(64) - 1) < 0.05
    assert abs(np.std(named["W3"]) * math.sqrt(64) / 0.1 - 1) < 0.15
    assert np.array_equal(p, les.init_params(seed=3, out_scale=0.1))


def test_calibration_statistics():
    rng = np.random.default_rng(1)
    X = torch.from_numpy(rng.standard_normal((4096, 5)) * [1, 2, 3, 4, 0] + [0, 1, 2, 3, 7]).float()
    A = torch.from_numpy(rng.standard_normal((4096, 9)) * 0.5).float()
    T = torch.from_numpy(rng.standard_normal((4096, 6)) * 0.2).float()
    c = les.calibrate(X, A, T)
    assert np.allclose(c["mean"], [0, 1, 2, 3, 7], atol=0.15)
    assert np.allclose(c["std"][:4], [1, 2, 3, 4], rtol=0.05)
    assert c["std"][4] == 1.0  # a constant input is left unscaled
    assert abs(c["s_A"] - 0.5 * 3.0) < 0.05      # rms |A| over 9 components of std 0.5
    assert abs(c["s_tau"] - 0.2) < 0.01


def test_shell_transfer_against_the_oracle_spectrum():
    n, kc = 32, 10
    cfg = oracle.Config(n, n, n)
    u = inputs.random_solenoidal_field(n, n, n, seed=5)
    # f = u: the transfer spectrum is twice the energy spectrum
    T_uu = les.shell_transfer(torch.from_numpy(u), torch.from_numpy(u), kc)
    E = oracle.diagnostics(u, cfg)["spectrum"]
    assert np.allclose(T_uu, 2 * E[: kc + 1], rtol=1e-13, atol=1e-16)
    # summed over every shell it is sum w Re(u* . f) with the oracle's
    # Hermitian weights, here on arrays with content on every stored mode
    # (the kx = n/2 plane included)
    rng = np.random.default_rng(4)
    shape = (3, n, n, n // 2 + 1)
    uf = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    T = les.shell_transfer(torch.from_numpy(uf), torch.from_numpy(f), 40)
    w = oracle.hermitian_weight(cfg)
    total = float(np.sum(w * np.real(np.sum(np.conj(uf) * f, axis=0))))
    assert abs(T.sum() - total) < 1e-13 * max(1.0, abs(total))
