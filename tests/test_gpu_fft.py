"""Unit tests of the line transforms the passes are built from, through the
plain 3D transforms of the C ABI (ps_fft_r2c / ps_fft_c2r): against a direct
DFT sum, numpy's FFT, and the round trip."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [16, 32, 48, 96, 128, 192, 256])
@pytest.mark.parametrize("nf", [1, 3])
def test_forward_and_backward_match_numpy(ps, n, nf):
    rng = np.random.default_rng(n + nf)
    x = rng.standard_normal((nf, n, n, n)).astype(np.float32)
    spec = torch.empty((nf, n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
    ps.ps_fft_r2c(n, nf, torch.from_numpy(x).cuda(), spec)
    ref = np.fft.rfftn(x.astype(np.float64), axes=(-3, -2, -1), norm="forward")
    got = spec.cpu().numpy().astype(np.complex128)
    assert relerr(got, ref) < 2e-6
    # backward of an exactly Hermitian spectrum (that of real data)
    h = np.fft.rfftn(rng.standard_normal((nf, n, n, n)), axes=(-3, -2, -1), norm="forward")
    phys = torch.empty((nf, n, n, n), dtype=torch.float32, device="cuda")
    hin = torch.from_numpy(h.astype(np.complex64)).cuda()
    ps.ps_fft_c2r(n, nf, hin, phys)
    assert torch.equal(hin.cpu(), torch.from_numpy(h.astype(np.complex64)))  # input untouched
    refp = np.fft.irfftn(h, s=(n, n, n), axes=(-3, -2, -1), norm="forward")
    assert relerr(phys.cpu().numpy().astype(np.float64), refp) < 2e-6


def test_forward_matches_a_direct_dft_sum(ps):
    """Selected coefficients against the definition (Eq. fftsum, normalised
    forward sum), summed point by point in float64."""
    n = 16
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, n, n, n)).astype(np.float32)
    spec = torch.empty((1, n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
    ps.ps_fft_r2c(n, 1, torch.from_numpy(x).cuda(), spec)
    got = spec.cpu().numpy()[0]
    idx = np.arange(n)
    z, y, xx = np.meshgrid(idx, idx, idx, indexing="ij")
    xd = x[0].astype(np.float64)
    for (r, q, p) in [(0, 0, 0), (1, 0, 0), (0, 3, 5), (15, 2, 8), (8, 8, 8), (5, 11, 7)]:
        phase = np.exp(-2j * np.pi * (p * xx + q * y + r * z) / n)
        want = np.sum(xd * phase) / n ** 3
        assert abs(got[r, q, p] - want) < 2e-7 * max(1.0, np.sqrt(np.mean(xd * xd)))


@pytest.mark.parametrize("n", [64, 512])
def test_round_trip(ps, n):
    rng = np.random.default_rng(n)
    x = torch.from_numpy(rng.standard_normal((2, n, n, n)).astype(np.float32)).cuda()
    spec = torch.empty((2, n, n, n // 2 + 1), dtype=torch.complex64, device="cuda")
    back = torch.empty_like(x)
    ps.ps_fft_r2c(n, 2, x, spec)
    ps.ps_fft_c2r(n, 2, spec, back)
    assert float(torch.linalg.vector_norm(back - x) / torch.linalg.vector_norm(x)) < 2e-6
