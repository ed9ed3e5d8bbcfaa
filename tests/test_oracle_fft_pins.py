"""Pins of the oracle's own transform (oracle/fft.py), CPU only.

The oracle computes the discrete Fourier sums of Eq. (fftsum) with a plain
recursive Cooley-Tukey factorisation.  These tests hold it to what the
definition and the mathematics fix, by routes that share none of its code:
the dense O(N^2) sum built here from cos/sin of float64 angles, exact
transforms of impulses and pure tones, the shift theorem, the round trip,
Parseval, and a third-party transform (numpy's pocketfft) as a cross-check."""

import math

import numpy as np
import pytest

from oracle import fft as offt


def direct_dft(x, sign):
    """X[k] = sum_n x[n] exp(sign 2 pi i k n/N) along the last axis, by the
    O(N^2) definition with k n reduced mod N before the angle is formed."""
    n = x.shape[-1]
    kn = np.mod(np.outer(np.arange(n), np.arange(n)), n)
    W = np.cos(2.0 * math.pi * kn / n) + 1j * sign * np.sin(2.0 * math.pi * kn / n)
    return x @ W.T


def rand_complex(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# lengths with every radix, mixtures of 2, 3 and 5, primes above 5 (dense
# fallback) and products with such primes
LENGTHS = list(range(1, 41)) + [48, 49, 60, 64, 77, 96, 120, 128, 143, 192, 256, 360, 512]


@pytest.mark.parametrize("n", LENGTHS)
@pytest.mark.parametrize("sign", [-1, +1])
def test_matches_the_direct_sum(n, sign):
    x = rand_complex((3, n), seed=n)
    got = offt.fft_last(x, sign)
    ref = direct_dft(x, sign)
    scale = np.linalg.norm(ref)
    # the direct sum itself carries O(N) eps of rounding per entry
    assert np.linalg.norm(got - ref) <= 4e-16 * max(n, 4) * scale


@pytest.mark.parametrize("n", [8, 12, 30, 96, 256])
def test_impulses_and_tones_are_exact(n):
    """An impulse at n0 transforms to exp(s 2 pi i k n0/N); the tone
    exp(-s 2 pi i k0 n/N) transforms to N at k0 and 0 elsewhere."""
    for n0 in (0, 1, n // 3, n - 1):
        x = np.zeros((1, n), dtype=np.complex128)
        x[0, n0] = 1.0
        got = offt.fft_last(x, -1)[0]
        kn = (np.arange(n) * n0) % n
        ang = 2.0 * math.pi * kn / n
        assert np.max(np.abs(got - (np.cos(ang) - 1j * np.sin(ang)))) < 1e-15
    for k0 in (0, 1, n // 2, n - 2):
        ang = 2.0 * math.pi * ((k0 * np.arange(n)) % n) / n
        tone = (np.cos(ang) - 1j * np.sin(ang))[None]
        got = offt.fft_last(tone, +1)[0]
        expect = np.zeros(n)
        expect[k0] = n
        assert np.max(np.abs(got - expect)) < 1e-13 * n


@pytest.mark.parametrize("n", [16, 45, 96, 100])
def test_shift_theorem_and_round_trip(n):
    x = rand_complex((4, n), seed=7 * n)
    X = offt.fft_last(x, -1)
    # x[n - 1] (circular shift by one) multiplies X[k] by exp(-2 pi i k/N)
    Xs = offt.fft_last(np.roll(x, 1, axis=-1), -1)
    ang = 2.0 * math.pi * np.arange(n) / n
    assert np.max(np.abs(Xs - X * (np.cos(ang) - 1j * np.sin(ang)))) < 1e-13 * np.max(np.abs(X))
    back = offt.fft_last(X, +1) / n
    assert np.max(np.abs(back - x)) < 1e-14 * np.max(np.abs(x)) * math.log2(n)
    # Parseval for the unnormalised pair
    assert abs(np.sum(np.abs(X) ** 2) - n * np.sum(np.abs(x) ** 2)) < 1e-13 * n * np.sum(np.abs(x) ** 2)


def test_transform_along_any_axis():
    x = rand_complex((6, 10, 12), seed=3)
    for ax in range(3):
        ref = np.moveaxis(direct_dft(np.moveaxis(x, ax, -1), -1), -1, ax)
        assert np.max(np.abs(offt.fft_axis(x, ax, -1) - ref)) < 1e-13


@pytest.mark.parametrize("shape", [(8, 6, 10), (12, 16, 8), (5, 7, 9)])
def test_real_transforms_match_the_direct_sum(shape):
    """rfft3 keeps kx = 0..Nx/2 of the normalised 3D sum; irfft3 of that half
    spectrum returns the data (odd lengths included)."""
    nz, ny, nx = shape
    u = np.random.default_rng(9).standard_normal((2, nz, ny, nx))
    full = direct_dft(u.astype(np.complex128), -1)
    full = np.moveaxis(direct_dft(np.moveaxis(full, -2, -1), -1), -1, -2)
    full = np.moveaxis(direct_dft(np.moveaxis(full, -3, -1), -1), -1, -3) / (nx * ny * nz)
    got = offt.rfft3(u)
    assert got.shape == (2, nz, ny, nx // 2 + 1)
    assert np.max(np.abs(got - full[..., : nx // 2 + 1])) < 1e-15 * nx * ny * nz
    assert np.max(np.abs(offt.irfft3(got, nz, ny, nx) - u)) < 1e-13


def test_tables_are_the_roots_of_unity():
    """Every DFT-matrix and twiddle entry is exp(s 2 pi i j/L) to within a
    few float64 roundings (of the angles formed in float64 here), with the
    symmetry w^(L-j) = conj(w^j) to one rounding, which a sign or index slip
    breaks."""
    for L in (2, 3, 5, 7, 16):
        F = offt.dft_matrix(L, -1)
        ang = 2.0 * math.pi * (np.outer(np.arange(L), np.arange(L)) % L) / L
        assert np.max(np.abs(F - (np.cos(ang) - 1j * np.sin(ang)))) < 1e-15
        assert np.max(np.abs(F[1, 1:] - np.conj(F[1, 1:][::-1]))) <= 2.3e-16
    for r, m in ((16, 32), (2, 3), (4, 24)):
        W = offt._twiddles(r, m, +1)[:, :, 0]
        ang = 2.0 * math.pi * (np.outer(np.arange(r), np.arange(m)) % (r * m)) / (r * m)
        assert np.max(np.abs(W - (np.cos(ang) + 1j * np.sin(ang)))) < 1e-15


def test_third_party_transform_agrees():
    """numpy's pocketfft, used here only as an outside cross-check."""
    x = rand_complex((5, 192), seed=1)
    assert np.max(np.abs(offt.fft_last(x, -1) - np.fft.fft(x))) < 1e-12
    u = np.random.default_rng(2).standard_normal((3, 32, 48, 64))
    ref = np.fft.rfftn(u, axes=(-3, -2, -1), norm="forward")
    assert np.max(np.abs(offt.rfft3(u) - ref)) < 1e-15 * np.max(np.abs(ref)) * 64
