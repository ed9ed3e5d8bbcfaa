"""Why the FP32 MHD induction term loses accuracy on large grids, and which
form would not: a CPU check on a float32 emulation (numpy's single-precision
FFT) of the induction term N_B = curl(u x B) of band-limited seeded u and B
(|p|, |q|, |r| <= 5), whose exact value the FP64 oracle gives on a 32^3 grid.

Curl form (the kernels' form, Eq. bMHD as i k x F[u x B]): the float32
product u x B and its transform carry rounding noise on every retained mode,
and the curl multiplies that noise by |k|, so the relative error of N_B
doubles with each doubling of the grid.  Advective form (B . grad) u -
(u . grad) B (equal for divergence-free u and B): the derivatives act on the
exact low-k fields before the products, so the noise is not amplified and
the error stays flat.  The GPU measurement shows the same growth (relative
L2 1.7e-6, 3.6e-6, 7.2e-6 at 128^3, 256^3, 512^3)."""

import numpy as np

import oracle
from paper_1808_01309_gb300 import inputs

M, K = 32, 10  # the exact grid and its 2/3 half-width


def embed(a, n):
    """Modes |p|, |q|, |r| <= K of a 32^3 spectral field at the same signed modes of n^3."""
    t = np.zeros((a.shape[0], n, n, n // 2 + 1), dtype=np.complex128)
    for zi in range(M):
        z = zi if zi < M // 2 else zi - M
        for yi in range(M):
            y = yi if yi < M // 2 else yi - M
            if abs(z) <= K and abs(y) <= K:
                t[:, z % n, y % n, : K + 1] = a[:, zi, yi, : K + 1]
    return t


def wavenumbers(n):
    s = np.fft.fftfreq(n, 1.0 / n)
    return (np.arange(n // 2 + 1).reshape(1, 1, -1).astype(np.float32),
            s.reshape(1, -1, 1).astype(np.float32), s.reshape(-1, 1, 1).astype(np.float32))


def phys32(h, n):
    """float32 physical field of a spectral field (Fourier-series coefficients)."""
    return np.fft.irfftn(h.astype(np.complex64) * np.float32(n ** 3), s=(n, n, n), axes=(-3, -2, -1))


def spec32(x, n):
    return np.fft.rfftn(x, axes=(-3, -2, -1)) / np.float32(n ** 3)


def induction_errors(n):
    u = inputs.random_solenoidal_field(M, M, M, seed=1, kmax=(5, 5, 5))
    b = inputs.random_solenoidal_field(M, M, M, seed=51, kmax=(5, 5, 5))
    cfg = oracle.Config(M, M, M)
    _, nb = oracle.mhd_nonlinear(np.concatenate([u, b]), cfg)
    exact = embed(nb, n)
    uh, bh = embed(u, n), embed(b, n)
    kx, ky, kz = wavenumbers(n)
    k = (kx, ky, kz)
    kn = (n + 2) // 3 - 1  # the grid's 2/3 half-width: every retained mode is compared
    keep = (kx <= kn) & (np.abs(ky) <= kn) & (np.abs(kz) <= kn)
    keep = np.broadcast_to(keep, exact.shape[1:])
    # curl form: i k x F[u x B]
    U, B = phys32(uh, n), phys32(bh, n)
    E = spec32(np.cross(U, B, axis=0), n)
    curl = np.stack([1j * (k[1] * E[2] - k[2] * E[1]), 1j * (k[2] * E[0] - k[0] * E[2]),
                     1j * (k[0] * E[1] - k[1] * E[0])])
    # advective form: (B . grad) u - (u . grad) B, gradients from the spectra
    gu = [[phys32(1j * k[j] * uh[i], n) for j in range(3)] for i in range(3)]
    gb = [[phys32(1j * k[j] * bh[i], n) for j in range(3)] for i in range(3)]
    adv = np.stack([sum(B[j] * gu[i][j] - U[j] * gb[i][j] for j in range(3)) for i in range(3)])
    adv = spec32(adv.astype(np.float32), n)

    def rel(x):
        d = (x - exact)[:, keep]
        return float(np.linalg.norm(d) / np.linalg.norm(exact[:, keep]))

    return rel(curl), rel(adv)


def test_curl_form_error_grows_with_the_grid_and_advective_form_does_not():
    e = {n: induction_errors(n) for n in (32, 64, 128)}
    curl = [e[n][0] for n in (32, 64, 128)]
    adv = [e[n][1] for n in (32, 64, 128)]
    # each doubling of the grid roughly doubles the curl form's error
    # (emulation: 2.1e-7, 3.6e-7, 6.9e-7 at 32^3, 64^3, 128^3)
    assert 1.5 < curl[1] / curl[0] < 2.5 and 1.5 < curl[2] / curl[1] < 2.5
    # the advective form's stays within FP32 rounding of a few transforms
    # (1.6e-7, 1.7e-7, 1.9e-7)
    assert max(adv) < 1e-6 and adv[2] / adv[0] < 1.5
    assert curl[2] > 2.5 * adv[2]
