"""Plain mixed-radix Cooley-Tukey transforms in float64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module, and it shares no code, table or constant with the CUDA
path.

The transform is the discrete Fourier sum of the paper's Eq. (fftsum) along
one axis, X[k] = sum_n x[n] exp(s 2 pi i k n / N) with s = -1 (forward) or
+1 (backward), unnormalised.  It is computed by the Cooley-Tukey
factorisation written out once and applied recursively:

  N = r m, input index n = m n1 + n2 (n1 < r, n2 < m),
  output index k = k1 + r k2 (k1 < r, k2 < m):

  X[k1 + r k2] = sum_{n2} w_m^{n2 k2} [ w_N^{n2 k1} ( sum_{n1} w_r^{n1 k1} x[m n1 + n2] ) ]

with w_L = exp(s 2 pi i / L): r-point DFTs over n1 for every n2, a twiddle
multiplication by w_N^{n2 k1}, then m-point transforms over n2 for every k1
(the recursion), and the output read with k1 fastest.  The radix r is the
first of 16, 8, 4, 2, 3, 5 dividing N (powers of two first: fewer levels of
the recursion, each of which moves the whole array); a length with no such
factor (1 or a prime above 5, or a product of those) is transformed by its
dense DFT matrix.  Every small DFT is the definition as a matrix product (one
library matmul over all independent lines at once).  DFT-matrix entries and
twiddles are
exp(s 2 pi i j/L) with the exponent j reduced mod L in integers and cos/sin
evaluated in numpy long double, then rounded to float64.

The real transforms of the state are built from the complex one: the forward
transform of real data keeps kx = 0..Nx/2 of the complex transform along x;
the backward transform rebuilds the full x spectrum from the stored half by
X[Nx - p] = conj(X[p]) (paper Sec. 2: the Hermitian symmetry of real data,
reading R3) and keeps the real part.
"""

from __future__ import annotations

import functools

import numpy as np

RADICES = (16, 8, 4, 2, 3, 5)


@functools.lru_cache(maxsize=None)
def _two_pi_ld():
    return np.longdouble(8) * np.arctan(np.longdouble(1))


def _roots(j: np.ndarray, length: int, sign: int) -> np.ndarray:
    """exp(sign 2 pi i j/length) for integer j, evaluated in long double."""
    jj = np.mod(j, length).astype(np.longdouble)
    ang = _two_pi_ld() * jj / np.longdouble(length)
    c = np.cos(ang).astype(np.float64)
    s = np.sin(ang).astype(np.float64)
    return c + 1j * sign * s


@functools.lru_cache(maxsize=None)
def dft_matrix(length: int, sign: int) -> np.ndarray:
    """F[k, n] = exp(sign 2 pi i k n/length): the DFT by its definition."""
    k = np.arange(length).reshape(-1, 1)
    n = np.arange(length).reshape(1, -1)
    return _roots(k * n, length, sign)


@functools.lru_cache(maxsize=None)
def _twiddles(r: int, m: int, sign: int) -> np.ndarray:
    """w_N^{k1 n2}, N = r m, as an (r, m, 1) array (k1, n2, broadcast batch)."""
    k1 = np.arange(r).reshape(-1, 1)
    n2 = np.arange(m).reshape(1, -1)
    return _roots(k1 * n2, r * m, sign).reshape(r, m, 1)


def _radix(n: int) -> int:
    """First radix of RADICES dividing n, or n itself (dense DFT)."""
    for r in RADICES:
        if n % r == 0:
            return r
    return n


def fft_first(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised DFT along axis 0 of a 2D array x[n, b] (b: independent
    lines), exp(sign 2 pi i k n/N), by the recursive Cooley-Tukey
    factorisation of the module docstring."""
    n, B = x.shape
    if n == 1:
        return np.array(x, dtype=np.complex128)
    r = _radix(n)
    if r == n:  # a radix, or a length without a factor 2, 3 or 5
        return dft_matrix(n, sign) @ x
    m = n // r
    # x[m n1 + n2, b] viewed as rows n1 of an (r, m B) matrix
    y = dft_matrix(r, sign) @ x.reshape(r, m * B)          # r-point DFTs over n1
    y = y.reshape(r, m, B) * _twiddles(r, m, sign)          # y[k1, n2, b] w_N^{k1 n2}
    y = np.ascontiguousarray(y.transpose(1, 0, 2))          # [n2, k1, b]
    z = fft_first(y.reshape(m, r * B), sign)                # [k2, (k1, b)]: m-point DFTs over n2
    return z.reshape(n, B)                                  # row k2 r + k1 = X[k1 + r k2]


def fft_axis(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """Unnormalised DFT of x along `axis` (any number of other axes)."""
    x = np.asarray(x, dtype=np.complex128)
    xa = np.moveaxis(x, axis, 0)
    shape = xa.shape
    y = fft_first(np.ascontiguousarray(xa).reshape(shape[0], -1), sign)
    return np.moveaxis(y.reshape(shape), 0, axis)


def fft_last(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised DFT along the last axis."""
    return fft_axis(x, -1, sign)


def rfft3(u: np.ndarray) -> np.ndarray:
    """Forward transform of real data over the last three axes (z, y, x),
    normalised by 1/(Nx Ny Nz), keeping kx = 0..Nx/2 (Eq. fftsum with readings
    R1-R3).  One 3D field at a time (leading axes are looped over)."""
    u = np.asarray(u, dtype=np.float64)
    nz, ny, nx = u.shape[-3:]
    nh = nx // 2 + 1
    lead = u.shape[:-3]
    out = np.empty(lead + (nz, ny, nh), dtype=np.complex128)
    for idx in np.ndindex(*lead):
        a = fft_axis(u[idx], -1, -1)[..., :nh]
        a = fft_axis(a, -2, -1)
        a = fft_axis(a, -3, -1)
        out[idx] = a / (nx * ny * nz)
    return out


def irfft3(uh: np.ndarray, nz: int, ny: int, nx: int) -> np.ndarray:
    """Backward transform (unnormalised sum with exp(+...)) of a half spectrum
    over the last three axes to real data on the nz x ny x nx grid: z and y
    transforms of the stored modes, the full x spectrum from the Hermitian
    symmetry X[Nx - p] = conj(X[p]), the x transform and its real part."""
    uh = np.asarray(uh, dtype=np.complex128)
    nh = nx // 2 + 1
    assert uh.shape[-3:] == (nz, ny, nh), "half spectrum shape"
    lead = uh.shape[:-3]
    out = np.empty(lead + (nz, ny, nx), dtype=np.float64)
    for idx in np.ndindex(*lead):
        a = fft_axis(uh[idx], -3, +1)
        a = fft_axis(a, -2, +1)
        full = np.empty((nz, ny, nx), dtype=np.complex128)
        full[..., :nh] = a
        full[..., nh:] = np.conj(a[..., nx - nh:0:-1])  # X[p] = conj(X[nx - p]), p = nh..nx-1
        out[idx] = fft_axis(full, -1, +1).real
    return out
