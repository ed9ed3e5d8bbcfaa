"""FP64 CPU oracle for the pseudospectral Navier-Stokes right-hand side.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code, table or helper with the CUDA path.

It is a plain, slow, obviously-correct restatement of what the method
computes (Rosenberg et al., arXiv:1808.01309, Sec. 2), in float64 numpy:

* the discrete Fourier expansion of Eq. (fftsum) with the forward sum
  normalised by 1/(Nx Ny Nz) and the backward sum unnormalised, computed by a
  plain recursive mixed-radix Cooley-Tukey transform (:mod:`oracle.fft`; no
  FFT library),
* the Galerkin ODEs for the Fourier coefficients (Sec. 2, after Eq. fftsum),
  with the nonlinear term formed pointwise in physical space (rotational
  form u x omega) and transformed back,
* the pressure acting as a projection onto divergence-free fields,
* 2/3-rule dealiasing, and
* an explicit Runge-Kutta step (2nd or 4th order, Sec. 2) written with the
  viscous integrating factor (Lawson form),
* the MHD system (Eqs. uMHD, bMHD) and the Boussinesq system (Eqs. mom,
  temp, divv) with the same transforms, projection and Lawson scheme.

The readings taken where the paper is silent or garbled are listed in the
module docstring of :mod:`oracle.spectral`.

Pinning status: every function is pinned by ``tests/test_oracle_fft_pins.py``
(the transform against the direct O(N^2) sum at lengths 1-512 incl. primes,
impulses, tones, shift theorem, round trip), ``tests/test_oracle_pins.py``
(brute-force DFT, Parseval, closed-form flows, exact rational Taylor
coefficients, conservation laws, alias-free brute-force convolution, RK order),
``tests/test_oracle_mhd_pins.py``, ``tests/test_oracle_boussinesq_pins.py``
(exact rational tendency, brute-force scalar convolution, ideal energy
conservation, internal-wave frequency and RK4 order, exact diffusion) and
``tests/test_oracle_les_pins.py``; ``tests/test_oracle_planted.py`` plants
25 plausible mistakes (transform, curl, product, projection, RK, mask,
weights, box lengths, every LES basis tensor, the adjoint) and checks that
each one fails a pin.
"""

from .spectral import (  # noqa: F401
    Config,
    retained_halfwidth,
    wavenumbers,
    dealias_mask,
    hermitian_weight,
    forward,
    inverse,
    curl_hat,
    project,
    nonlinear,
    rhs,
    rk_step,
    diagnostics,
    mhd_nonlinear,
    mhd_rhs,
    mhd_rk_step,
    mhd_diagnostics,
    boussinesq_nonlinear,
    boussinesq_rhs,
    boussinesq_rk_step,
    boussinesq_diagnostics,
)
