"""Element-wise parity check shared by the GPU tests.

A field computed by the CUDA path is compared with the oracle's in two ways:
the relative L2 distance over the whole field, and a per-mode bound
max |got - ref| <= tol * max |ref|, so that a handful of wrong modes (one kx
column, a plane next to the Nyquist index, a tile edge) cannot hide in the
L2 norm of tens of millions of correct ones."""

import numpy as np


def parity_errors(got, ref):
    """(relative L2 distance, max |got - ref| / max |ref|)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    d = got - ref
    l2 = float(np.linalg.norm(d.ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))
    mx = float(np.max(np.abs(d)) / max(np.max(np.abs(ref)), 1e-300))
    return l2, mx


def assert_parity(got, ref, tol, what=""):
    l2, mx = parity_errors(got, ref)
    assert l2 <= tol, f"{what}: relative L2 {l2:.3e} > {tol:.1e}"
    assert mx <= tol, f"{what}: per-mode max error {mx:.3e} of max |ref| > {tol:.1e}"


# Band-limited fields at full size.  A field on |p|, |q|, |r| <= 5 has
# quadratic products on |p|, |q|, |r| <= 10, which a 32^3 grid (2/3
# half-width 10) holds without truncation or aliasing, as does any larger
# grid: the oracle's 32^3 result, placed at the same signed modes, is the
# exact result on the larger grid.
BAND_M, BAND_K = 32, 10


def embed_on_device(a, n, torch, dtype):
    """Places the modes |p|, |q|, |r| <= BAND_K of a 32^3 spectral field
    a[c, z, y, x] at the same signed modes of an n^3 field on the device."""
    m, K = BAND_M, BAND_K
    t = torch.zeros((a.shape[0], n, n, n // 2 + 1), dtype=dtype, device="cuda")
    src = torch.from_numpy(np.ascontiguousarray(a[:, :, :, : K + 1])).to("cuda", dtype)
    rows = [(i, (i if i < m // 2 else i - m) % n) for i in range(m) if abs(i if i < m // 2 else i - m) <= K]
    for zi, z in rows:
        for yi, y in rows:
            t[:, z, y, : K + 1] = src[:, zi, yi]
    return t


def assert_device_parity(got, exact, torch, tol, what=""):
    """assert_parity on device tensors (relative L2 and per-mode bound)."""
    d = got - exact
    l2 = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(exact))
    mx = float(d.abs().max() / exact.abs().max())
    assert l2 <= tol, f"{what}: relative L2 {l2:.3e} > {tol:.1e}"
    assert mx <= tol, f"{what}: per-mode max error {mx:.3e} of max |ref| > {tol:.1e}"
