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
