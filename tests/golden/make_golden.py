"""Writes the golden fixtures of this directory by exact rational Fourier
arithmetic (tests/exact_fourier.py: advective form, Gaussian rationals, no
FFT and no rounding), independently of the oracle and of the CUDA path.

Each fixture lists the nonzero Fourier coefficients of the inviscid Galerkin
tendency -P[(u . grad) u] of a trigonometric velocity field on the 2 pi box
(the right-hand side of Eq. mom with Eq. divv, Sec. 2, for nu = 0 and no
forcing), one line per mode and component:  p q r component re im, the
numbers written as exact fractions.  Run:  python -m tests.golden.make_golden
"""

from __future__ import annotations

import os
from fractions import Fraction

from tests import exact_fourier as xf

HERE = os.path.dirname(os.path.abspath(__file__))

FIELDS = {
    # Taylor & Green (1937): u = (sin x cos y cos z, -cos x sin y cos z, 0)
    "taylor_green": ("Taylor-Green vortex u = (sin x cos y cos z, -cos x sin y cos z, 0)",
                     [(0, 1, ("s", 1), ("c", 1), ("c", 1)), (1, -1, ("c", 1), ("s", 1), ("c", 1))]),
    # crossed shear: u = (sin y, 0, sin x)
    "crossed_shear": ("crossed shear u = (sin y, 0, sin x)",
                      [(0, 1, ("1", 0), ("s", 1), ("1", 0)), (2, 1, ("s", 1), ("1", 0), ("1", 0))]),
    # two-scale field with modes up to 3 on each axis
    "two_scale": ("two-scale field u = (sin 2y cos z, sin 3z, cos 2x sin y)",
                  [(0, 1, ("1", 0), ("s", 2), ("c", 1)), (1, 1, ("1", 0), ("1", 0), ("s", 3)),
                   (2, 1, ("c", 2), ("s", 1), ("1", 0))]),
}


def fmt(x: Fraction) -> str:
    return f"{x.numerator}/{x.denominator}" if x.denominator != 1 else f"{x.numerator}"


def write(name, title, terms):
    u = xf.trig_modes(terms)
    rate = xf.euler_rate(u)
    lines = [f"# {title}",
             "# inviscid Galerkin tendency -P[(u . grad) u] (Eq. mom with Eq. divv, Sec. 2; nu = 0, no forcing)",
             "# exact rational arithmetic (tests/exact_fourier.py), full spectrum, 2 pi box",
             "# p q r component re im"]
    for (p, q, r) in sorted(rate):
        v = rate[(p, q, r)]
        for c in range(3):
            if not v[c].is_zero():
                lines.append(f"{p} {q} {r} {c} {fmt(v[c].re)} {fmt(v[c].im)}")
    e0 = xf.inner(u, u) / 2
    w = xf.curl(u)
    lines.append(f"# energy {fmt(e0)} enstrophy {fmt(xf.inner(w, w) / 2)}")
    with open(os.path.join(HERE, name + ".txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


def main():
    for name, (title, terms) in FIELDS.items():
        write(name, title, terms)


if __name__ == "__main__":
    main()
