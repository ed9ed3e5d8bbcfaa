"""Exact rational Fourier arithmetic for trigonometric-polynomial velocity
fields: an independent route to the Galerkin right-hand side used to pin the
oracle.  It uses the advective form -P[(u . grad) u] (not the rotational form
of the oracle), sums the convolution pair by pair, and works in Gaussian
rationals, so there is no rounding, no FFT and no dealiasing."""

from __future__ import annotations

from fractions import Fraction


class G:
    """Gaussian rational a + b i."""

    __slots__ = ("re", "im")

    def __init__(self, re=0, im=0):
        self.re = Fraction(re)
        self.im = Fraction(im)

    def __add__(self, o):
        return G(self.re + o.re, self.im + o.im)

    def __sub__(self, o):
        return G(self.re - o.re, self.im - o.im)

    def __mul__(self, o):
        if isinstance(o, G):
            return G(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)
        o = Fraction(o)
        return G(self.re * o, self.im * o)

    __rmul__ = __mul__

    def __neg__(self):
        return G(-self.re, -self.im)

    def conj(self):
        return G(self.re, -self.im)

    def abs2(self):
        return self.re * self.re + self.im * self.im

    def is_zero(self):
        return self.re == 0 and self.im == 0

    def __complex__(self):
        return complex(float(self.re), float(self.im))


I = G(0, 1)


def trig_modes(terms):
    """Full-spectrum coefficients {(p,q,r): [G,G,G]} of a sum of products of
    cos/sin of integer multiples of x, y, z (2 pi box)."""
    def axis(kind, m):
        if kind == "1" or m == 0:
            return [(0, G(1))] if kind != "s" else []
        if kind == "c":
            return [(m, G(Fraction(1, 2))), (-m, G(Fraction(1, 2)))]
        return [(m, G(0, Fraction(-1, 2))), (-m, G(0, Fraction(1, 2)))]

    out = {}
    for comp, amp, (kx, mx), (ky, my), (kz, mz) in terms:
        for p, cx in axis(kx, mx):
            for q, cy in axis(ky, my):
                for r, cz in axis(kz, mz):
                    v = out.setdefault((p, q, r), [G(), G(), G()])
                    v[comp] = v[comp] + cx * cy * cz * Fraction(amp)
    return out


def _clean(f):
    return {k: v for k, v in f.items() if not all(c.is_zero() for c in v)}


def add(a, b):
    out = {k: list(v) for k, v in a.items()}
    for k, v in b.items():
        w = out.setdefault(k, [G(), G(), G()])
        out[k] = [w[c] + v[c] for c in range(3)]
    return _clean(out)


def scale(a, s):
    return {k: [c * s for c in v] for k, v in a.items()}


def advect(u, v):
    """((u . grad) v)^(k) = sum_{p+q=k} sum_j u_j(p) (i q_j) v(q)."""
    out = {}
    for p, up in u.items():
        for q, vq in v.items():
            s = up[0] * q[0] + up[1] * q[1] + up[2] * q[2]
            if s.is_zero():
                continue
            s = I * s
            k = (p[0] + q[0], p[1] + q[1], p[2] + q[2])
            w = out.setdefault(k, [G(), G(), G()])
            out[k] = [w[c] + s * vq[c] for c in range(3)]
    return _clean(out)


def project(a):
    """P(k) a = a - k (k . a)/|k|^2, zero at k = 0."""
    out = {}
    for k, v in a.items():
        k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2]
        if k2 == 0:
            continue
        kd = v[0] * k[0] + v[1] * k[1] + v[2] * k[2]
        out[k] = [v[c] - kd * Fraction(k[c], k2) for c in range(3)]
    return _clean(out)


def curl(a):
    out = {}
    for k, v in a.items():
        out[k] = [I * (v[2] * k[1] - v[1] * k[2]),
                  I * (v[0] * k[2] - v[2] * k[0]),
                  I * (v[1] * k[0] - v[0] * k[1])]
    return _clean(out)


def euler_rate(u):
    """Inviscid Galerkin tendency -P[(u . grad) u]."""
    return scale(project(advect(u, u)), -1)


def inner(a, b):
    """sum_k Re(a(k)* . b(k)) over the full spectrum."""
    s = Fraction(0)
    for k, v in a.items():
        w = b.get(k)
        if w is None:
            continue
        for c in range(3):
            s += (v[c].conj() * w[c]).re
    return s
