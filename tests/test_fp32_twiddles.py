"""Why the FP32 passes use correctly rounded twiddles and not compensated
(hi + lo) pairs: in an FP32 transform the rounding of the twiddle products
and of the butterfly additions dominates the error, so storing each twiddle
as an FP32 pair (w_hi + w_lo, w_lo the FP32 rounding of w - w_hi) and
multiplying by both changes the transform error by about 1 %, while it costs
a second complex multiplication per twiddle.  Even an ideal twiddle product
(formed exactly, then rounded once) lowers it only by about 15 %.

This is a CPU check on a float32 emulation of a radix-2 transform of length
512 (the kernels' radix-8 schedule has fewer twiddle multiplications, so
the twiddle share of its error is smaller still)."""

import numpy as np


def fft32(x, mode):
    n = len(x)
    bits = n.bit_length() - 1
    rev = np.array([int(format(i, f"0{bits}b")[::-1], 2) for i in range(n)])
    x = x.astype(np.complex64)[rev]
    length = 2
    while length <= n:
        k = np.arange(length // 2)
        w = np.exp(-2j * np.pi * k / length)
        w_hi = w.astype(np.complex64)
        a = x.reshape(-1, length)
        u, v = a[:, : length // 2].copy(), a[:, length // 2:].copy()
        if mode == "rounded":
            t = v * w_hi
        elif mode == "compensated":
            w_lo = (w - w_hi.astype(np.complex128)).astype(np.complex64)
            t = (v * w_hi + v * w_lo).astype(np.complex64)
        else:  # exact product, one rounding
            t = (v.astype(np.complex128) * w).astype(np.complex64)
        a[:, : length // 2] = u + t
        a[:, length // 2:] = u - t
        x = a.reshape(-1)
        length *= 2
    return x


def test_compensated_twiddles_do_not_pay_in_fp32():
    rng = np.random.default_rng(0)
    err = {m: [] for m in ("rounded", "compensated", "exact")}
    for _ in range(20):
        z = rng.standard_normal(512) + 1j * rng.standard_normal(512)
        ref = np.fft.fft(z)
        for m in err:
            err[m].append(np.linalg.norm(fft32(z, m) - ref) / np.linalg.norm(ref))
    e = {m: float(np.mean(v)) for m, v in err.items()}
    assert 5e-8 < e["rounded"] < 2e-7                    # a few FP32 roundings per level
    assert abs(e["compensated"] / e["rounded"] - 1) < 0.03  # compensation: about 1 %
    assert 0.75 < e["exact"] / e["rounded"] < 0.95       # even exact products: about 15 %
