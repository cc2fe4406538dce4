"""The exact digit splitting behind the FP64-class tensor-core residuals, checked as a method
on the CPU with exact integer and rational arithmetic (no GPU, no oracle):

  * a double x with |x| < 2^e is the balanced base-256 number
    F = round(x 2^(55 - e)) = sum_{s=0..6} d_s 256^(6-s), d_1..d_6 in [-128, 127], |d_0| <= 128,
    so every digit is an integer that bf16 holds exactly, and |x - F 2^(e-55)| <= 2^(e-56);
  * a digit product has magnitude <= 2^14, so the order sums over a 64-wide k chunk of
    (g + 1) digit pairs, two real products each, stay below 2^24 (exact in FP32);
  * keeping the orders g = s + t <= 6 bounds the product error at a few units of 2^-52 of
    sum |Z||X| on rows and columns of very different scale, and dropping order 6 does not.
The GPU kernels implement these steps; tests/test_gpu_digit_gemm.py checks them directly against
the exact rational product on these operands, and the refined solves use them throughout.
"""
import math
import random
import struct
from fractions import Fraction

import numpy as np

BIAS = 0x0080808080808080  # 128 in each of the seven byte positions


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _fixed(x, e):
    """round(x 2^(55 - e)) from the bit pattern (ties away from zero)."""
    b = _bits(x)
    be, m = (b >> 52) & 0x7FF, b & ((1 << 52) - 1)
    if be:
        m |= 1 << 52
    else:
        be = 1
    sh = be - 1020 - e
    f = m << sh if sh >= 0 else ((m + (1 << (-sh - 1))) >> (-sh) if sh >= -60 else 0)
    return -f if b >> 63 else f


def _digits(x, e):
    g = (_fixed(x, e) + BIAS) & ((1 << 64) - 1)
    return [((g >> (8 * (6 - s))) & (0x1FF if s == 0 else 0xFF)) - 128 for s in range(7)]


def _exponent(values):
    m = max(abs(v) for v in values)
    return math.frexp(m)[1] if m > 0 else 0


def test_balanced_digits_reconstruct_the_rounded_value():
    rng = random.Random(7)
    vals = [rng.choice((-1, 1)) * rng.random() * 10 ** rng.uniform(-25, 8) for _ in range(4000)]
    vals += [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 0.5, -0.5, 3.5, 2.5, 1 - 2**-53, 127.75]
    for i in range(0, len(vals), 40):
        row = vals[i:i + 40]
        e = _exponent(row)
        for x in row:
            d = _digits(x, e)
            assert -128 <= d[0] <= 128 and all(-128 <= v <= 127 for v in d[1:])
            F = sum(v * 256 ** (6 - s) for s, v in enumerate(d))
            assert F == _fixed(x, e)
            assert abs(Fraction(x) - Fraction(F) * Fraction(2) ** (e - 55)) <= Fraction(2) ** (e - 56)


def test_order_sums_of_a_64_wide_chunk_fit_fp32():
    # worst case: every digit at its largest magnitude, order 6 (7 digit pairs, 2 real products)
    assert 7 * 2 * 64 * 128 * 128 < 2**24


def _product_error(gmax, seed=3, M=12, N=6, K=64):
    rng = np.random.default_rng(seed)
    rs = 10.0 ** rng.uniform(-3, 3, M)
    cs = 10.0 ** rng.uniform(-3, 3, N)
    Z = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * rs[:, None]
    for i in range(min(M, K)):
        Z[i, i] = complex(50 * Z[i, i].real, Z[i, i].imag)
    X = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))) * cs[None, :]
    ez = [_exponent(list(Z[i].real) + list(Z[i].imag)) for i in range(M)]
    ex = [_exponent(list(X[:, j].real) + list(X[:, j].imag)) for j in range(N)]
    dzr = [[_digits(Z[i, k].real, ez[i]) for k in range(K)] for i in range(M)]
    dzi = [[_digits(Z[i, k].imag, ez[i]) for k in range(K)] for i in range(M)]
    dxr = [[_digits(X[k, j].real, ex[j]) for k in range(K)] for j in range(N)]
    dxi = [[_digits(X[k, j].imag, ex[j]) for k in range(K)] for j in range(N)]
    worst = 0.0
    for i in range(M):
        for j in range(N):
            acc_r, acc_i = 0, 0  # sum_g V_g 256^(gmax - g), exact integers
            for g in range(gmax + 1):
                vr = vi = 0
                for s in range(g + 1):
                    t = g - s
                    if s > 6 or t > 6:
                        continue
                    for k in range(K):
                        a, b = dzr[i][k][s], dzi[i][k][s]
                        c, d = dxr[j][k][t], dxi[j][k][t]
                        vr += a * c - b * d
                        vi += a * d + b * c
                acc_r += vr * 256 ** (gmax - g)
                acc_i += vi * 256 ** (gmax - g)
            scale = Fraction(2) ** (ez[i] + ex[j] - 14 - 8 * gmax)
            exact_r = sum(Fraction(Z[i, k].real) * Fraction(X[k, j].real) - Fraction(Z[i, k].imag) * Fraction(X[k, j].imag)
                          for k in range(K))
            exact_i = sum(Fraction(Z[i, k].real) * Fraction(X[k, j].imag) + Fraction(Z[i, k].imag) * Fraction(X[k, j].real)
                          for k in range(K))
            err = math.hypot(float(acc_r * scale - exact_r), float(acc_i * scale - exact_i))
            worst = max(worst, err / float(np.sum(np.abs(Z[i]) * np.abs(X[:, j]))))
    return worst


def test_seven_digits_to_order_six_give_fp64_class_products():
    assert _product_error(6) < 4e-15


def test_dropping_order_six_is_visible():
    assert _product_error(5) > 2e-14
