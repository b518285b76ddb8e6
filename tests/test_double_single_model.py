"""The double-single accumulation of reading R14 (FP64-accuracy products
from FP32 arithmetic), modelled exactly on the CPU: every FP32 operation is
IEEE round-to-nearest (numpy float32), a fused multiply-add rounds the exact
a*b + c once (exact rational arithmetic).  The model follows the same steps
as the kernels: operands split as hi = rn32(v), lo = rn32(v - hi); per real
term p = rn32(ah bh), e = fma(ah, bh, -p) (exact), e += ah bl, e += al bh
(two fmas); the running pair (s, c) takes TwoSum(s, p) and c += t + e.  The
claim checked: a complex dot product of n terms ends within a few 2^-48 of
sum |b||x| of the exact FP64-input result, i.e. far inside the 1e-12 the GPU
tests ask of the double-single kernels, and some 2^24 times tighter than
rounding the operands to FP32.  Dropping a cross term or the TwoSum
correction breaks the bound."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def rn32(q):
    """Round an exact rational to the nearest float32 (ties to even)."""
    if q == 0:
        return F32(0.0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    # scale so that 2^23 <= m < 2^24
    while True:
        m = a * Fraction(2) ** (23 - e)
        if m >= 2 ** 24:
            e += 1
        elif m < 2 ** 23:
            e -= 1
        else:
            break
    n, r = divmod(m.numerator, m.denominator)
    rem = Fraction(r, m.denominator)
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return F32(sign * float(Fraction(n) * Fraction(2) ** (e - 23)))


def fma32(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def ds_mac(s, c, ah, al, bh, bl):
    p = F32(ah * bh)
    e = fma32(ah, bh, -p)
    e = fma32(ah, bl, e)
    e = fma32(al, bh, e)
    t_s = F32(s + p)
    bb = F32(t_s - s)
    t = F32(F32(s - F32(t_s - bb)) + F32(p - bb))
    c = F32(c + F32(t + e))
    return t_s, c


def split(v):
    hi = F32(v)
    return hi, F32(v - np.float64(hi))


def ds_dot(b, x):
    """sum_j b_j x_j (complex FP64 inputs) in the double-single model."""
    rh = rl = ih = il = F32(0.0)
    for bj, xj in zip(b, x):
        brh, brl = split(bj.real)
        bih, bil = split(bj.imag)
        xrh, xrl = split(xj.real)
        xih, xil = split(xj.imag)
        rh, rl = ds_mac(rh, rl, xrh, xrl, brh, brl)
        rh, rl = ds_mac(rh, rl, -xih, -xil, bih, bil)
        ih, il = ds_mac(ih, il, xrh, xrl, bih, bil)
        ih, il = ds_mac(ih, il, xih, xil, brh, brl)
    return complex(float(rh) + float(rl), float(ih) + float(il))


def exact_dot(b, x):
    re = sum(Fraction(bj.real) * Fraction(xj.real) - Fraction(bj.imag) * Fraction(xj.imag) for bj, xj in zip(b, x))
    im = sum(Fraction(bj.real) * Fraction(xj.imag) + Fraction(bj.imag) * Fraction(xj.real) for bj, xj in zip(b, x))
    return re, im


def test_rn32_matches_numpy_on_representable_sums():
    rng = np.random.default_rng(1)
    for _ in range(200):
        a, b = F32(rng.standard_normal()), F32(rng.standard_normal())
        assert rn32(Fraction(float(a)) + Fraction(float(b))) == F32(a + b)
        assert rn32(Fraction(float(a)) * Fraction(float(b))) == F32(a * b)


def test_double_single_dot_error_bound():
    rng = np.random.default_rng(2)
    n = 96
    for scale in (1.0, 1e-3, 1e4):
        b = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * scale
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        got = ds_dot(b, x)
        re, im = exact_dot(b, x)
        mag = float(sum(abs(bj) * abs(xj) for bj, xj in zip(b, x)))
        err = abs(complex(float(Fraction(got.real) - re), float(Fraction(got.imag) - im)))
        assert err <= 8 * 2.0 ** -48 * mag, (scale, err / mag)
        # rounding the operands to FP32 alone (no lo parts) is ~2^24 times worse
        plain = sum(complex(F32(bj.real), F32(bj.imag)) * complex(F32(xj.real), F32(xj.imag))
                    for bj, xj in zip(b, x))
        assert err < 1e-4 * abs(plain - complex(float(re), float(im))) + 1e-300
