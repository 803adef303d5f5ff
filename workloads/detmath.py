"""Elementary functions from IEEE add, subtract, multiply and divide only.

The generators call exp, log, sin, cos and tanh on many values. numpy's versions
of these come from the platform's math library and its vector paths, which are
allowed to differ in the last bit between machines (an x86 host and an Arm
host give different tanh for some arguments), and numpy's matrix product goes
through BLAS, whose summation order and fused multiply-adds also vary. A
problem generated on one machine would then differ in a few ulps from the same
problem generated on another, and a solution cached on one could not be
compared with a solve on the other at the 1e-10 level of an ill-conditioned
system.

Every function here uses only elementwise float64 +, -, *, /, rint, floor and
exact power-of-two scaling (ldexp/frexp), each correctly rounded by IEEE 754,
in a fixed order, so the results are bit-identical on every IEEE machine. They
are accurate to a few ulps (checked against numpy in the tests), which is all a
problem generator needs.

Methods: Cody and Waite's additive range reduction (the reduction constant
split into a short head, exact when multiplied by the small integer quotient,
and a tail), then Taylor polynomials in nested (Horner) form on the reduced
interval; log through log(f) = 2 atanh((f - 1) / (f + 1)) on f in
[1/sqrt(2), sqrt(2)). The split constants were computed with 50-digit
arithmetic: LN2_HI is ln 2 rounded to 32 fractional bits, PIO2_1 is pi/2 rounded
to 30 bits and PIO2_2 the next 30 bits of the remainder.
"""
import numpy as np

LN2_HI = 0.6931471806019545
LN2_LO = -4.2009150726810846e-11
INV_LN2 = 1.4426950408889634
PIO2_1 = 1.5707963267341256
PIO2_2 = 6.077100541540537e-11
PIO2_3 = -3.50343439808993e-19
TWO_OVER_PI = 0.6366197723675814
LN10 = 2.302585092994046
SQRT_HALF = 0.7071067811865476


def _taylor_nested(r, degree, start=1):
    """sum_{k>=0} r^k / (start)(start+1)...(start+k-1) up to r^degree, i.e. for start = 1 the
    exponential series 1 + r (1 + r/2 (1 + r/3 (...))), evaluated innermost first."""
    acc = np.ones_like(r)
    for k in range(start + degree - 1, start - 1, -1):
        acc = 1.0 + (r / float(k)) * acc
    return acc


def exp(x):
    """e^x for float64 x (|x| < 700)."""
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x * INV_LN2)
    r = (x - k * LN2_HI) - k * LN2_LO          # |r| <= ~0.347
    p = _taylor_nested(r, 16)                  # remainder r^17/17! < 2e-22
    return np.ldexp(p, k.astype(np.int64))


def expm1(x):
    """e^x - 1, accurate in relative terms for small |x| (Taylor series x (1 + x/2 (1 + x/3 ...))
    for |x| < 1, e^x - 1 otherwise)."""
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 1.0
    xs = np.where(small, x, 0.0)
    # x * sum_{k>=0} x^k / (k+1)!  = x (1 + x/2 (1 + x/3 (1 + ...)))
    acc = np.ones_like(xs)
    for k in range(24, 1, -1):                 # remainder 1/25! < 1e-25
        acc = 1.0 + (xs / float(k)) * acc
    ps = xs * acc
    big = exp(np.where(small, 0.0, x)) - 1.0
    return np.where(small, ps, big)


def tanh(z):
    """tanh z = e / (e + 2) with e = expm1(2 |z|), odd in z; |z| >= 20 gives +-1."""
    z = np.asarray(z, dtype=np.float64)
    a = np.minimum(np.abs(z), 20.0)
    e = expm1(2.0 * a)
    t = e / (e + 2.0)
    return np.where(z < 0.0, -t, t)


def _reduce_pio2(x):
    """x = q (pi/2) + r with |r| <= ~pi/4 and q an integer (|x| < 2^20)."""
    q = np.rint(x * TWO_OVER_PI)
    r = ((x - q * PIO2_1) - q * PIO2_2) - q * PIO2_3
    return q.astype(np.int64), r


def _sin_poly(r):
    # r (1 - r^2/(2*3) (1 - r^2/(4*5) (1 - ...))), up to r^23
    r2 = r * r
    acc = np.ones_like(r)
    for k in range(22, 0, -2):
        acc = 1.0 - (r2 / float(k * (k + 1))) * acc
    return r * acc


def _cos_poly(r):
    # 1 - r^2/(1*2) (1 - r^2/(3*4) (1 - ...)), up to r^24
    r2 = r * r
    acc = np.ones_like(r)
    for k in range(23, 0, -2):
        acc = 1.0 - (r2 / float(k * (k + 1))) * acc
    return acc


def sin(x):
    x = np.asarray(x, dtype=np.float64)
    q, r = _reduce_pio2(x)
    s, c = _sin_poly(r), _cos_poly(r)
    qm = q & 3
    out = np.where(qm == 0, s, np.where(qm == 1, c, np.where(qm == 2, -s, -c)))
    return out


def cos(x):
    x = np.asarray(x, dtype=np.float64)
    q, r = _reduce_pio2(x)
    s, c = _sin_poly(r), _cos_poly(r)
    qm = q & 3
    out = np.where(qm == 0, c, np.where(qm == 1, -s, np.where(qm == 2, -c, s)))
    return out


def log(x):
    """Natural log of positive finite x."""
    x = np.asarray(x, dtype=np.float64)
    f, e = np.frexp(x)                          # x = f 2^e, f in [0.5, 1)
    low = f < SQRT_HALF
    f = np.where(low, 2.0 * f, f)
    e = np.where(low, e - 1, e).astype(np.float64)
    s = (f - 1.0) / (f + 1.0)                   # |s| <= 0.1716
    s2 = s * s
    # atanh(s) = s (1 + s^2/3 + s^4/5 + ...), Horner in s^2, up to s^2k with k = 14
    acc = np.zeros_like(s)
    for k in range(14, 0, -1):
        acc = s2 * (1.0 / float(2 * k + 1) + acc)
    logf = 2.0 * (s + s * acc)
    return e * LN2_HI + (e * LN2_LO + logf)


def pow10(x):
    """10^x = e^(x ln 10)."""
    return exp(np.asarray(x, dtype=np.float64) * LN10)
