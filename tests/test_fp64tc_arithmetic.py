"""The exact-digit arithmetic behind the FP64_TC products, restated here in
plain Python integers (independent of the CUDA code), and its error bound.

Scheme (Ozaki, Ogita, Oishi and Rump, 2012: split floating-point operands into
slices whose products a low-precision unit sums exactly): every row is scaled
by S = 2^(e-1022), e its largest biased exponent, so |x| < S; the magnitude
|x| / S is cut into 8 digits of 7 bits, x = sign S sum_{p=1..8} d_p 2^(-7p)
(bits below 2^-56 S truncated).  A product keeps the digit pairs with
p + q <= 9 (36 of 64): per chunk of 32 values of k the level sums
L_t = sum_{p+q=t} sum_k d_p d_q are integers below 2^22, so BF16 products
with FP32 accumulation are exact; the levels are folded into two int64 words
and rounded to FP64 once.

Bound checked: |v - w.y| <= 2^-53 |v| + C K S_w S_y with
C = 127^2 sum_{t>=10} n_t 2^(-7t) + 2 * 2^-56 ~ 1.24e-16 (the dropped pairs,
n_t of them at level t, and the truncated bits of both operands)."""
from fractions import Fraction

import numpy as np

BOUND_C = 1.25e-16


def _bits(x):
    return int(np.frombuffer(np.float64(x).tobytes(), dtype=np.uint64)[0])


def _expo(x):
    return (_bits(x) >> 52) & 0x7FF


def _digits(x, emax):
    """sign and d_1..d_8 of x in a row whose largest biased exponent is emax."""
    b = _bits(x)
    ex = (b >> 52) & 0x7FF
    f = 0
    if ex:
        m = (b & ((1 << 52) - 1)) | (1 << 52)
        sh = ex - emax + 3                      # f = |x| 2^(1078 - emax) < 2^56
        f = m << sh if sh >= 0 else (m >> -sh if sh > -64 else 0)
    assert f < 1 << 56
    sg = -1 if b >> 63 else 1
    return sg, [(f >> (56 - 7 * p)) & 127 for p in range(1, 9)]


def _product(w, y):
    """v ~ sum_k w_k y_k by the digit scheme; also the level-sum maximum."""
    ea = max(_expo(v) for v in w)
    eb = max(_expo(v) for v in y)
    dw = [_digits(v, ea) for v in w]
    dy = [_digits(v, eb) for v in y]
    hi = lo = 0
    lmax = 0
    for k0 in range(0, len(w), 32):
        lev = [0] * 17                          # levels t = p + q, 2..16
        for k in range(k0, min(len(w), k0 + 32)):
            (sa, a), (sb, b) = dw[k], dy[k]
            for p in range(1, 9):
                for q in range(1, 10 - p):      # p + q <= 9
                    lev[p + q] += sa * sb * a[p - 1] * b[q - 1]
        lmax = max(lmax, max(abs(v) for v in lev))
        hi += sum(lev[t] << (7 * (5 - t)) for t in range(2, 6))
        lo += sum(lev[t] << (7 * (9 - t)) for t in range(6, 10))
    assert abs(hi) < 1 << 53 and abs(lo) < 1 << 53          # exact as doubles
    # one rounding of hi 2^-35 + lo 2^-63, scaled by S_w S_y (a power of two)
    e = (ea - 1022) + (eb - 1022)
    v = float(Fraction(hi, 1 << 35) + Fraction(lo, 1 << 63)) * 2.0 ** e
    return v, Fraction(2) ** e, lmax


def test_bound_constant():
    drop = sum(Fraction(127 ** 2 * n) * Fraction(2) ** (-7 * t)
               for t, n in zip(range(10, 17), range(7, 0, -1)))
    assert float(drop + 2 * Fraction(2) ** -56) < BOUND_C


def test_digit_products_within_bound():
    rng = np.random.default_rng(7)
    worst = 0.0
    for trial in range(150):
        K = int(rng.integers(1, 80))
        w = rng.standard_normal(K) * 10.0 ** rng.uniform(-3, 3, K)
        y = rng.standard_normal(K) * 10.0 ** rng.uniform(-3, 3, K)
        if trial % 5 == 0:
            w[: K // 2] = 0.0
        if trial % 7 == 0:                       # equal magnitudes: digits near 127
            y[:] = np.sign(y) * (2.0 - 2.0 ** -52)
        v, scale, lmax = _product(w, y)
        assert lmax < 1 << 22                    # every FP32 partial sum is exact
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(w, y))
        err = abs(Fraction(v) - exact)
        assert err <= Fraction(2) ** -53 * abs(Fraction(v)) + Fraction(BOUND_C) * K * scale
        worst = max(worst, float(err / (K * scale)))
    assert worst < BOUND_C


def test_exact_for_short_significands():
    """Entries with at most 7 significant bits are represented exactly by
    their leading digits, so small integer rows multiply exactly."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        K = int(rng.integers(1, 70))
        w = rng.integers(-127, 128, K).astype(np.float64)
        y = rng.integers(-127, 128, K).astype(np.float64)
        v, _, _ = _product(w, y)
        assert v == float(np.dot(w.astype(np.int64), y.astype(np.int64)))
