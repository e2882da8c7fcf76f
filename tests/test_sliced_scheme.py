"""The arithmetic of the sliced tensor-core Schur updates (the dgemm updates
of Sec. 4.4 made FP64-accurate on bf16 tensor cores by exact integer
splitting, after Ozaki et al.), checked on the host in exact integer and
rational arithmetic.  These are properties of the method the sliced kernels
implement, restated here from its definition; the kernels themselves are
checked against the oracle by the GPU tests.

For one output entry C_ij -= sum_q L_iq d_q L_jq over K <= 64 panel columns:
  * each column is balanced by h_q = floor(floor(log2 |d_q|) / 2):
    a_q = L_iq 2^h_q, b_q = fl(L_jq d_q) 2^-h_q, so a_q^2 and b_q^2 are
    within a factor 4 of L^2 |d_q| whatever the spread of the pivots;
  * a row gets one power-of-two scale 2^E (|entries| < 2^E) and its entries
    become 56-bit integers X = rint(a 2^(56 - E)), written as eight balanced
    base-2^7 digits x_0..x_7 (|x_t| <= 64 for t >= 1, |x_0| <= 128), each
    exactly a bf16;
  * the digit products with t + u = d are summed into S_d (d <= 7, 36
    products); every partial sum is an integer below 40960 K <= 2^21.4, so
    FP32 accumulation is exact in any order;
  * hi = sum_{d<4} S_d 2^(7 (3 - d)), lo = sum_{d>=4} S_d 2^(7 (7 - d)),
    T = hi 2^28 + lo is kept as floor(T / 2^8) (below 2^62) and the product
    is that integer times 2^(E_a + E_b - 55), rounded once to a double.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

NDIG = 8      # digits per operand
BASE = 7      # bits per digit
KMAX = 64     # panel columns per accumulation (a pair of 32-column panels)


def balanced_digits(x):
    """Eight balanced base-2^7 digits of an integer |x| <= 2^56, most
    significant first: x = sum_t d[t] 2^(7 (7 - t))."""
    d = [0] * NDIG
    for t in range(NDIG - 1, 0, -1):
        r = ((x + 64) % 128) - 64
        d[t] = r
        x = (x - r) // 128
    d[0] = x
    return d


def is_bf16(v):
    """v (an integer) is exactly representable in bf16 (8 significant bits)."""
    f = np.float32(v)
    bits = f.view(np.uint32)
    return int(bits & np.uint32(0xFFFF)) == 0 and float(f) == v


def frexp_exp(v):
    """The E with 2^(E-1) <= |v| < 2^E (v != 0), from the binary exponent."""
    return math.frexp(v)[1]


def balance_shift(dq):
    """h = floor(floor(log2 |d|) / 2) for a normal pivot d (0 for d = 0)."""
    if dq == 0.0:
        return 0
    return (math.frexp(dq)[1] - 1) >> 1


def row_scale(vals):
    """The smallest E with |v| < 2^E for every nonzero v of the row."""
    es = [frexp_exp(v) for v in vals if v != 0.0]
    return max(es) if es else None


def to_int56(v, E):
    """rint(v 2^(56 - E)), ties away from zero (|v| < 2^E, so |X| <= 2^56)."""
    s = Fraction(v) * Fraction(2) ** (56 - E)
    mag = abs(s)
    q = int(mag)
    if mag - q >= Fraction(1, 2):
        q += 1
    return q if s >= 0 else -q


def round_half_up_53(t, e):
    """t 2^e as a double: |t| rounded to 53 significant bits, halves up
    (away from zero), sign applied after."""
    a = abs(t)
    if a == 0:
        return 0.0
    n = a.bit_length()
    if n > 53:
        sh = n - 53
        a = (a + (1 << (sh - 1))) >> sh
        e += sh
    v = math.ldexp(float(a), e)
    return -v if t < 0 else v


def sliced_product(Li, Lj, d, balance=True):
    """The sliced approximation of sum_q L_iq d_q L_jq, with its scales
    (balance=False: every h_q = 0, to show what the balancing is for)."""
    h = [balance_shift(x) if balance else 0 for x in d]
    a = [math.ldexp(Li[q], h[q]) for q in range(len(d))]
    b = [math.ldexp(Lj[q] * d[q], -h[q]) for q in range(len(d))]
    Ea, Eb = row_scale(a), row_scale(b)
    if Ea is None or Eb is None:
        return 0.0, 0, 0, [0] * NDIG, 0
    X = [balanced_digits(to_int56(v, Ea)) for v in a]
    Y = [balanced_digits(to_int56(v, Eb)) for v in b]
    S = [0] * NDIG
    for q in range(len(d)):
        for t in range(NDIG):
            for u in range(NDIG - t):
                S[t + u] += X[q][t] * Y[q][u]
    hi = sum(S[dd] << (BASE * (3 - dd)) for dd in range(4))
    lo = sum(S[dd] << (BASE * (7 - dd)) for dd in range(4, 8))
    tq = (hi << 20) + (lo >> 8)  # floor(T / 2^8), T = hi 2^28 + lo
    return round_half_up_53(tq, Ea + Eb - 55), Ea, Eb, S, tq


def per_column_bound(d):
    """The largest |S_d| one panel column adds: the products t + u = d with
    |x_0|, |y_0| up to 128 and the other digits up to 64."""
    return sum((128 if t == 0 else 64) * (128 if d - t == 0 else 64) for t in range(d + 1))


def test_digits_exact_bounded_and_bf16():
    rng = random.Random(1)
    cases = [0, 1, -1, 63, 64, 65, -64, -65, 127, 128, 2 ** 56, -(2 ** 56), 2 ** 56 - 1, -(2 ** 56 - 1),
             2 ** 49, 2 ** 49 - 1, 64 * sum(128 ** t for t in range(7)), -64 * sum(128 ** t for t in range(7))]
    cases += [rng.randint(-(2 ** 56), 2 ** 56) for _ in range(5000)]
    for x in cases:
        d = balanced_digits(x)
        assert sum(dt << (BASE * (NDIG - 1 - t)) for t, dt in enumerate(d)) == x
        assert all(abs(dt) <= 64 for dt in d[1:]), (x, d)
        assert abs(d[0]) <= 128, (x, d)
        assert all(is_bf16(dt) for dt in d)


def test_accumulators_exact_in_fp32():
    per_col = [per_column_bound(d) for d in range(NDIG)]
    assert max(per_col) == 40960
    assert 40960 * KMAX < 2 ** 22
    # worst-case magnitudes summed in a random order in FP32 stay exact
    rng = np.random.default_rng(2)
    for d in range(NDIG):
        terms = []
        for _ in range(KMAX):
            for t in range(d + 1):
                sa = 128 if t == 0 else 64
                sb = 128 if d - t == 0 else 64
                terms.append(int(rng.choice([-1, 1])) * sa * sb)
        for _ in range(20):
            rng.shuffle(terms)
            acc = np.float32(0.0)
            for v in terms:
                acc = np.float32(acc + np.float32(v))
            assert int(acc) == sum(terms)


def test_balancing_keeps_both_operands_within_factor_four():
    rng = random.Random(3)
    for _ in range(2000):
        L = rng.uniform(-10, 10)
        d = rng.choice([-1, 1]) * 10.0 ** rng.uniform(-8, 8)
        h = balance_shift(d)
        a2 = math.ldexp(L, h) ** 2
        b2 = math.ldexp(L * d, -h) ** 2
        ref = L * L * abs(d)
        assert ref / 4 * (1 - 1e-14) <= a2 <= ref * (1 + 1e-14)
        assert ref * (1 - 1e-14) <= b2 <= 4 * ref * (1 + 1e-14)


def test_recombination_fits_int64():
    # the largest possible |S_d| for K = 64, all with one sign
    S = [per_column_bound(d) * KMAX for d in range(NDIG)]
    hi = sum(S[d] << (BASE * (3 - d)) for d in range(4))
    lo = sum(S[d] << (BASE * (7 - d)) for d in range(4, 8))
    assert hi < 2 ** 42 and lo < 2 ** 42
    assert abs((hi << 20) + (lo >> 8)) < 2 ** 63


@pytest.mark.parametrize("spread", [0.0, 4.0, 8.0])
def test_sliced_product_error_bound(spread):
    """|sliced - exact| <= 2^(E_a + E_b) (K 2^-52 + 2^-55) + 2^-52 |sliced|:
    per column the rounding of fl(L_jq d_q) (2^-53), the two 56-bit operand
    roundings (2^-56 together) and the dropped digit products t + u >= 8
    (below 2^-55), all relative to 2^(E_a + E_b); then the floor of T / 2^8
    and the final rounding.  Pivots spread over 10^(-spread)..10^spread."""
    rng = random.Random(4 + int(spread))
    for trial in range(60):
        K = rng.choice([1, 7, 32, 33, 64])
        Li = [rng.uniform(-3, 3) * (0 if rng.random() < 0.1 else 1) for _ in range(K)]
        Lj = [rng.uniform(-3, 3) * (0 if rng.random() < 0.1 else 1) for _ in range(K)]
        d = [rng.choice([-1, 1]) * 10.0 ** rng.uniform(-spread, spread) for _ in range(K)]
        approx, Ea, Eb, S, tq = sliced_product(Li, Lj, d)
        exact = sum(Fraction(Li[q]) * Fraction(d[q]) * Fraction(Lj[q]) for q in range(K))
        if Ea == 0 and Eb == 0 and approx == 0.0:
            assert exact == 0 or all(x == 0 for x in Li) or all(x == 0 for x in Lj)
            continue
        assert all(abs(s) <= 40960 * K for s in S)
        assert abs(tq) < 2 ** 62
        scale = Fraction(2) ** (Ea + Eb)
        bound = scale * (K * Fraction(1, 2 ** 52) + Fraction(1, 2 ** 55)) + abs(Fraction(approx)) / 2 ** 52
        assert abs(Fraction(approx) - exact) <= bound, (trial, K, float(abs(Fraction(approx) - exact)), float(bound))


def test_balancing_keeps_fp64_accuracy_across_pivot_spreads():
    """Two columns whose products are both 1: one with large L and a tiny
    pivot, one with small L and a huge pivot.  Unbalanced, the row scales of
    a and b both come from the large entries (1e4), so the products are
    resolved only to about 2^-54 of 1e8: a relative error near 1e-8, which
    refinement could not remove at these pivot spreads.  Balanced, both
    operands of each column are near 1 and the result is FP64-accurate."""
    Li = [1e4, 1e-4]
    Lj = [1e4, 1e-4]
    d = [1e-8, 1e8]
    exact = sum(Fraction(Li[q]) * Fraction(d[q]) * Fraction(Lj[q]) for q in range(2))
    bal, _, _, _, _ = sliced_product(Li, Lj, d)
    unb, _, _, _, _ = sliced_product(Li, Lj, d, balance=False)
    assert abs(Fraction(bal) - exact) / exact < Fraction(1, 2 ** 50)
    assert abs(Fraction(unb) - exact) / exact > Fraction(1, 10 ** 12)
