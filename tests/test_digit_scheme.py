"""The integer-digit scheme of the tensor-core operator passes (CPU).

The tensor-core passes (kf_opts.tc_operator) cut kernel values v in [0, 1]
into 7 unsigned 7-bit digits and every column of x, scaled by a power of two
tau >= max |x|, into 7 balanced digits; digit products summed over a
128-row window in the tensor core's FP32 accumulator must be exact, and the
8 groups p + q <= 7 must carry the product to about 2^-49 tau per entry.
These checks restate the scheme in integer arithmetic (Ozaki, Ogita, Oishi
and Rump, Numer. Algorithms 59, 2012) and pin its bounds: the window
sums stay below 2^24 for the largest digits the cuts can produce, the
truncated sum agrees with exact rational arithmetic to the stated error, and
the read-out's two int64 sums convert to FP64 exactly and carry the groups'
weights.
"""
import math
from fractions import Fraction

import numpy as np

ND, WIN = 7, 128


def v_digits(v):
    """7 unsigned digits of round(v 2^49) for v in [0, 1]: a_0 <= 128, a_p < 128."""
    V = int(round(Fraction(v) * 2 ** 49))
    V = max(0, min(V, 2 ** 49))
    return [V >> 42] + [(V >> (7 * (6 - p))) & 127 for p in range(1, ND)]


def x_digits(x, e):
    """7 balanced digits of round(x 2^(49 - e)) for |x| < 2^e: d_0 in [-128, 128], others in [-64, 63]."""
    X = int(round(Fraction(x) * Fraction(2) ** (49 - e)))
    d = [0] * ND
    for p in range(ND - 1, 0, -1):
        d[p] = ((X + 64) & 127) - 64
        X = (X - d[p]) >> 7
    d[0] = X
    return d


def test_digit_ranges_and_reconstruction():
    rng = np.random.default_rng(11)
    for v in list(rng.random(200)) + [0.0, 1.0, 2.0 ** -30, 1 - 2.0 ** -53]:
        a = v_digits(v)
        assert 0 <= a[0] <= 128 and all(0 <= t < 128 for t in a[1:])
        rec = sum(Fraction(t, 2 ** (7 * (p + 1))) for p, t in enumerate(a))
        assert abs(rec - Fraction(v)) <= Fraction(1, 2 ** 50)
    for x in list(rng.standard_normal(200)) + [-1.0, 1.0 - 2.0 ** -20, -(1.0 - 2.0 ** -53)]:
        e = int(np.frexp(abs(x))[1])  # tau = 2^e > |x|, as the kernels choose it from the column maximum
        d = x_digits(x, e)
        assert -128 <= d[0] <= 128 and all(-64 <= t <= 63 for t in d[1:])
        rec = Fraction(2) ** e * sum(Fraction(t, 2 ** (7 * (q + 1))) for q, t in enumerate(d))
        assert abs(rec - Fraction(x)) <= Fraction(2) ** e / 2 ** 50


def test_window_group_sums_fit_fp32_exactly():
    """The largest digit magnitudes (a_0 = 128, a_p = 127; d_0 = 128, d_q = 64)
    over a full 128-row window: every group sum stays below 2^24."""
    amax = [128] + [127] * (ND - 1)
    dmax = [128] + [64] * (ND - 1)
    for g in range(8):
        bound = WIN * sum(amax[p] * dmax[g - p] for p in range(ND) if 0 <= g - p < ND)
        assert bound < 2 ** 24, (g, bound)


def test_truncated_sum_matches_exact_arithmetic():
    """sum_i v_i x_i from the digit pairs p + q <= 7 of 300 rows (three windows)
    against exact rational arithmetic: within 2^-48 tau sum |v| (the dropped
    pairs and the two roundings)."""
    rng = np.random.default_rng(12)
    n = 300
    v = np.exp(-rng.random(n) * 20)
    x = rng.standard_normal(n) * np.exp(rng.uniform(-4, 4, n))
    e = int(np.frexp(np.abs(x).max())[1])  # 2^e > max |x|
    A = [v_digits(t) for t in v]
    Dg = [x_digits(t, e) for t in x]
    total = Fraction(0)
    for w0 in range(0, n, WIN):  # one window at a time, as the tensor core sums them
        for g in range(8):
            acc = sum(A[i][p] * Dg[i][g - p] for i in range(w0, min(n, w0 + WIN))
                      for p in range(ND) if 0 <= g - p < ND)
            assert abs(acc) < 2 ** 24
            total += Fraction(acc, 2 ** (7 * (g + 2)))
    approx = total * Fraction(2) ** e
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(v, x))
    bound = Fraction(2) ** e / 2 ** 48 * sum(Fraction(float(a)) for a in v)
    assert abs(approx - exact) <= bound


def _readout(A, Dg, e, rows):
    """The kernels' read-out: per 128-row window the 8 exact group sums; over
    the windows two int64 sums, hi = sum_{g<=3} acc_g 2^(7(3-g)) and
    lo = sum_{g>=4} acc_g 2^(7(7-g)); the value 2^(e-35) hi + 2^(e-63) lo in
    FP64 (two exact conversions, two exact scalings, one rounded addition)."""
    hi = lo = 0
    weighted = Fraction(0)  # the same group sums at their weights 2^(-7(g+2)), exactly
    for w0 in range(0, rows, WIN):
        for g in range(8):
            acc = sum(A[i][p] * Dg[i][g - p] for i in range(w0, min(rows, w0 + WIN))
                      for p in range(ND) if 0 <= g - p < ND)
            weighted += Fraction(acc, 2 ** (7 * (g + 2)))
            if g <= 3:
                hi += acc << (7 * (3 - g))
            else:
                lo += acc << (7 * (7 - g))
    return hi, lo, math.ldexp(float(hi), e - 35) + math.ldexp(float(lo), e - 63), weighted * Fraction(2) ** e


def test_readout_int64_sums_convert_exactly():
    """Eight windows (a 1024-row chunk or leaf, the most one read-out sums) of
    the largest digits: |hi| and |lo| stay below 2^53, so both convert to
    FP64 without rounding and the read-out rounds once, in its addition."""
    amax = [128] + [127] * (ND - 1)
    dmax = [128] + [64] * (ND - 1)
    A, Dg = [amax] * (8 * WIN), [dmax] * (8 * WIN)
    hi, lo, _, _ = _readout(A, Dg, 0, 8 * WIN)
    assert 0 < hi < 2 ** 53 and 0 < lo < 2 ** 53


def test_readout_matches_exact_group_sum():
    """The read-out's shifts (7(3-g) with 2^-35, 7(7-g) with 2^-63) against
    the group weights 2^(-7(g+2)) summed exactly: equal up to the one
    rounding of the final addition."""
    rng = np.random.default_rng(13)
    n = 1000  # eight windows, the last one ragged
    v = rng.random(n)
    x = rng.standard_normal(n) * 3.0
    e = int(np.frexp(np.abs(x).max())[1])
    A = [v_digits(t) for t in v]
    Dg = [x_digits(t, e) for t in x]
    _, _, val, exact = _readout(A, Dg, e, n)
    assert abs(Fraction(val) - exact) <= abs(exact) * Fraction(1, 2 ** 53)
