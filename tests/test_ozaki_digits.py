"""The arithmetic of the tensor-core FP64 products (MSP_F64_TC), restated in
exact integer arithmetic on the CPU, so that the bounds the kernel relies on
are checked independently of the GPU:
  * every operand row, scaled to its largest entry, becomes an integer
    |m| < 2^54 with eight balanced base-128 digits, |d_0| <= 33 and
    |d_s| <= 64, each exact in BF16 (an integer of at most 8 bits);
  * a K = 64 sum of digit products and a group of at most eight of them
    (s + t = g) stay below 2^21, so the FP32 accumulators of the tensor
    cores hold them exactly (and the 1.5 * 2^23 offset reads them back);
  * the groups g = 0..7, combined with weights 2^(46 - 7g) in 64-bit
    integers (the last rounded), give the product within 2^-48 K max|a_r|
    max|b_c| of the exact one (the worst case of the left-out digit pairs
    s + t > 7 is about 2^-49.2 of it; an FP64 dot product's own worst case is
    K 2^-53 sum|a||b|, up to 2^-47 of it), also for rows whose entries span
    many orders of magnitude.
The digits are built here the way the kernel builds them (three pieces of
14, 21 and 21 bits, peeled from the least significant digit up); the exact
product is a sum of Python integers.
"""
import math

import numpy as np
import pytest

K = 64


def row_exponent(row):
    """Largest biased exponent of the row (0 for a zero row)."""
    e = 0
    for x in row:
        if x != 0.0:
            e = max(e, math.frexp(abs(x))[1] + 1022)
    return e


def fixed_abs(x, emax):
    """round(|x| 2^(54 - (emax - 1022))) with ties away from zero in the
    last bit, as the kernel's shift-and-round of the 53-bit significand."""
    if x == 0.0:
        return 0
    m, e = math.frexp(abs(x))          # |x| = m 2^e, 0.5 <= m < 1
    mant = int(m * (1 << 53))          # 53-bit significand
    biased = e + 1022
    sh = biased - emax + 1
    if sh >= 0:
        return mant << sh
    if sh > -56:
        return (mant + (1 << (-sh - 1))) >> (-sh)
    return 0


def peel(v):
    """One balanced base-128 digit: q = rint(v / 128) (ties to even), d = v - 128 q."""
    q = round(v / 128)                 # Python rounds half to even, as the FP32 offset does
    return v - 128 * q, q


def digits(m):
    """Eight balanced base-128 digits of 0 <= m < 2^54, most significant first,
    from the pieces bits 0..13, 14..34, 35..55."""
    d = [0] * 8
    v = m & 0x3FFF
    d[7], v = peel(v)
    d[6], v = peel(v)
    v += (m >> 14) & 0x1FFFFF
    d[5], v = peel(v)
    d[4], v = peel(v)
    d[3], v = peel(v)
    v += m >> 35
    d[2], v = peel(v)
    d[1], v = peel(v)
    d[0] = v
    return d


def split(M):
    """Signed digits [rows][K][8] and row exponents of an FP64 matrix."""
    rows, cols = M.shape
    E = [row_exponent(M[r]) for r in range(rows)]
    D = np.zeros((rows, cols, 8), dtype=np.int64)
    for r in range(rows):
        for k in range(cols):
            m = fixed_abs(M[r, k], E[r])
            assert m < (1 << 54)
            dd = digits(m)
            assert sum(dd[s] * 128 ** (7 - s) for s in range(8)) == m
            sg = -1 if M[r, k] < 0 else 1
            D[r, k] = [sg * x for x in dd]
    return D, E


def product(A, B):
    """The kernel's product A B^T: group sums, their integer combination, FP64."""
    DA, EA = split(A)
    DB, EB = split(B)
    assert np.abs(DA[:, :, 0]).max() <= 33 and np.abs(DB[:, :, 0]).max() <= 33
    assert np.abs(DA[:, :, 1:]).max() <= 64 and np.abs(DB[:, :, 1:]).max() <= 64
    P = [sum(DA[:, :, s] @ DB[:, :, g - s].T for s in range(g + 1)) for g in range(8)]  # exact int64
    for g in range(8):
        assert np.abs(P[g]).max() < (1 << 21)  # exact in FP32, readable through the 1.5 * 2^23 offset
    out = np.zeros((A.shape[0], B.shape[0]))
    for r in range(A.shape[0]):
        for c in range(B.shape[0]):
            V = 0
            for g in range(0, 8, 2):  # groups g and g + 1 joined in 32 bits, weight 2^(39 - 7g)
                q = int(P[g][r, c]) * 128 + int(P[g + 1][r, c])
                assert abs(q) < (1 << 29)
                V += (q << (39 - 7 * g)) if g < 6 else (q + 4) >> 3
            assert abs(V) < (1 << 63)
            out[r, c] = math.ldexp(float(V), EA[r] + EB[c] - 2100)  # one rounding (to nearest even)
    return out, EA, EB


def exact(A, B):
    """A B^T exactly (FP64 entries as exact rationals), rounded to FP64 once."""
    from fractions import Fraction
    out = np.zeros((A.shape[0], B.shape[0]))
    for r in range(A.shape[0]):
        fa = [Fraction(x) for x in A[r]]
        for c in range(B.shape[0]):
            out[r, c] = float(sum(a * Fraction(b) for a, b in zip(fa, B[c])))
    return out


@pytest.mark.parametrize("spread", [0, 6, 30])
def test_digit_products_reach_fp64_accuracy(spread):
    """Rows whose entries span 10^0, 10^6 and 10^30: the product entry is
    within 2^-48 K max|a_r| max|b_c| of the exact sum, the worst case of the
    scheme; random digits land far inside it."""
    rng = np.random.default_rng(11 + spread)
    A = rng.normal(size=(6, K)) * 10.0 ** rng.uniform(-spread, 0, size=(6, K))
    B = rng.normal(size=(5, K)) * 10.0 ** rng.uniform(-spread, 0, size=(5, K))
    A[2, :] = 0.0        # a zero row
    A[3, 10:] = 0.0      # a short row
    got, _, _ = product(A, B)
    ref = exact(A, B)
    bound = 2.0 ** -48 * K * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]
    assert np.all(np.abs(got - ref) <= bound)
    assert np.all(np.abs(got - ref) <= bound / 64)  # typical: well inside the worst case
    assert not got[2].any()
    # the FP64 dot product's own bound (K 2^-53 sum |a||b|) is of the same class
    fp64 = A @ B.T
    assert np.all(np.abs(fp64 - ref) <= K * 2.0 ** -53 * (np.abs(A) @ np.abs(B).T) + 1e-300)


def test_digits_of_extreme_values():
    """The largest representable integer and entries at the row maximum and
    far below it: digit bounds, exact reconstruction, BF16 exactness."""
    for m in [0, 1, 63, 64, 65, 127, 128, (1 << 54) - 1, (1 << 53) + 12345, 0x2AAAAAAAAAAAAA]:
        d = digits(m)
        assert sum(d[s] * 128 ** (7 - s) for s in range(8)) == m
        assert abs(d[0]) <= 33 and all(abs(x) <= 64 for x in d[1:])
        for x in d:  # an integer of at most 8 bits is exact in BF16 (8-bit significand)
            assert abs(x) < 256
    row = np.array([1.0, -1.0 + 2.0 ** -52, 2.0 ** -40, 2.0 ** -60, -0.0])
    e = row_exponent(row)
    assert fixed_abs(row[0], e) == 1 << 53   # |x| < 2^1 = 2^(e - 1022): m = |x| 2^53
    assert fixed_abs(row[1], e) == (1 << 53) - 2
    assert fixed_abs(row[2], e) == 1 << 13
    assert fixed_abs(row[3], e) == 0         # below half a unit of 2^-53: rounded to zero
    assert fixed_abs(row[4], e) == 0
