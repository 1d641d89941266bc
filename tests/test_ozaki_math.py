"""CPU checks of the arithmetic of the FP64-accurate tensor-core product
(exponent-aligned BF16 slices: Ozaki, Ogita, Oishi, Rump 2012, in the variant
with fixed-point digits of Ootomo, Ozaki, Yokota 2024), emulated exactly in
Python integers.  These pin the design's own arithmetic, not the paper's.

Scheme (one exponent per row of A and per column of B):
  * F = round(x 2^(55 - e)) for x in a row of A (e: the smallest e with
    |x| < 2^e over the row), split into 7 balanced base-256 digits d_0..d_6
    (F = sum_p d_p 2^(8 (6 - p)), |d_p| <= 128, each exactly a BF16 value);
  * T_g = sum_k sum_{p+q=g} dA_p dB_q for g = 0..6 (the products with
    p + q > 6 are dropped); over 128 consecutive k every T_g is below 2^24 in
    magnitude, so FP32 accumulation of it is exact;
  * per 128 k: hi += sum_{g<=4} T_g 2^(8 (4 - g)) (64-bit), lo += T_5 +
    round(T_6 / 256) (32-bit); C = 2^(ea + eb - 46) (hi + lo 2^-8).
"""

import math
from fractions import Fraction

import numpy as np

DIGITS = 7


def exponent_of(x: float) -> int:
    """Smallest e with |x| < 2^e (None for x == 0)."""
    if x == 0.0:
        return None
    m, e = math.frexp(abs(x))  # |x| = m 2^e, 0.5 <= m < 1
    return e


def row_exponent(v) -> int:
    es = [exponent_of(float(x)) for x in v if x != 0.0]
    return max(es) if es else 0


def fixed_point(x: float, e: int) -> int:
    """round(x 2^(55 - e)), ties away from zero on the magnitude."""
    f = Fraction(abs(x)) * Fraction(2) ** (55 - e)
    n = math.floor(f + Fraction(1, 2))
    return n if x >= 0 else -n


def digits(F: int):
    d = [0] * DIGITS
    r = F
    for p in range(DIGITS - 1, 0, -1):
        lo = ((r + 128) & 255) - 128
        d[p] = lo
        r = (r - lo) >> 8
    d[0] = r
    return d


def oz_product(A, B, chunk=128):
    """Emulated product: exact digit arithmetic as the kernel does it (including the
    rounding of T_6 to 2^-40 per chunk), and the largest |T_g| seen."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[1]
    ea = [row_exponent(A[i]) for i in range(M)]
    eb = [row_exponent(B[:, j]) for j in range(N)]
    DA = [[digits(fixed_point(A[i, k], ea[i])) for k in range(K)] for i in range(M)]
    DB = [[digits(fixed_point(B[k, j], eb[j])) for k in range(K)] for j in range(N)]
    C = np.zeros((M, N))
    worst = 0
    for i in range(M):
        for j in range(N):
            hi = lo = 0
            for k0 in range(0, K, chunk):
                T = [0] * DIGITS
                for k in range(k0, min(K, k0 + chunk)):
                    a, b = DA[i][k], DB[j][k]
                    for g in range(DIGITS):
                        T[g] += sum(a[p] * b[g - p] for p in range(g + 1))
                worst = max(worst, max(abs(t) for t in T))
                hi += sum(T[g] << (8 * (4 - g)) for g in range(5))
                lo += T[5] + ((T[6] + 128) >> 8)
            assert abs(lo) < 2 ** 31 and abs(hi) < 2 ** 63
            C[i, j] = float((Fraction(hi) + Fraction(lo, 256)) * Fraction(2) ** (ea[i] + eb[j] - 46))
    return C, worst


def exact_product(A, B):
    M, K = A.shape
    N = B.shape[1]
    C = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            C[i, j] = float(sum(Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K)))
    return C


def test_digits_reconstruct_and_fit_bf16():
    rng = np.random.default_rng(0)
    for x in np.concatenate([rng.standard_normal(200), [1.0, -1.0, 0.75, 2.0 ** -30, -(1 - 2.0 ** -53)]]):
        e = exponent_of(x)
        F = fixed_point(x, e)
        d = digits(F)
        assert sum(dp << (8 * (6 - p)) for p, dp in enumerate(d)) == F
        assert all(abs(dp) <= 128 for dp in d)
        assert abs(d[0]) >= 32  # the leading digit carries the top bits of a row maximum
        # |x - F 2^(e-55)| <= 2^(e-56): the representation is exact to 56 bits of the row scale
        assert abs(Fraction(x) - Fraction(F) * Fraction(2) ** (e - 55)) <= Fraction(2) ** (e - 56)


def test_exact_groups_stay_below_fp32_integer_range():
    rng = np.random.default_rng(1)
    # worst case for the digit sums: every entry at the row maximum with the same sign
    A = np.full((2, 128), 1.0 - 2.0 ** -9)
    B = np.full((128, 2), -(1.0 - 2.0 ** -9))
    _, worst = oz_product(A, B)
    assert worst <= 2 ** 24
    A = rng.standard_normal((3, 256))
    B = rng.standard_normal((256, 3))
    _, worst = oz_product(A, B)
    assert worst <= 2 ** 24
    # the bound itself: |d_p d_q| <= 2^14, at most 7 pairs per group, 128 terms
    assert 7 * 128 * 2 ** 14 <= 2 ** 24


def test_product_error_within_fp64_bound():
    rng = np.random.default_rng(2)
    for (M, K, N, scale) in ((4, 300, 3, 1.0), (3, 513, 2, 1e-200), (2, 64, 5, 1e150)):
        A = rng.standard_normal((M, K)) * scale
        B = rng.standard_normal((K, N))
        A[0, :5] = 0.0
        C, _ = oz_product(A, B)
        ref = exact_product(A, B)
        # the stated bound: representation 2^-56 of the row (column) scale, dropped
        # digit products 6.2 K 2^(ea + eb - 56), one final rounding
        ea = np.ldexp(1.0, np.array([[row_exponent(A[i])] for i in range(M)]))
        eb = np.ldexp(1.0, np.array([[row_exponent(B[:, j]) for j in range(N)]]))
        bound = (2.0 ** -56 * (ea * np.abs(B).sum(axis=0, keepdims=True) + np.abs(A).sum(axis=1, keepdims=True) * eb)
                 + 6.2 * K * ea * eb * 2.0 ** -56 + 2.0 ** -53 * np.abs(ref))
        assert np.all(np.abs(C - ref) <= bound)
        assert np.all(np.abs(C - ref) <= 2 * K * np.finfo(float).eps * (np.abs(A) @ np.abs(B)) + 1e-300)


def test_dropping_the_tail_pairs_or_a_digit_is_detected():
    """Six digits (or a product formed without the p + q = 6 pairs) misses the FP64
    bound on rows with a wide dynamic range: every digit is needed."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 200))
    B = rng.standard_normal((200, 3))
    ea = [row_exponent(A[i]) for i in range(3)]
    eb = [row_exponent(B[:, j]) for j in range(3)]
    ref = exact_product(A, B)
    for drop in (6, 5):
        C = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                total = 0
                for k in range(200):
                    a = digits(fixed_point(A[i, k], ea[i]))
                    b = digits(fixed_point(B[k, j], eb[j]))
                    for g in range(drop):
                        total += sum(a[p] * b[g - p] for p in range(g + 1)) << (8 * (12 - g))
                C[i, j] = float(Fraction(total) * Fraction(2) ** (ea[i] + eb[j] - 110))
        # a product formed without them is off by more than the stated bound allows
        Ea = np.ldexp(1.0, np.array(ea))[:, None]
        Eb = np.ldexp(1.0, np.array(eb))[None, :]
        bound = (2.0 ** -56 * (Ea * np.abs(B).sum(axis=0, keepdims=True) + np.abs(A).sum(axis=1, keepdims=True) * Eb)
                 + 6.2 * 200 * Ea * Eb * 2.0 ** -56 + 2.0 ** -53 * np.abs(ref))
        assert np.any(np.abs(C - ref) > bound)
