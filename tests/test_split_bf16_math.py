"""The arithmetic behind the mixed form's tensor-core products for dense A, checked
on CPU with exact BF16 rounding in numpy (no GPU code involved).

A value is split greedily into three BF16 pieces, each the round-to-nearest BF16
of what the previous pieces left (8 significant bits each), so the pieces
reconstruct it to 24 bits.  The product keeps the six cross terms A_i X_j with
i + j <= 2; every dropped term is O(2^-24) of |A||X|.  The bound stated for the
product is |Y - A X| <= c u |A| |X| with u = 2^-24, which this file pins at c = 5:
the reconstruction errors of A and X (<= u each) plus the three dropped terms
(<= 2u + u^2).  Fewer terms miss FP32 accuracy (three terms leave ~2^-16), and a
single BF16 product stays near 2^-9.
"""

import numpy as np
import pytest

U24 = 2.0 ** -24


def round_bf16(x):
    """Round-to-nearest-even to 8 significant bits (BF16's precision; the values here
    stay inside BF16's exponent range)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def split3(x):
    p0 = round_bf16(x)
    r1 = x - p0                              # exact in FP64
    p1 = round_bf16(r1)
    r2 = r1 - p1
    p2 = round_bf16(r2)
    return p0, p1, p2


def test_round_bf16_is_round_to_nearest_even_at_eight_bits():
    assert round_bf16(1.0 + 2.0 ** -8) == 1.0                  # tie, even mantissa stays
    assert round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie, rounds to even upward
    assert round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7
    assert round_bf16(-3.0) == -3.0 and round_bf16(0.0) == 0.0
    x = np.random.default_rng(0).standard_normal(10000)
    y = round_bf16(x)
    assert np.all(np.abs(x - y) <= 2.0 ** -9 * 2.0 ** np.ceil(np.log2(np.abs(x))))   # half an ulp
    assert np.all(round_bf16(y) == y)


@pytest.mark.parametrize("scale_bits", [0, 20])
def test_three_pieces_reconstruct_to_24_bits(scale_bits):
    rng = np.random.default_rng(scale_bits)
    x = rng.standard_normal(100_000) * 2.0 ** rng.uniform(-scale_bits, scale_bits, 100_000)
    p0, p1, p2 = split3(x)
    assert np.all(np.abs(x - (p0 + p1 + p2)) <= U24 * np.abs(x))
    assert np.all(np.abs(p1) <= 2.0 ** -8 * np.abs(x)) and np.all(np.abs(p2) <= 2.0 ** -16 * np.abs(x))
    # two pieces are not enough for FP32 accuracy
    assert np.max(np.abs(x - (p0 + p1)) / np.abs(x)) > 64 * U24


def _product(Ap, Xp, terms):
    # products of BF16 values are exact in FP64; the FP64 sums add ~K 2^-53, far below u
    return sum(Ap[i] @ Xp[j] for i, j in terms)


def test_six_cross_terms_give_fp32_accuracy_and_fewer_do_not():
    rng = np.random.default_rng(7)
    m, kdim, w = 300, 2000, 24
    A = rng.standard_normal((m, kdim)) * np.exp(rng.uniform(-3, 3, (m, 1)))
    X = rng.standard_normal((kdim, w))
    Ap, Xp = split3(A), split3(X)
    exact = A @ X
    scale = np.abs(A) @ np.abs(X)
    six = [(i, j) for i in range(3) for j in range(3) if i + j <= 2]
    assert len(six) == 6
    err6 = np.abs(_product(Ap, Xp, six) - exact)
    assert np.all(err6 <= 5 * U24 * scale)
    # the three dropped terms are O(u): adding them changes the result by less than 3u |A||X|
    dropped = [(1, 2), (2, 1), (2, 2)]
    assert np.all(np.abs(_product(Ap, Xp, dropped)) <= 3 * U24 * scale)
    # normwise: six terms within u; three terms (i + j <= 1) or one BF16 product are far
    # from FP32 accuracy (random-sign errors: ~2^-16 and ~2^-9 relative)
    rel = lambda Y: np.linalg.norm(Y - exact) / np.linalg.norm(exact)   # noqa: E731
    assert rel(_product(Ap, Xp, six)) <= U24
    assert rel(_product(Ap, Xp, [(0, 0), (0, 1), (1, 0)])) > 20 * U24
    assert 1e-3 < rel(Ap[0] @ Xp[0]) < 1e-2     # BF16 alone: the ~1e-3 floor
