"""Tensor-core split-BF16 products (tcgen05 + TMA) of the mixed form against the
exact product.

The pieces must reconstruct A to 24 significant bits (|A - A0 - A1 - A2| <=
2^-24 |A| elementwise, plus the BF16 subnormal floor), and Y = P X must meet an
FP32-class bound |Y - A X| <= (k + 16) 2^-22 (|A| |X|) for inner dimension k:
the six kept cross terms drop only O(2^-24)-relative terms, and the FP32
accumulation in tensor memory adds at most a gamma_k-type error.  Shapes span a
ragged last row tile, a ragged last K block, several CTAs per tile (long K),
several tiles per CTA (short K), w not a multiple of 16 and w > 128 (two
column panels).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _bf16_to_f64(t):
    return t.float().double().cpu().numpy()


@pytest.mark.parametrize("m,n", [(300, 200), (64, 1000), (1000, 64)])
def test_split_reconstructs_to_24_bits(tsvd, torch_cuda, m, n):
    torch = torch_cuda
    rng = np.random.default_rng(m * n)
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-20, 20, size=(m, n)))
    At = torch.from_numpy(A).cuda()
    for trans in (False, True):
        P = tsvd.bf16x3_split(At, trans=trans)
        pcs = P.pieces()
        rec = sum(_bf16_to_f64(pcs[i]) for i in range(3))
        ref = A.T if trans else A
        assert rec.shape == ref.shape
        assert np.all(np.abs(rec - ref) <= 2.0 ** -24 * np.abs(ref) + 1e-38)
        # the leading piece is a BF16 rounding of the entry (unit roundoff 2^-8), the others
        # are each at most that of what remains
        p0, p1 = _bf16_to_f64(pcs[0]), _bf16_to_f64(pcs[1])
        assert np.all(np.abs(p0 - ref) <= 2.0 ** -8 * np.abs(ref))
        assert np.all(np.abs(p1) <= 2.0 ** -8 * np.abs(p0) * (1 + 2.0 ** -7))


@pytest.mark.parametrize("m,n,w", [(300, 200, 20), (1000, 777, 128), (4097, 1000, 64), (128, 64, 16),
                                   (100, 5000, 100), (1, 64, 1), (2000, 300, 200), (777, 129, 48)])
def test_mm_bf16x6_fp32_bound(tsvd, torch_cuda, m, n, w):
    torch = torch_cuda
    rng = np.random.default_rng(m + 7 * n + w)
    A = rng.standard_normal((m, n))
    X = rng.standard_normal((n, w)).astype(np.float32)
    At = torch.from_numpy(A).cuda()
    P = tsvd.bf16x3_split(At)
    Xd = torch.from_numpy(X).cuda()
    Y = tsvd.mm_bf16x6(P, Xd).cpu().numpy().astype(np.float64)
    X64 = X.astype(np.float64)
    ref = A @ X64
    bound = (n + 16) * 2.0 ** -22 * (np.abs(A) @ np.abs(X64))
    err = np.abs(Y - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    rel = np.max(err) / np.max(np.abs(A) @ np.abs(X64))
    print(f"bf16x6 {m}x{n}x{w}: max |err| / max(|A||X|) = {rel:.2e}")
    # deterministic: the same call gives the same bits
    Y2 = tsvd.mm_bf16x6(P, Xd).cpu().numpy().astype(np.float64)
    assert np.array_equal(Y, Y2)


def test_mm_bf16x6_transposed_pieces(tsvd, torch_cuda):
    """A^T X from the pieces of A^T (the S2/S4 product of the mixed form)."""
    torch = torch_cuda
    rng = np.random.default_rng(5)
    A = rng.standard_normal((900, 333))
    X = rng.standard_normal((900, 64)).astype(np.float32)
    P = tsvd.bf16x3_split(torch.from_numpy(A).cuda(), trans=True)
    assert (P.rows, P.cols) == (333, 900)
    Y = tsvd.mm_bf16x6(P, torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    ref = A.T @ X.astype(np.float64)
    assert np.all(np.abs(Y - ref) <= (900 + 16) * 2.0 ** -22 * (np.abs(A.T) @ np.abs(X.astype(np.float64))))
