"""Why the mixed form's thick restart keeps FP64 master copies of the kept Ritz
vectors: a numpy emulation of that form on CPU.

The emulation stores every tall block (the bases P, Pbar and the kept vectors) in
FP32, rounds every product with A and every projection update to FP32, and keeps
the small algebra (the QR factors of each block, B and its SVD) and the final
two-sided Rayleigh-Ritz step in FP64, as the library's mixed form does.  The
restart keeps s Ritz pairs (B starts with diag(Sigma_s) and the coupling block of
the residual block).

If the kept vectors are carried in FP32 from cycle to cycle, their rounding is not
represented in B: the Lanczos estimate keeps falling while the FP64 residual of
the returned triplets stalls.  Forming the kept vectors in FP64 (from the FP32
columns and the previous FP64 masters) lowers that floor below the tolerance.
"""

import numpy as np

import workloads


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _orth(Y, P):
    """Two projection passes against P with FP32-rounded updates, then an FP64 QR
    of the result stored in FP32 (the CGS-CQR2 step of the mixed form)."""
    for _ in range(2):
        if P.shape[1]:
            Y = _f32(Y - _f32(P @ (P.T @ Y)))
    Q, R = np.linalg.qr(Y)
    return _f32(Q), R


def _mixed_thick_lanczos(A, k, b, r, keep, tol, cycles, masters):
    """Residual history of the emulated mixed-form LancSVD with thick restart."""
    m, n = A.shape
    A32 = A.astype(np.float32)
    mul = lambda X: _f32(A32 @ X.astype(np.float32))        # noqa: E731
    tmul = lambda X: _f32(A32.T @ X.astype(np.float32))     # noqa: E731
    rb = r * b
    Q1 = _f32(np.linalg.qr(np.random.default_rng(0).standard_normal((m, b)))[0])
    s0, Pk, Pbk, Sk, Qlast = 0, None, None, None, None
    hist = []
    for _ in range(cycles):
        nblk = r if s0 == 0 else (rb - s0) // b
        d = s0 + nblk * b
        P, Pb, B = np.zeros((n, d)), np.zeros((m, d)), np.zeros((d, d))
        if s0 == 0:
            Pb[:, :b] = Q1
        else:
            P[:, :s0], Pb[:, :s0] = _f32(Pk), _f32(Pbk)     # the bases hold FP32 copies
            B[:s0, :s0] = np.diag(Sk)
            Pb[:, s0:s0 + b] = Qlast
        for i in range(nblk):
            c0, c1 = s0 + i * b, s0 + (i + 1) * b
            Y = tmul(Pb[:, c0:c1])
            H = P[:, :c0].T @ Y
            Qi, T = _orth(Y, P[:, :c0])
            if i == 0 and s0:
                B[c0:c1, :s0] = H.T                         # coupling block
            P[:, c0:c1], B[c0:c1, c0:c1] = Qi, T.T
            Qn, Ri = _orth(mul(Qi), Pb[:, :c1])
            if i + 1 < nblk:
                Pb[:, c1:c1 + b], B[c1:c1 + b, c0:c1] = Qn, Ri
            else:
                Rr, Qlast = Ri, Qn
        Ub, s, Vbt = np.linalg.svd(B)
        Vb = Vbt.T
        rho = np.max(np.linalg.norm(Rr @ Vb[d - b:, :k], axis=0)) / s[0]
        Pm, Pbm = P.copy(), Pb.copy()
        if masters and s0:
            Pm[:, :s0], Pbm[:, :s0] = Pk, Pbk               # FP64 masters of the kept part
        U = np.linalg.qr(Pbm @ Ub[:, :k])[0]
        V = np.linalg.qr(Pm @ Vb[:, :k])[0]
        u, sg, vt = np.linalg.svd(U.T @ (A @ V))            # FP64 Rayleigh-Ritz
        U, V = U @ u, V @ vt.T
        res = max(np.linalg.norm(A @ V - U * sg, axis=0).max(),
                  np.linalg.norm(A.T @ U - V * sg, axis=0).max()) / sg[0]
        hist.append((rho, res))
        if rho <= tol and res <= tol:
            break
        if masters:
            Pk, Pbk = Pm @ Vb[:, :keep], Pbm @ Ub[:, :keep]
        else:
            Pk, Pbk = _f32(P @ Vb[:, :keep]), _f32(Pb @ Ub[:, :keep])
        Sk, s0 = s[:keep], keep
    return hist


def test_fp64_masters_of_the_kept_vectors_lower_the_residual_floor():
    A = workloads.csr_uniform(20_000, 20_000, 10, seed=1)
    tol = 1e-7
    plain = _mixed_thick_lanczos(A, 16, 16, 8, 32, tol, 12, masters=False)
    kept64 = _mixed_thick_lanczos(A, 16, 16, 8, 32, tol, 12, masters=True)
    # FP32 kept vectors: the estimate falls far below tol, the true residual does not
    assert len(plain) == 12
    assert min(rho for rho, _ in plain) < 0.1 * tol
    assert min(res for _, res in plain) > tol
    # FP64 masters: converged within the same budget, the residual well below the stall
    rho, res = kept64[-1]
    assert rho <= tol and res <= tol
    assert res < 0.6 * min(r for _, r in plain)
