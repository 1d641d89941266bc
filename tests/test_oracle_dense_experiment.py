"""The paper's dense experiment (Sec. 4.2) in miniature, on the oracle: with the
spectrum falling from 10 to 1e-14 over the first n/2 values, LancSVD with b = 16
and a 64-dimensional Krylov space (4 blocks) after p restart cycles is at least
as accurate, for the 1st and 10th triplet, as RandSVD with block width 16 after
6p iterations (the paper's "about 6 times" claim; its residual R_j =
||A v_j - s_j u_j|| / s_j, reading G1)."""

import numpy as np

import oracle
import workloads


def test_lancsvd_matches_randsvd_with_six_times_the_iterations():
    m, n = 8000, 800
    A, _, _, _ = workloads.dense_householder_spectrum(m, n, seed=6, sigma=workloads.spectrum_paper_dense(n))

    def R(s, U, V):
        return np.linalg.norm(A @ V - U * s, axis=0) / s

    for p in (1, 2):
        s, U, V, _ = oracle.blanczos(A, 10, 16, 4, seed=6, tol=0.0, max_restarts=p - 1)
        rl = R(s, U, V)
        s, U, V, _ = oracle.rsvd(A, 10, 6, 6 * p - 1, seed=6)
        rr = R(s, U, V)
        assert rl[0] <= rr[0] and rl[9] <= rr[9], (p, rl[[0, 9]], rr[[0, 9]])
