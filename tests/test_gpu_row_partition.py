"""Row-partitioned LancSVD (tsvd_set_row_partition) against the one-process solve:
two processes share the GPU, each holding half of A's rows, and exchange their
Gram matrices, projections and A^T products over a gloo group (host buffers).
After the same fixed number of cycles the singular values agree to 1e-10 and the
singular subspaces (V replicated, U stacked from the processes' rows) to 1e-8; the
converged solve takes the same number of cycles.  Cases: the 512 x 256 dense matrix
of known spectrum, an 8000 x 800 one, and a 20,000 x 5,000 CSR matrix."""

import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = {
    "dense512": dict(kind="dense", m=512, n=256, seed=0, k=10, b=16, r=4),
    "dense8000": dict(kind="dense", m=8000, n=800, seed=5, k=20, b=32, r=4),
    "csr20k": dict(kind="csr", m=20_000, n=5_000, d=10, seed=4, k=16, b=16, r=8),
}


def _matrix(cfg):
    import workloads
    if cfg["kind"] == "dense":
        return workloads.dense_known_spectrum(cfg["m"], cfg["n"], seed=cfg["seed"])[0]
    return workloads.csr_uniform(cfg["m"], cfg["n"], cfg["d"], seed=cfg["seed"])


def _on_gpu(tsvd, torch, A):
    if isinstance(A, np.ndarray):
        return torch.from_numpy(np.ascontiguousarray(A)).cuda()
    return tsvd.CsrMatrix.from_scipy(A)


def _solve_kw(cfg, converge):
    return dict(seed=7, tol=1e-8 if converge else 0.0, max_restarts=30 if converge else 1)


def _rank(rank, world, port, name, converge, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    import paper_2403_06218_gb300 as tsvd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        cfg = CASES[name]
        A = _matrix(cfg)
        lo, hi = tsvd.row_block(cfg["m"], world, rank)
        part = tsvd.RowPartition(lo, cfg["m"], tsvd.torch_allreduce())
        res = tsvd.blanczos(_on_gpu(tsvd, torch, A[lo:hi]), cfg["k"], cfg["b"], cfg["r"], partition=part,
                            **_solve_kw(cfg, converge))
        np.savez(os.path.join(out, f"r{rank}.npz"), s=res.sigma.cpu().numpy(), U=res.U.cpu().numpy(),
                 V=res.V.cpu().numpy(), cycles=res.info["iterations"], resid=res.info["resid_max"])
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sin(X, Y):
    """Largest sine of the principal angles between span(X) and span(Y) (orthonormal)."""
    return float(np.linalg.norm(X - Y @ (Y.T @ X), 2))


@pytest.mark.parametrize("name,converge", [("dense512", False), ("dense8000", False), ("csr20k", False),
                                           ("dense8000", True)])
def test_partitioned_lancsvd_matches_one_process(tsvd, tmp_path, name, converge):
    import torch
    import torch.multiprocessing as mp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = CASES[name]
    mp.spawn(_rank, args=(2, _free_port(), name, converge, str(tmp_path)), nprocs=2, join=True)
    parts = [np.load(tmp_path / f"r{r}.npz") for r in range(2)]
    ref = tsvd.blanczos(_on_gpu(tsvd, torch, _matrix(cfg)), cfg["k"], cfg["b"], cfg["r"], **_solve_kw(cfg, converge))
    s0, U0, V0 = ref.sigma.cpu().numpy(), ref.U.cpu().numpy(), ref.V.cpu().numpy()
    # replicated outputs are identical on both processes
    assert np.array_equal(parts[0]["s"], parts[1]["s"]) and np.array_equal(parts[0]["V"], parts[1]["V"])
    s, V = parts[0]["s"], parts[0]["V"]
    U = np.vstack([p["U"] for p in parts])
    ds = float(np.max(np.abs(s - s0) / s0))
    su, sv = _sin(U, U0), _sin(V, V0)
    print(f"{name} converge={converge}: sigma {ds:.1e}, sin U {su:.1e}, sin V {sv:.1e}, cycles "
          f"{int(parts[0]['cycles'])} vs {ref.info['iterations']}")
    assert ds <= 1e-10 and su <= 1e-8 and sv <= 1e-8
    if converge:
        assert int(parts[0]["cycles"]) == ref.info["iterations"]
        assert float(parts[0]["resid"]) <= 1e-8
