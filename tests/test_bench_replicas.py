"""The N > 1 path of bench.py on CPU: world_size-2 gloo process group.  Each rank
solves its own problem (seed + rank); the only collective is the max-over-ranks
time reduction; ranks other than 0 print nothing (the reference arm exits 0 there)."""

import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.replica_env()
    cfg = bench.WORKLOADS["dense512-lanczos"]
    A = bench._make_matrix(dict(cfg, m=64, n=32), r)
    t = bench.max_over_ranks(1.5 + r, dist, "cpu")
    out[rank] = (w, r, local, bench.replica_seed(cfg, r), float(A[0, 0]), t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_slowest_time_and_solve_their_own_problem():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    (w0, r0, l0, s0, a0, t0), (w1, r1, l1, s1, a1, t1) = res[0], res[1]
    assert (w0, r0, l0) == (2, 0, 0) and (w1, r1, l1) == (2, 1, 1)
    assert s1 == s0 + 1 and a0 != a1          # independent replicas
    assert t0 == t1 == 2.5                    # max over ranks


def test_reference_arm_exits_quietly_on_other_ranks(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=0, workload="sparse100k-lanczos-thick")
    assert bench.run_reference(args, bench.WORKLOADS[args.workload]) == 0
    assert capsys.readouterr().out == ""


def test_max_over_ranks_alone_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
