"""Host side of the row-partitioned LancSVD on CPU: the even row split, and the
reduction callback the library calls (a RowPartition over a world-size-2 gloo group
sums the processes' buffers in place; a failing exchange reports failure instead of
raising through the C ABI).  The GPU path itself is tested in
tests/test_gpu_row_partition.py."""

import ctypes as C
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2403_06218_gb300 import api


def test_row_block_covers_every_row_once():
    for rows, world in ((10, 3), (20_000, 2), (7, 7), (5, 8)):
        blocks = [api.row_block(rows, world, r) for r in range(world)]
        assert blocks[0][0] == 0 and blocks[-1][1] == rows
        assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
        sizes = [hi - lo for lo, hi in blocks]
        assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = api.row_block(9, world, rank)
        part = api.RowPartition(lo, 9, api.torch_allreduce())
        buf = np.arange(12, dtype=np.float64) * (rank + 1)
        ptr = buf.ctypes.data_as(C.POINTER(C.c_double))
        rc = part._cb(None, ptr, buf.size)  # the call the library makes
        bad = api.RowPartition(lo, 9, lambda arr: (_ for _ in ()).throw(RuntimeError("link down")))
        rc_bad = bad._cb(None, ptr, 3)
        np.save(os.path.join(out, f"r{rank}.npy"), np.r_[rc, rc_bad, buf, float(isinstance(bad.error, RuntimeError))])
    finally:
        dist.destroy_process_group()


def test_gloo_reduction_callback_sums_over_two_processes(tmp_path):
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    want = np.arange(12, dtype=np.float64) * 3  # ranks contribute x1 and x2
    for r in range(2):
        got = np.load(tmp_path / f"r{r}.npy")
        assert got[0] == 0 and got[1] == 1 and got[-1] == 1
        assert np.array_equal(got[2:-1], want)


def test_partition_rejects_rows_outside_the_matrix():
    with pytest.raises(ValueError):
        api.RowPartition(10, 10, lambda a: None)
