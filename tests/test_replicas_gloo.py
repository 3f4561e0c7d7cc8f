"""The N > 1 path of bench.py (replicas only: the path does not shard, so ranks exchange
nothing but timing scalars) with world_size 2 on the CPU over gloo: barrier, max over
ranks of the time, sum over ranks of the units, and rank-0-only reporting."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    import bench
    r, w, lr = bench.dist_init(backend="gloo")
    assert (r, w, lr) == (rank, ws, rank)
    # rank r "took" 10 + r ms and processed 100 units
    summ = bench.replica_summary(10.0 + r, 100.0, w)
    out[rank] = (summ["ms"], summ["units"], summ["ranks"])
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
    assert out[0] == (11.0, 200.0, 2) and out[1] == (11.0, 200.0, 2)


def test_single_process_is_identity():
    import bench
    assert bench.replica_summary(5.0, 7.0, 1) == {"ms": 5.0, "units": 7.0, "ranks": 1}
