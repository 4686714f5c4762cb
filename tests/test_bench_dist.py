"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1 agree on the
maximum of their per-rank times (the whole-job time), pass the barrier, and
only rank 0 would print.  No GPU is involved."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    r, w = bench.dist_setup()
    assert (r, w) == (rank, ws)
    bench.barrier(w)
    t = bench.reduce_max(1.5 + rank, w)
    out[rank] = t
    import torch.distributed as dist
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_max_timing():
    ws = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.25, 1) == 3.25


def test_graph_launch_count():
    """sim_step(n) runs eight-step graphs while eight steps remain, then
    four-step ones, then single steps; the bench counts one hi/lo split per
    graph launch on top of the per-step kernels."""
    sys.path.insert(0, ROOT)
    import bench
    expect = {1: 1, 3: 3, 4: 1, 7: 4, 8: 1, 12: 2, 16: 2, 20: 3, 23: 6}
    assert {n: bench.graph_launches(n) for n in expect} == expect
