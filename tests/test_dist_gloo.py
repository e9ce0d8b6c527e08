"""Host logic of the N-rank benchmark (barrier, max of times and sum of
elements over ranks) on two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r = bench.dist_init("gloo")
    bench.barrier()
    mx = bench.max_over_ranks(10.0 * (rank + 1), "cpu")
    sm = bench.sum_over_ranks(rank + 1.5, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{w} {r} {mx} {sm}")
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_times_and_elements(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        w, r, mx, sm = open(tmp_path / f"r{rank}.txt").read().split()
        assert int(w) == 2 and int(r) == rank
        assert float(mx) == 20.0 and float(sm) == 4.0


def test_single_process_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5 and bench.sum_over_ranks(2.0) == 2.0
