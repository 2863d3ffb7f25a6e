"""The multi-process path of bench.py on CPU: two gloo ranks (world size 2)
set up through bench.dist_setup, meet at its barrier and agree on the
maximum of their timings (the timing rule is max over ranks).  The GPU arm
runs the same helpers over NCCL; nothing in the method is sharded, so the
ranks are independent replicas and this is all the communication there is."""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    args = types.SimpleNamespace(impl="reference")
    w, r, local = bench.dist_setup(args)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    m = bench.max_over_ranks(w, 1.0 + 1.5 * rank, "cpu")
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{m}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max_over_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    vals = [float(open(tmp_path / f"rank{r}.txt").read()) for r in range(world)]
    assert vals == [2.5, 2.5]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1, 3.25, "cpu") == 3.25
    bench.barrier(1)
