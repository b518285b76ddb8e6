"""The multi-process plumbing of bench.py on CPU (gloo, world size 2).

The solve path does not shard (each GPU solves its own problem: replicas),
so the only cross-rank steps are the barriers around the timed region, the
maximum of the per-rank times and rank 0 alone printing (and alone running
the reference arm).  These run here with the gloo backend on 127.0.0.1."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _child(rank, world, port, out_dir):
    import argparse
    import torch.distributed as dist
    from paper_1911_04576_gb300 import workloads as W
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_init()
    dist.barrier()
    # per-rank times 3.0 and 5.0 ms: the job's time is the slower rank's
    ms = bench.max_over_ranks(dist, 3.0 + 2.0 * rank, "cpu")
    dist.barrier()
    ran = None
    if rank == 1:
        # the reference arm runs on rank 0 only; other ranks leave at once
        args = argparse.Namespace(steps=1, warmup=0)
        ran = bench.reference_arm(args, W, W.WORKLOADS["lattice3x3_k324"])
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%d %d %d %r %r\n" % (ws, r, local, ms, ran))


def test_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_child, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        ws, r, local, ms, ran = open(tmp_path / ("rank%d.txt" % rank)).read().split()
        assert (int(ws), int(r), int(local)) == (2, rank, rank)
        assert float(ms) == 5.0
        assert ran == "None"


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(None, 7.5, "cpu") == 7.5
    assert bench.dist_init()[0] == int(os.environ.get("WORLD_SIZE", "1"))
