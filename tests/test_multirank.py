"""Multi-rank path on CPU (gloo, world size 2): each rank decomposes its own
layout (host half of the library), no data exchange; timing aggregation
gives total segments and the slowest rank's time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2303_14335_gb300 import mpld, shard, synth


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L = synth.unit_disk_layout(3000, 3, seed=shard.rank_seed(2, rank), mean_deg=3.0, p_stitch=0.2)
    prob = mpld.mpld_build_matrix(L, mpld.make_params(flags=mpld.MPLD_HOST_ONLY))
    info = mpld.mpld_problem_info(prob)
    seconds = 1.0 + rank            # stand-in per-rank time
    segs, slowest = shard.aggregate(dist, L.n_seg, seconds, "cpu")
    got = [None] * world
    dist.all_gather_object(got, (L.n_seg, info.n_components, int(L.conf_u.sum())))
    dist.barrier()
    if rank == 0:
        out.put((segs, slowest, got))
    dist.destroy_process_group()


def test_two_ranks_shard_independent_layouts():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    segs, slowest, got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert slowest == 2.0
    assert segs == got[0][0] + got[1][0]
    assert got[0] != got[1]                   # different layouts per rank
    L0 = synth.unit_disk_layout(3000, 3, seed=2, mean_deg=3.0, p_stitch=0.2)
    assert got[0][0] == L0.n_seg              # rank 0 keeps the workload's seed


def test_rank_seed():
    assert shard.rank_seed(2, 0) == 2 and shard.rank_seed(2, 3) == 3002
