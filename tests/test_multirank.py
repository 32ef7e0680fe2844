"""Multi-rank paths on CPU (gloo, world size 2).

* One layout over two ranks: both build the same problem (host half of the
  library), split its instances with mpld_shard_instances (longest
  processing time first), search only their own share -- here with the CPU
  oracle's instance search standing in for the GPU -- gather the
  per-instance results, and finish with mpld_finish_from.  The gathered
  layout equals a one-rank decomposition bit for bit.
* Independent layouts per rank (the benchmark's weak-scaling form): timing
  aggregation gives total segments and the slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2303_14335_gb300 import mpld, shard, synth

BUDGET = 4000


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def layout():
    return synth.unit_disk_layout(3000, 3, seed=2, mean_deg=3.0, p_stitch=0.2)


def search_share(L, prob, mine):
    """The CPU stand-in for the GPU search of this rank's instances:
    (instance, nodes, cost, status, masks) per owned instance."""
    _, _, _, comp_of = mpld.mpld_component_results(prob, results=False)
    conf = np.stack([L.conf_u, L.conf_v], 1)
    st = np.stack([L.st_u, L.st_v], 1)
    out = []
    for c in mine:
        seg = np.flatnonzero(comp_of == c)
        loc = -np.ones(L.n_seg, dtype=np.int64)
        loc[seg] = np.arange(len(seg))
        cc = [(loc[a], loc[b]) for a, b in conf if loc[a] >= 0 and loc[b] >= 0]
        ss = [(loc[a], loc[b]) for a, b in st if loc[a] >= 0 and loc[b] >= 0]
        r = oracle.solve_instance(len(seg), L.k, cc, ss, budget=BUDGET)
        out.append((int(c), r.nodes, r.cost, r.status, r.x.astype(np.int8)))
    return out


def shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L = layout()
    prob = mpld.mpld_build_matrix(L, mpld.make_params(flags=mpld.MPLD_HOST_ONLY))
    owner = mpld.mpld_shard_instances(prob, world)
    mine = np.flatnonzero(owner == rank)
    part = search_share(L, prob, mine)
    parts = [None] * world
    dist.all_gather_object(parts, (rank, part))
    sizes = mpld.mpld_instance_sizes(prob)
    off = np.concatenate([[0], np.cumsum(sizes)])
    C = len(sizes)
    nodes = np.zeros(C, np.int64)
    cost = np.zeros(C, np.int64)
    status = -np.ones(C, np.int32)
    masks = np.zeros(int(off[-1]), np.int8)
    seen = np.zeros(C, np.int32)
    for r, items in parts:
        for c, nd, co, stt, x in items:
            nodes[c], cost[c], status[c] = nd, co, (mpld.MPLD_BUDGET if stt == oracle.BUDGET else 0)
            masks[off[c]:off[c + 1]] = x
            seen[c] += 1
            assert owner[c] == r
    rc, mask, res = mpld.mpld_finish_from(prob, nodes, cost, status, masks)
    dist.barrier()
    q.put((rank, len(mine), int(seen.min()), int(seen.max()), mask, res.cost, res.nodes,
           res.n_conflicts, res.n_stitches, owner))
    prob.close()
    dist.destroy_process_group()


def test_one_layout_sharded_over_two_ranks_equals_one_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=240) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    L = layout()
    ref = oracle.decompose(L, budget=BUDGET, nthreads=4)
    counts = []
    for rank, n_mine, smin, smax, mask, cost, nodes, ncf, nst, owner in got:
        assert smin == smax == 1                       # every instance searched exactly once
        assert np.array_equal(mask, ref.mask)          # bit for bit
        assert (cost, nodes, ncf, nst) == (ref.cost, ref.nodes, ref.n_conflicts, ref.n_stitches)
        counts.append(n_mine)
    assert sum(counts) == ref.n_components and min(counts) > 0
    assert np.array_equal(got[0][-1], got[1][-1])     # both ranks computed the same shares


def test_shares_are_longest_processing_time_first():
    L = layout()
    prob = mpld.mpld_build_matrix(L, mpld.make_params(flags=mpld.MPLD_HOST_ONLY))
    try:
        sizes = mpld.mpld_instance_sizes(prob)
        _, _, _, comp_of = mpld.mpld_component_results(prob, results=False)
        # work of each instance: segments + adjacency entries (both directions
        # of every conflict and stitch edge inside it)
        work = sizes.astype(np.int64).copy()
        for u, v in list(zip(L.conf_u, L.conf_v)) + list(zip(L.st_u, L.st_v)):
            if comp_of[u] >= 0 and comp_of[u] == comp_of[v]:
                work[comp_of[u]] += 2
        for world in (1, 2, 3, 8):
            owner = mpld.mpld_shard_instances(prob, world)
            # the rule restated: by decreasing work (stable), each to the least
            # loaded rank, ties to the lower rank
            want = np.zeros(len(work), np.int32)
            load = np.zeros(world, np.int64)
            for c in sorted(range(len(work)), key=lambda c: -work[c]):
                r = int(np.argmin(load))
                want[c] = r
                load[r] += work[c]
            assert np.array_equal(owner, want)
        with pytest.raises(mpld.MpldError):
            mpld.mpld_shard_instances(prob, 0)
    finally:
        prob.close()


def weak_worker(rank, world, port, out):
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
    procs = [ctx.Process(target=weak_worker, args=(r, 2, port, q)) for r in range(2)]
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
