"""One layout's instances searched in shares (the multi-GPU form) on one GPU.

The shares of mpld_shard_instances are searched one after another with
mpld_search_subset_async, each share's per-instance results copied back with
mpld_fetch_instances, merged, and finished with mpld_finish_from; the layout
must equal mpld_solve_batch's and the oracle's bit for bit, with the default
search and with the budgeted split search.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2303_14335_gb300 import mpld, synth

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def stream():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.cuda.Stream()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("split", [False, True])
def test_shares_merged_equal_one_search(world, split, stream):
    L = synth.unit_disk_layout(20000, 3, seed=2, mean_deg=3.0, p_stitch=0.2)
    budget = 6000
    prm = mpld.make_params(node_budget=budget, flags=mpld.MPLD_SPLIT_BUDGET if split else 0)
    s = stream.cuda_stream
    prob = mpld.mpld_build_matrix(L, None, s)
    try:
        owner = mpld.mpld_shard_instances(prob, world)
        sizes = mpld.mpld_instance_sizes(prob)
        C = len(sizes)
        nodes = np.zeros(C, np.int64)
        cost = np.zeros(C, np.int64)
        status = -np.ones(C, np.int32)
        masks = np.zeros(int(sizes.sum()), np.int8)
        off = np.concatenate([[0], np.cumsum(sizes)])
        for r in range(world):
            mine = np.flatnonzero(owner == r)
            mpld.mpld_search_subset_async(prob, mine, prm, s)
            nd, co, stt, ms = mpld.mpld_fetch_instances(prob, s)
            assert (stt[owner != r] == -1).all() and (stt[mine] >= 0).all()
            nodes[mine], cost[mine], status[mine] = nd[mine], co[mine], stt[mine]
            for c in mine:
                masks[off[c]:off[c + 1]] = ms[off[c]:off[c + 1]]
        rc, mask, res = mpld.mpld_finish_from(prob, nodes, cost, status, masks)
        rc1, masks1, res1 = mpld.mpld_solve_batch([prob], prm, s)
    finally:
        prob.close()
    ref = oracle.decompose(L, flags=oracle.SPLIT_BUDGET if split else 0, budget=budget,
                           nthreads=NTHREADS)
    assert np.array_equal(mask, masks1[0]) and np.array_equal(mask, ref.mask)
    assert (res.cost, res.nodes) == (res1[0].cost, res1[0].nodes) == (ref.cost, ref.nodes)
    assert rc == rc1


def test_subset_refuses_bad_lists(stream):
    L = synth.unit_disk_layout(3000, 3, seed=4, mean_deg=3.0, p_stitch=0.2)
    prob = mpld.mpld_build_matrix(L, None, stream.cuda_stream)
    try:
        C = mpld.mpld_problem_info(prob).n_components
        for bad in ([0, 0], [C], [-1]):
            with pytest.raises(mpld.MpldError):
                mpld.mpld_search_subset_async(prob, bad, None, stream.cuda_stream)
        with pytest.raises(mpld.MpldError):
            mpld.mpld_search_subset_async(
                prob, [0], mpld.make_params(flags=mpld.MPLD_PARALLEL_EXACT), stream.cuda_stream)
    finally:
        prob.close()
