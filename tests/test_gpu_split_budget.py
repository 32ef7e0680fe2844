"""The budgeted split search (MPLD_SPLIT_BUDGET) on the GPU vs the oracle's
SPLIT_BUDGET mode, element by element.

The mode's result does not depend on timing: the first search and every
subtree search have their own budgets and bounds, so masks, costs, per-
instance node counts and statuses must all equal the oracle's, for the
register form (at most 128 segments, 64 at k = 8) and the general form
(larger instances, state in global memory), on the batched path (one layout
or several), the plain path, several launch shapes, both column rules, and
the full-size layouts of the benchmark.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2303_14335_gb300 import mpld, synth

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))
SINGLE = mpld.MPLD_NO_SIMPLIFY | mpld.MPLD_SINGLE_INSTANCE
SPLIT = mpld.MPLD_SPLIT_BUDGET
BFS = mpld.MPLD_COLUMN_BFS


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def stream(torch_cuda):
    return torch_cuda.cuda.Stream()


def gpu_run(L, flags=0, budget=0, path="batch", stream=0, warps=0, slot=0, search_flags=SPLIT,
            time_limit_ms=0):
    prob = mpld.mpld_build_matrix(L, mpld.make_params(flags=flags), stream)
    prm = mpld.make_params(node_budget=budget, warps_per_cta=warps, slot_bytes=slot,
                           flags=search_flags, time_limit_ms=time_limit_ms)
    try:
        if path == "plain":
            rc, mask, res = mpld.mpld_solve(prob, prm, stream)
        else:
            rc, masks, ress = mpld.mpld_solve_batch([prob], prm, stream)
            mask, res = masks[0], ress[0]
        nodes, cost, status, comp_of = mpld.mpld_component_results(prob)
    finally:
        prob.close()
    return dict(rc=rc, mask=mask, res=res, nodes=nodes, cost=cost, status=status, comp_of=comp_of)


def assert_same(g, ref, L):
    assert np.array_equal(g["mask"], ref.mask), "masks differ"
    assert g["res"].cost == ref.cost
    assert g["res"].n_conflicts == ref.n_conflicts and g["res"].n_stitches == ref.n_stitches
    assert np.array_equal(g["cost"], ref.comp_cost)
    assert np.array_equal(g["nodes"], ref.comp_nodes)
    assert g["res"].nodes == ref.nodes
    st = np.where(g["status"] == mpld.MPLD_OK, oracle.OK, oracle.BUDGET)
    assert np.array_equal(st, ref.comp_status)
    assert np.all((g["status"] == mpld.MPLD_OK) | (g["status"] == mpld.MPLD_BUDGET))
    assert (g["rc"] == mpld.MPLD_BUDGET) == (ref.status == oracle.BUDGET)


def single_cases():
    out = []
    for s in range(24):
        d = synth.uniform(8181, np.arange(3 * s, 3 * s + 3, dtype=np.uint64))
        k = 2 + int(d[0] * 7)            # 2..8: both field widths
        n = 10 + int(d[1] * 40)
        out.append((n, k, 5100 + s, 0.2 + 0.4 * d[2]))
    return out


@pytest.mark.parametrize("n,k,seed,p", single_cases())
def test_single_instance_register_form(n, k, seed, p, stream):
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=n // 4, identity_polygons=False)
    for budget in (300, 5000):
        ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE |
                               oracle.SPLIT_BUDGET, budget=budget)
        for path in ("batch", "plain"):
            assert_same(gpu_run(L, flags=SINGLE, budget=budget, path=path,
                                stream=stream.cuda_stream), ref, L)


@pytest.mark.parametrize("n,k,deg", [(200, 3, 4.5), (300, 4, 5.0), (150, 5, 6.0), (90, 8, 9.0),
                                     (506, 3, 4.5)])
def test_single_instance_general_form(n, k, deg, stream):
    # beyond the register form: each subtree search keeps its state in the
    # warp's own global region
    L = synth.unit_disk_layout(n, k, seed=60 + n, mean_deg=deg, p_stitch=0.25)
    for budget in (2000, 30000):
        ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE |
                               oracle.SPLIT_BUDGET, budget=budget)
        assert ref.status == oracle.BUDGET
        for path in ("batch", "plain"):
            assert_same(gpu_run(L, flags=SINGLE, budget=budget, path=path,
                                stream=stream.cuda_stream), ref, L)


@pytest.mark.parametrize("k", [3, 4])
def test_single_instance_column_rule(k, stream):
    L = synth.unit_disk_layout(120 if k == 3 else 180, k, seed=71, mean_deg=4.5, p_stitch=0.2)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE |
                           oracle.SPLIT_BUDGET | oracle.COLUMN_BFS, budget=8000)
    assert_same(gpu_run(L, flags=SINGLE, budget=8000, stream=stream.cuda_stream,
                        search_flags=SPLIT | BFS), ref, L)


@pytest.mark.parametrize("n,k,deg,ps,seed,budget", [
    (20000, 3, 3.0, 0.2, 2, 6000), (10000, 4, 5.0, 0.3, 3, 6000), (3000, 8, 9.0, 0.1, 4, 4000)])
def test_layouts_every_launch_shape(n, k, deg, ps, seed, budget, stream):
    L = synth.unit_disk_layout(n, k, seed=seed, mean_deg=deg, p_stitch=ps)
    ref = oracle.decompose(L, flags=oracle.SPLIT_BUDGET, budget=budget, nthreads=NTHREADS)
    assert ref.n_budget_components > 0
    for warps in (0, 1, 4, 16):
        assert_same(gpu_run(L, budget=budget, stream=stream.cuda_stream, warps=warps), ref, L)


def test_layout_column_rule(stream):
    L = synth.unit_disk_layout(20000, 3, seed=5, mean_deg=3.0, p_stitch=0.2)
    ref = oracle.decompose(L, flags=oracle.SPLIT_BUDGET | oracle.COLUMN_BFS, budget=6000,
                           nthreads=NTHREADS)
    assert_same(gpu_run(L, budget=6000, stream=stream.cuda_stream, search_flags=SPLIT | BFS),
                ref, L)


def test_several_layouts_in_one_call(stream):
    Ls = [synth.unit_disk_layout(8000, 3, seed=21, mean_deg=3.0, p_stitch=0.2),
          synth.unit_disk_layout(4000, 4, seed=22, mean_deg=5.0, p_stitch=0.3)]
    probs = [mpld.mpld_build_matrix(L, None, stream.cuda_stream) for L in Ls]
    try:
        rc, masks, ress = mpld.mpld_solve_batch(
            probs, mpld.make_params(node_budget=5000, flags=SPLIT), stream.cuda_stream)
        for L, m, r, p in zip(Ls, masks, ress, probs):
            ref = oracle.decompose(L, flags=oracle.SPLIT_BUDGET, budget=5000, nthreads=NTHREADS)
            nodes, cost, status, _ = mpld.mpld_component_results(p)
            assert np.array_equal(m, ref.mask) and r.cost == ref.cost and r.nodes == ref.nodes
            assert np.array_equal(nodes, ref.comp_nodes) and np.array_equal(cost, ref.comp_cost)
    finally:
        for p in probs:
            p.close()


def test_repeated_calls_and_other_modes_between(stream):
    # one handle: the captured two-launch graph replayed, with the plain
    # search and exhaustive search in between
    L = synth.unit_disk_layout(5000, 3, seed=31, mean_deg=3.0, p_stitch=0.2)
    ref = oracle.decompose(L, flags=oracle.SPLIT_BUDGET, budget=4000, nthreads=NTHREADS)
    ref0 = oracle.decompose(L, budget=4000, nthreads=NTHREADS)
    prob = mpld.mpld_build_matrix(L, None, stream.cuda_stream)
    try:
        for sf in (SPLIT, SPLIT, 0, SPLIT, 0, SPLIT):
            rc, masks, ress = mpld.mpld_solve_batch(
                [prob], mpld.make_params(node_budget=4000, flags=sf), stream.cuda_stream)
            want = ref if sf else ref0
            assert np.array_equal(masks[0], want.mask) and ress[0].cost == want.cost
            assert ress[0].nodes == want.nodes
    finally:
        prob.close()


def test_exhaustive_without_budget(stream):
    # node budget 0: the first search is exhaustive and its answer stands
    L = synth.random_graph(14, 3, seed=41, p_edge=0.5, n_stitch=3, identity_polygons=False)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE)
    g = gpu_run(L, flags=SINGLE, budget=0, stream=stream.cuda_stream)
    assert_same(g, ref, L)


def test_refused_combinations(stream):
    L = synth.unit_disk_layout(2000, 3, seed=51, mean_deg=3.0, p_stitch=0.2)
    prob = mpld.mpld_build_matrix(L, mpld.make_params(flags=mpld.MPLD_CLIQUE_BOUND),
                                  stream.cuda_stream)
    try:
        with pytest.raises(mpld.MpldError) as e:
            mpld.mpld_solve_batch([prob], mpld.make_params(node_budget=100, flags=SPLIT),
                                  stream.cuda_stream)
        assert e.value.code == mpld.MPLD_E_INVALID
    finally:
        prob.close()
    prob = mpld.mpld_build_matrix(L, None, stream.cuda_stream)
    try:
        with pytest.raises(mpld.MpldError) as e:
            mpld.mpld_solve_batch(
                [prob], mpld.make_params(flags=SPLIT | mpld.MPLD_PARALLEL_EXACT), stream.cuda_stream)
        assert e.value.code == mpld.MPLD_E_INVALID
    finally:
        prob.close()


@pytest.mark.parametrize("name", ["k3_n200k_p02_batched", "k4_n100k_p03_batched",
                                  "k3_n400_p025_plain"])
def test_full_size_workloads(name, stream):
    L, mode = synth.workload(name)
    single = mode == "single"
    ref = oracle.decompose(L, flags=oracle.SPLIT_BUDGET | (
        oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE if single else 0), budget=65536,
        nthreads=NTHREADS)
    assert_same(gpu_run(L, flags=SINGLE if single else 0, budget=65536,
                        stream=stream.cuda_stream), ref, L)
