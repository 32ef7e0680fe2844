"""CUDA path vs the CPU oracle, element by element (integer work: bit-exact).

Every comparison covers the per-segment masks, the integer cost, the
conflict and stitch counts, the per-instance search node counts and the
status.  The oracle and the library get the same seeded inputs and the same
node budget; their search order is the same by construction (first
minimum-cost leaf of the canonical depth-first order), so the node counts
match too.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2303_14335_gb300 import mpld, synth

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))
SINGLE = mpld.MPLD_NO_SIMPLIFY | mpld.MPLD_SINGLE_INSTANCE


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def stream(torch_cuda):
    return torch_cuda.cuda.Stream()


def edges(L):
    return list(zip(L.conf_u.tolist(), L.conf_v.tolist())), list(zip(L.st_u.tolist(), L.st_v.tolist()))


def gpu_run(L, flags=0, budget=0, path="batch", stream=0, warps=0, slot=0, time_limit_ms=0,
            search_flags=0, cta=0):
    prob = mpld.mpld_build_matrix(L, mpld.make_params(flags=flags), stream)
    prm = mpld.make_params(node_budget=budget, warps_per_cta=warps, slot_bytes=slot,
                           time_limit_ms=time_limit_ms, flags=search_flags, cta_segments=cta)
    if path == "plain":
        rc, mask, res = mpld.mpld_solve(prob, prm, stream)
    else:
        rc, masks, ress = mpld.mpld_solve_batch([prob], prm, stream)
        mask, res = masks[0], ress[0]
    nodes, cost, status, comp_of = mpld.mpld_component_results(prob)
    prob.close()
    return dict(rc=rc, mask=mask, res=res, nodes=nodes, cost=cost, status=status, comp_of=comp_of)


def assert_same(g, ref, L):
    assert np.array_equal(g["mask"], ref.mask), "masks differ"
    assert g["res"].cost == ref.cost
    assert g["res"].n_conflicts == ref.n_conflicts and g["res"].n_stitches == ref.n_stitches
    assert g["res"].nodes == ref.nodes
    assert g["res"].n_components == ref.n_components
    assert g["res"].n_removed_segments == ref.n_removed_segments
    assert np.array_equal(g["comp_of"], ref.comp_of)
    assert np.array_equal(g["nodes"], ref.comp_nodes)
    assert np.array_equal(g["cost"], ref.comp_cost)
    st = np.where(g["status"] == mpld.MPLD_OK, oracle.OK, oracle.BUDGET)
    assert np.array_equal(st, ref.comp_status)
    assert (g["rc"] == mpld.MPLD_BUDGET) == (ref.status == oracle.BUDGET)
    conf, stt = edges(L)
    x = g["mask"]
    assert np.all((x >= 0) & (x < L.k))
    assert g["res"].cost == L.cost_conflict * sum(x[a] == x[b] for a, b in conf) + \
        L.cost_stitch * sum(x[a] != x[b] for a, b in stt)


# ---------------------------------------------------------------- small graphs

def small_cases():
    out = []
    for s in range(48):
        d = synth.uniform(4242, np.arange(3 * s, 3 * s + 3, dtype=np.uint64))
        k = 2 + int(d[0] * 7)            # 2..8: both field widths
        n = 3 + int(d[1] * 16)
        out.append((n, k, 7000 + s, 0.25 + 0.5 * d[2]))
    return out


@pytest.mark.parametrize("n,k,seed,p", small_cases())
def test_small_single_instance(n, k, seed, p, stream):
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=n // 4, identity_polygons=False)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=200000)
    for path in ("batch", "plain"):
        g = gpu_run(L, flags=SINGLE, budget=200000, path=path, stream=stream.cuda_stream)
        assert_same(g, ref, L)


def test_golden_cases(stream):
    import json
    here = os.path.join(os.path.dirname(__file__), "golden")
    for fn in ("hand_traces.json", "fig1_four_clique.json"):
        for c in json.load(open(os.path.join(here, fn)))["cases"]:
            L = synth.graph_from_edges(c["n"], c["k"], c["conf"], c["stitch"])
            g = gpu_run(L, flags=SINGLE, stream=stream.cuda_stream)
            want = c.get("cost", c.get("min_cost"))
            assert g["res"].cost == want
            if "x" in c:
                assert g["mask"].tolist() == c["x"] and g["res"].nodes == c["nodes"]


@pytest.mark.parametrize("budget", [1, 40, 333, 5000])
def test_budget_parity(budget, stream):
    L = synth.unit_disk_layout(40, 3, seed=91, mean_deg=5.0, p_stitch=0.25)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=budget)
    g = gpu_run(L, flags=SINGLE, budget=budget, stream=stream.cuda_stream)
    assert_same(g, ref, L)


# ---------------------------------------------------------------- workloads

def test_workload_k3_n24_plain_exact(stream):
    L, mode = synth.workload("k3_n24_plain")
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE)
    for path in ("batch", "plain"):
        g = gpu_run(L, flags=SINGLE, path=path, stream=stream.cuda_stream)
        assert_same(g, ref, L)
        assert g["rc"] == mpld.MPLD_OK


def test_workload_k3_n400_budgeted(stream):
    L, mode = synth.workload("k3_n400_p025_plain")
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=300000)
    g = gpu_run(L, flags=SINGLE, budget=300000, stream=stream.cuda_stream)
    assert_same(g, ref, L)


@pytest.mark.parametrize("name", ["k3_n200k_p02_batched", "k4_n100k_p03_batched"])
def test_batched_workloads_full_size(name, stream):
    L, mode = synth.workload(name)
    ref = oracle.decompose(L, budget=3000, nthreads=NTHREADS)
    g = gpu_run(L, budget=3000, stream=stream.cuda_stream)
    assert_same(g, ref, L)


@pytest.mark.parametrize("name", ["k3_n200k_p02_batched", "k4_n100k_p03_batched"])
def test_batched_workloads_bench_budget_sampled(name, stream):
    # the benchmark's budget: whole-layout invariants plus a sample of
    # instances solved one by one by the oracle
    budget = 1 << 16
    L, mode = synth.workload(name)
    g = gpu_run(L, budget=budget, stream=stream.cuda_stream)
    conf, st = edges(L)
    comp_of = g["comp_of"]
    assert g["res"].cost == int(g["cost"].sum())
    C = len(g["nodes"])
    order = np.argsort(-np.bincount(comp_of[comp_of >= 0], minlength=C), kind="stable")
    sample = list(order[:6]) + list(range(0, C, max(1, C // 40)))
    cu, cv = L.conf_u, L.conf_v
    su, sv = L.st_u, L.st_v
    for c in sorted(set(int(s) for s in sample)):
        segs = np.nonzero(comp_of == c)[0]
        loc = np.full(L.n_seg, -1, dtype=np.int64)
        loc[segs] = np.arange(len(segs))
        mc = (loc[cu] >= 0) & (loc[cv] >= 0)
        ms = (loc[su] >= 0) & (loc[sv] >= 0)
        r = oracle.solve_instance(len(segs), L.k, np.stack([loc[cu[mc]], loc[cv[mc]]], 1),
                                  np.stack([loc[su[ms]], loc[sv[ms]]], 1), budget=budget)
        assert r.cost == g["cost"][c] and r.nodes == g["nodes"][c]
        assert np.array_equal(r.x, g["mask"][segs])


# ------------------------------------------- the paper's column rule (rule 1)

BFS = mpld.MPLD_COLUMN_BFS


@pytest.mark.parametrize("n,k,seed,p", small_cases()[::2])
def test_rule1_small_single_instance(n, k, seed, p, stream):
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=n // 4, identity_polygons=False)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE | oracle.COLUMN_BFS,
                           budget=200000)
    for path in ("batch", "plain"):
        g = gpu_run(L, flags=SINGLE, budget=200000, path=path, stream=stream.cuda_stream,
                    search_flags=BFS)
        assert_same(g, ref, L)


@pytest.mark.parametrize("budget", [1, 40, 333, 5000])
def test_rule1_budget_parity(budget, stream):
    L = synth.unit_disk_layout(40, 3, seed=91, mean_deg=5.0, p_stitch=0.25)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE | oracle.COLUMN_BFS,
                           budget=budget)
    g = gpu_run(L, flags=SINGLE, budget=budget, stream=stream.cuda_stream, search_flags=BFS)
    assert_same(g, ref, L)


def test_rule1_k8_several_words(stream):
    L = synth.unit_disk_layout(700, 8, seed=3, mean_deg=9.0)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE | oracle.COLUMN_BFS,
                           budget=20000)
    assert_same(gpu_run(L, flags=SINGLE, budget=20000, stream=stream.cuda_stream, search_flags=BFS),
                ref, L)


@pytest.mark.parametrize("name", ["k3_n200k_p02_batched", "k4_n100k_p03_batched"])
def test_rule1_batched_workloads_full_size(name, stream):
    L, mode = synth.workload(name)
    ref = oracle.decompose(L, flags=oracle.COLUMN_BFS, budget=3000, nthreads=NTHREADS)
    g = gpu_run(L, budget=3000, stream=stream.cuda_stream, search_flags=BFS)
    assert_same(g, ref, L)
    # the rule changes the search, not the problem: a plain-path run agrees
    # with the batched one
    p = gpu_run(L, budget=3000, path="plain", stream=stream.cuda_stream, search_flags=BFS)
    assert np.array_equal(p["mask"], g["mask"]) and np.array_equal(p["nodes"], g["nodes"])


def test_rule1_graph_cache_keeps_rules_apart(stream):
    # same problem, same shape, the two rules alternately: a cached graph of
    # one rule must never serve the other
    L = synth.unit_disk_layout(8000, 3, seed=14, mean_deg=3.0, p_stitch=0.2)
    prob = mpld.mpld_build_matrix(L, None, stream.cuda_stream)
    refs = {f: oracle.decompose(L, flags=f and oracle.COLUMN_BFS, budget=1000, nthreads=NTHREADS)
            for f in (0, BFS)}
    for f in (0, BFS, 0, BFS):
        rc, m, r = mpld.mpld_solve_batch([prob], mpld.make_params(node_budget=1000, flags=f),
                                         stream.cuda_stream)
        assert np.array_equal(m[0], refs[f].mask) and r[0].nodes == refs[f].nodes
    prob.close()


# ------------------------------------------- biconnected blocks as instances

BIC = mpld.MPLD_BICONNECTED


@pytest.mark.parametrize("n,k,seed,p", small_cases()[1::3])
def test_blocks_small_graphs(n, k, seed, p, stream):
    L = synth.random_graph(n, k, seed=seed, p_edge=p * 0.6, n_stitch=n // 4, identity_polygons=False)
    for bflags, oflags in ((mpld.MPLD_NO_SIMPLIFY | BIC, oracle.NO_SIMPLIFY | oracle.BICONNECTED),
                           (BIC, oracle.BICONNECTED)):
        ref = oracle.decompose(L, flags=oflags, budget=200000)
        for path in ("batch", "plain"):
            assert_same(gpu_run(L, flags=bflags, budget=200000, path=path, stream=stream.cuda_stream),
                        ref, L)


@pytest.mark.parametrize("name", ["k3_n200k_p02_batched", "k4_n100k_p03_batched"])
@pytest.mark.parametrize("budget", [3000, 1 << 16])
def test_blocks_batched_workloads_full_size(name, budget, stream):
    L, mode = synth.workload(name)
    ref = oracle.decompose(L, flags=oracle.BICONNECTED, budget=budget, nthreads=NTHREADS)
    g = gpu_run(L, flags=BIC, budget=budget, stream=stream.cuda_stream)
    assert_same(g, ref, L)
    assert ref.max_component < L.n_seg


def test_blocks_with_column_rule(stream):
    L = synth.unit_disk_layout(6000, 3, seed=21, mean_deg=4.5, p_stitch=0.2)
    ref = oracle.decompose(L, flags=oracle.BICONNECTED | oracle.COLUMN_BFS, budget=2000,
                           nthreads=NTHREADS)
    assert_same(gpu_run(L, flags=BIC, budget=2000, stream=stream.cuda_stream, search_flags=BFS), ref, L)


# ------------------------------------------------ second bound mode (cliques)

CQ = mpld.MPLD_CLIQUE_BOUND


@pytest.mark.parametrize("n,k,seed,p", small_cases()[2::3])
def test_clique_bound_small_graphs(n, k, seed, p, stream):
    L = synth.random_graph(n, k, seed=seed, p_edge=min(0.9, p + 0.2), n_stitch=n // 4,
                           identity_polygons=False)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE | oracle.CLIQUE_BOUND,
                           budget=200000)
    for path in ("batch", "plain"):
        assert_same(gpu_run(L, flags=SINGLE | CQ, budget=200000, path=path, stream=stream.cuda_stream),
                    ref, L)


@pytest.mark.parametrize("budget", [1, 40, 333, 5000])
def test_clique_bound_budgets(budget, stream):
    L = synth.unit_disk_layout(40, 3, seed=91, mean_deg=6.0, p_stitch=0.25)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE | oracle.CLIQUE_BOUND,
                           budget=budget)
    assert_same(gpu_run(L, flags=SINGLE | CQ, budget=budget, stream=stream.cuda_stream), ref, L)


@pytest.mark.parametrize("k", [3, 4, 8])
def test_clique_bound_large_instance(k, stream):
    # instances above 32 field words take the shared-memory search
    L = synth.unit_disk_layout(300, k, seed=5, mean_deg=2.0 * k)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE | oracle.CLIQUE_BOUND,
                           budget=20000)
    assert ref.max_component > 128
    assert_same(gpu_run(L, flags=SINGLE | CQ, budget=20000, stream=stream.cuda_stream), ref, L)


@pytest.mark.parametrize("name", ["k3_n200k_p02_batched", "k4_n100k_p03_batched"])
def test_clique_bound_batched_workloads(name, stream):
    L, mode = synth.workload(name)
    ref = oracle.decompose(L, flags=oracle.CLIQUE_BOUND, budget=3000, nthreads=NTHREADS)
    assert_same(gpu_run(L, flags=CQ, budget=3000, stream=stream.cuda_stream), ref, L)


def test_clique_bound_with_blocks_and_column_rule(stream):
    L = synth.unit_disk_layout(6000, 3, seed=23, mean_deg=5.0, p_stitch=0.2)
    for fl, ofl, sf in ((CQ | BIC, oracle.CLIQUE_BOUND | oracle.BICONNECTED, 0),
                        (CQ, oracle.CLIQUE_BOUND | oracle.COLUMN_BFS, BFS)):
        ref = oracle.decompose(L, flags=ofl, budget=2000, nthreads=NTHREADS)
        assert_same(gpu_run(L, flags=fl, budget=2000, stream=stream.cuda_stream, search_flags=sf),
                    ref, L)


# ------------------------------------------- whole-CTA teams for large instances

@pytest.mark.parametrize("n,k,seed,p", small_cases()[::4])
def test_cta_teams_small_graphs(n, k, seed, p, stream):
    # a low threshold sends every instance to a CTA team
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=n // 4, identity_polygons=False)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=200000)
    for path in ("batch", "plain"):
        assert_same(gpu_run(L, flags=SINGLE, budget=200000, path=path, stream=stream.cuda_stream,
                            cta=2), ref, L)


@pytest.mark.parametrize("name", ["k3_n200k_p02_batched", "k4_n100k_p03_batched"])
def test_cta_teams_with_warps_in_one_launch(name, stream):
    # instances of 40+ segments go to CTA teams, the rest to warps
    L, mode = synth.workload(name)
    ref = oracle.decompose(L, budget=3000, nthreads=NTHREADS)
    for warps in (0, 1, 16):
        assert_same(gpu_run(L, budget=3000, stream=stream.cuda_stream, warps=warps, cta=40), ref, L)


def test_cta_teams_with_options(stream):
    L = synth.unit_disk_layout(6000, 3, seed=27, mean_deg=5.0, p_stitch=0.2)
    for fl, ofl, sf in ((CQ, oracle.CLIQUE_BOUND, 0), (0, oracle.COLUMN_BFS, BFS),
                        (BIC, oracle.BICONNECTED, 0)):
        ref = oracle.decompose(L, flags=ofl, budget=2000, nthreads=NTHREADS)
        assert_same(gpu_run(L, flags=fl, budget=2000, stream=stream.cuda_stream, search_flags=sf,
                            cta=16), ref, L)


def test_cta_team_large_instance_default_threshold(stream):
    # one 5,000-segment instance: above the default threshold
    L = synth.unit_disk_layout(5000, 3, seed=31, mean_deg=2.5)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=6000)
    assert ref.max_component >= 4096
    for cta in (0, -1):
        assert_same(gpu_run(L, flags=SINGLE, budget=6000, stream=stream.cuda_stream, cta=cta), ref, L)
    # 16-byte slots leave no room for the column classes: every thread of the
    # CTA scans instead
    assert_same(gpu_run(L, flags=SINGLE, budget=6000, stream=stream.cuda_stream, slot=16), ref, L)
    for path in ("batch", "plain"):
        assert_same(gpu_run(L, flags=SINGLE, budget=6000, path=path, stream=stream.cuda_stream),
                    ref, L)


@pytest.mark.parametrize("k,rule", [(3, 0), (3, 1), (4, 0), (8, 0), (2, 1)])
def test_giant_instance_column_classes(k, rule, stream):
    # about 11,000 segments in one instance, searched by warp 0 of a CTA with
    # its column classes in shared memory, under both column rules
    L = synth.unit_disk_layout(9000 if k < 8 else 6000, k, seed=41 + k,
                               mean_deg=4.5 if k < 8 else 9.0, p_stitch=0.2)
    of = oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE | (oracle.COLUMN_BFS if rule else 0)
    ref = oracle.decompose(L, flags=of, budget=3000)
    assert ref.max_component >= 4096
    for cta in (0, 2000):
        assert_same(gpu_run(L, flags=SINGLE, budget=3000, stream=stream.cuda_stream, cta=cta,
                            search_flags=BFS if rule else 0), ref, L)
    # and with no room for the classes: the scan by every thread of the CTA
    assert_same(gpu_run(L, flags=SINGLE, budget=3000, stream=stream.cuda_stream, slot=16,
                        search_flags=BFS if rule else 0), ref, L)


def test_column_classes_backtracking_and_high_degree(stream):
    # instances sent to the one-warp search with column classes (threshold
    # 100): a budget well past the first leaf makes it backtrack, with the
    # counts and offsets in shared memory; a hub of 300 neighbours leaves a
    # degree above 255, and the counts then stay in global memory
    L = synth.unit_disk_layout(700, 3, seed=61, mean_deg=4.5, p_stitch=0.2)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=30000)
    for path in ("batch", "plain"):
        assert_same(gpu_run(L, flags=SINGLE, budget=30000, path=path, stream=stream.cuda_stream,
                            cta=100), ref, L)
    conf = set(zip(L.conf_u.tolist(), L.conf_v.tolist()))
    st = list(zip(L.st_u.tolist(), L.st_v.tolist()))
    conf |= {(0, j) for j in range(1, 301)} - set(st)
    H = synth.graph_from_edges(L.n_seg, 3, sorted(conf), st, polygon_of=L.polygon_of)
    for k in (3, 4):
        H.k = k
        ref = oracle.decompose(H, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=30000)
        for path in ("batch", "plain"):
            assert_same(gpu_run(H, flags=SINGLE, budget=30000, path=path,
                                stream=stream.cuda_stream, cta=100), ref, H)


# ------------------------- a budget that ends the search at its first leaf

def descent_room(n, k, ne2, ns2):
    """Shared-memory bytes the first-descent form needs for its state, then
    with the adjacency offsets, the conflict lists and the stitch lists
    beside it (the layout the kernel carves, restated)."""
    a16 = lambda b: (b + 15) // 16 * 16
    w = (n + 31) // 32
    sw = (w + 31) // 32
    classes = 4 * ((k + 1) * (w + sw + 1) + w + sw)
    fb = 1 if k <= 7 else 2
    base = a16(classes) + a16(fb * ((n + 3) // 4) * 4) + a16(n)
    offs = base + 2 * (a16(2 * (n + 1)) + a16(4 * ((n >> 6) + 1)))
    cn = offs + a16(2 * ne2)
    return [base, offs, cn, cn + a16(2 * ns2)]


def entries(L):
    conf, st = edges(L)
    return 2 * len({(min(a, b), max(a, b)) for a, b in conf}), \
        2 * len({(min(a, b), max(a, b)) for a, b in st})


@pytest.mark.parametrize("k,rule", [(3, 0), (3, 1), (4, 0), (2, 1), (5, 1), (8, 0)])
def test_first_descent_of_a_giant_instance(k, rule, stream):
    # node budgets of at most n + 1 end the search at its first leaf: the
    # descent alone, by one warp, with the adjacency in shared memory as the
    # room allows (every tier), and the full search's scan (16-byte slots)
    L = synth.unit_disk_layout(4500 if k < 8 else 3000, k, seed=71 + k,
                               mean_deg=4.5 if k < 8 else 3.0, p_stitch=0.2 if k < 8 else 0.0)
    n = L.n_seg
    ne2, ns2 = entries(L)
    bounds = descent_room(n, k, ne2, ns2)
    assert bounds[-1] < 200 * 1024
    of = oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE | (oracle.COLUMN_BFS if rule else 0)
    sf = BFS if rule else 0
    for budget in (n + 1, 1000):
        ref = oracle.decompose(L, flags=of, budget=budget)
        assert ref.max_component == n and ref.nodes == n + 1
        scan = gpu_run(L, flags=SINGLE, budget=budget, stream=stream.cuda_stream, slot=16,
                       search_flags=sf, cta=2000)
        assert_same(scan, ref, L)
        rooms = [(lo + hi) // 2 for lo, hi in zip(bounds, bounds[1:])] + [bounds[-1] + 4096]
        for room in rooms:
            slot = (room // 8 + 15) // 16 * 16
            g = gpu_run(L, flags=SINGLE, budget=budget, stream=stream.cuda_stream, warps=8,
                        slot=slot, search_flags=sf, cta=2000)
            assert_same(g, ref, L)
            assert g["res"].work == scan["res"].work
        if k == 8:
            # few neighbours, eight masks, no stitches: the first leaf costs
            # nothing, which ends the search before the budget does
            assert ref.cost == 0 and ref.comp_status[0] == oracle.OK


def test_first_descent_hub_and_split_first_phase(stream):
    # a hub with 100 conflict neighbours (several passes of one warp over a
    # neighbour list), and the budgeted split search's first phase on CTA
    # teams, whose per-search share is below n + 1
    L = synth.unit_disk_layout(4500, 3, seed=77, mean_deg=4.0, p_stitch=0.2)
    conf, st = edges(L)
    conf = set(conf) | ({(0, j) for j in range(1, 101)} - set(st))
    for k in (3, 4):
        H = synth.graph_from_edges(L.n_seg, k, sorted(conf), st, polygon_of=L.polygon_of)
        ref = oracle.decompose(H, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=2000)
        assert ref.nodes == H.n_seg + 1
        for path in ("batch", "plain"):
            assert_same(gpu_run(H, flags=SINGLE, budget=2000, path=path, stream=stream.cuda_stream),
                        ref, H)
    M = synth.unit_disk_layout(30000, 3, seed=79, mean_deg=3.5, p_stitch=0.2)
    ref = oracle.decompose(M, flags=oracle.SPLIT_BUDGET, budget=3000, nthreads=NTHREADS)
    for cta in (40, 100):
        assert_same(gpu_run(M, budget=3000, stream=stream.cuda_stream, cta=cta,
                            search_flags=mpld.MPLD_SPLIT_BUDGET), ref, M)


# ------------------------------ exact search with the warps of a CTA splitting an instance

PAR = mpld.MPLD_PARALLEL_EXACT


def assert_same_answer(g, ref, L):
    """assert_same without the node counts: with the subtrees split over
    warps, how many nodes are visited depends on when each warp sees a better
    incumbent; the answer (first minimum-cost leaf) does not."""
    assert np.array_equal(g["mask"], ref.mask), "masks differ"
    assert g["res"].cost == ref.cost
    assert g["res"].n_conflicts == ref.n_conflicts and g["res"].n_stitches == ref.n_stitches
    assert g["res"].n_components == ref.n_components
    assert np.array_equal(g["comp_of"], ref.comp_of)
    assert np.array_equal(g["cost"], ref.comp_cost)
    assert np.all(g["status"] == mpld.MPLD_OK) and g["rc"] == mpld.MPLD_OK
    assert ref.status == oracle.OK
    assert np.all(g["nodes"] >= 1)
    conf, stt = edges(L)
    x = g["mask"]
    assert g["res"].cost == L.cost_conflict * sum(x[a] == x[b] for a, b in conf) + \
        L.cost_stitch * sum(x[a] != x[b] for a, b in stt)


SPLIT_CASES = [(k, n) for k in (2, 3, 4, 5, 6) for n in (16, 18, 20)] + \
    [(8, 16), (8, 18), (2, 24), (3, 24), (5, 24), (6, 24)]


@pytest.mark.parametrize("k,n", SPLIT_CASES)
def test_split_search_single_instance(k, n, stream):
    # every field width and row count of the register form; 8 and 16 warps
    L = synth.random_graph(n, k, seed=900 + n + k, p_edge=0.5, n_stitch=n // 4, identity_polygons=False)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE)
    assert_same_answer(gpu_run(L, flags=SINGLE, path="plain", stream=stream.cuda_stream,
                               search_flags=PAR), ref, L)
    for warps in (0, 16):
        assert_same_answer(gpu_run(L, flags=SINGLE, stream=stream.cuda_stream, warps=warps,
                                   search_flags=PAR), ref, L)


@pytest.mark.parametrize("k,n", [(3, 20), (4, 18), (6, 18)])
def test_split_search_column_rule(k, n, stream):
    L = synth.random_graph(n, k, seed=900 + n + k, p_edge=0.5, n_stitch=n // 4, identity_polygons=False)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE | oracle.COLUMN_BFS)
    for path in ("batch", "plain"):
        assert_same_answer(gpu_run(L, flags=SINGLE, path=path, stream=stream.cuda_stream,
                                   search_flags=PAR | BFS), ref, L)


def test_split_search_k3_n24_workload(stream):
    L, mode = synth.workload("k3_n24_plain")
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE)
    for path in ("batch", "plain"):
        assert_same_answer(gpu_run(L, flags=SINGLE, path=path, stream=stream.cuda_stream,
                                   search_flags=PAR), ref, L)


@pytest.mark.parametrize("n,k,deg,ps,seed", [(1000, 3, 2.6, 0.2, 5), (600, 4, 4.0, 0.3, 7)])
def test_split_search_layouts(n, k, deg, ps, seed, stream):
    # simplified layouts: instances of 16+ segments split, the rest on warps,
    # in one launch; with the build options too
    L = synth.unit_disk_layout(n, k, seed=seed, mean_deg=deg, p_stitch=ps)
    for fl, ofl, sf in ((0, 0, 0), (CQ, oracle.CLIQUE_BOUND, 0), (BIC, oracle.BICONNECTED, 0),
                        (0, oracle.COLUMN_BFS, BFS)):
        if k == 4 and sf:
            continue      # the column rule's exact tree is 135M nodes here
        ref = oracle.decompose(L, flags=ofl, budget=0, nthreads=NTHREADS)
        for warps in (0, 16):
            assert_same_answer(gpu_run(L, flags=fl, stream=stream.cuda_stream, warps=warps,
                                       search_flags=PAR | sf), ref, L)


def test_split_search_queue_and_cta_forms(stream):
    # 19 instances of 16+ segments: the 16 largest go to the grid-wide queue
    # (one after another, masks recovered by replaying the winning subtree),
    # the other 3 to CTAs in the batched launch, the rest to warps
    L = synth.unit_disk_layout(9000, 3, seed=16, mean_deg=2.35, p_stitch=0.2)
    for fl, ofl, sf in ((0, 0, 0), (CQ, oracle.CLIQUE_BOUND, 0), (0, oracle.COLUMN_BFS, BFS)):
        ref = oracle.decompose(L, flags=ofl, budget=0, nthreads=NTHREADS)
        sizes = np.bincount(ref.comp_of[ref.comp_of >= 0], minlength=ref.n_components)
        assert (sizes >= 16).sum() == 19
        for warps in (0, 16):
            # a 5 s limit per instance (these take milliseconds): a search
            # that ran away would fail the test instead of holding the GPU
            assert_same_answer(gpu_run(L, flags=fl, stream=stream.cuda_stream, warps=warps,
                                       search_flags=PAR | sf, time_limit_ms=5000), ref, L)


def test_split_search_several_problems(stream):
    # a batch of several layouts: 17 split instances (1 + 16), the 16 largest
    # to the queue launch, the smallest to a CTA in the batched launch
    Ls = [synth.unit_disk_layout(1000, 3, seed=5, mean_deg=2.6, p_stitch=0.2),
          synth.unit_disk_layout(5000, 3, seed=12, mean_deg=2.4, p_stitch=0.2)]
    probs = [mpld.mpld_build_matrix(L, None, stream.cuda_stream) for L in Ls]
    try:
        rc, masks, ress = mpld.mpld_solve_batch(probs, mpld.make_params(flags=PAR), stream.cuda_stream)
        assert rc == mpld.MPLD_OK
        for L, m, r in zip(Ls, masks, ress):
            ref = oracle.decompose(L, budget=0, nthreads=NTHREADS)
            assert np.array_equal(m, ref.mask) and r.cost == ref.cost
    finally:
        for p in probs:
            p.close()


def test_split_search_beside_unsplit_large_instances(stream):
    # a 200-segment ring (k = 3) and a 70-segment ring at k = 8 do not fit the
    # register form: whole-CTA search, while the 20-segment graph is split
    conf = [(i, (i + 1) % 200) for i in range(200)]
    R = synth.random_graph(20, 3, seed=77, p_edge=0.5, identity_polygons=False)
    conf += [(200 + a, 200 + b) for a, b in zip(R.conf_u.tolist(), R.conf_v.tolist())]
    L = synth.graph_from_edges(220, 3, conf)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY)
    assert ref.max_component == 200
    for path in ("batch", "plain"):
        assert_same_answer(gpu_run(L, flags=mpld.MPLD_NO_SIMPLIFY, path=path, stream=stream.cuda_stream,
                                   search_flags=PAR), ref, L)
    L = synth.graph_from_edges(70, 8, [(i, (i + 1) % 70) for i in range(70)] + [(0, 35), (10, 50)])
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE)
    assert_same_answer(gpu_run(L, flags=SINGLE, stream=stream.cuda_stream, search_flags=PAR), ref, L)


def test_split_search_repeated_calls(stream):
    # one handle, the grid-wide form replayed from its captured graph, with
    # searches of the other forms in between
    L = synth.random_graph(20, 3, seed=923, p_edge=0.5, n_stitch=5, identity_polygons=False)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE)
    prob = mpld.mpld_build_matrix(L, mpld.make_params(flags=SINGLE), stream.cuda_stream)
    try:
        for sf in (PAR, PAR, 0, PAR, PAR | BFS, PAR):
            rc, masks, ress = mpld.mpld_solve_batch([prob], mpld.make_params(flags=sf), stream.cuda_stream)
            if sf & BFS:
                continue
            assert rc == mpld.MPLD_OK and np.array_equal(masks[0], ref.mask) and ress[0].cost == ref.cost
            if not sf:
                assert ress[0].nodes == ref.nodes
    finally:
        prob.close()


def test_split_search_time_limit(stream):
    # 5 ms against a tree of about 5e8 nodes: every warp stops by itself and
    # the incumbent is a consistent layout
    L = synth.random_graph(20, 8, seed=928, p_edge=0.5, n_stitch=5, identity_polygons=False)
    g = gpu_run(L, flags=SINGLE, time_limit_ms=5, stream=stream.cuda_stream, search_flags=PAR)
    assert g["rc"] == mpld.MPLD_BUDGET
    assert g["status"][0] == mpld.MPLD_TIMEOUT
    conf, st = edges(L)
    x = g["mask"]
    assert np.all((x >= 0) & (x < 8))
    assert g["res"].cost == g["cost"][0] == 10 * sum(x[a] == x[b] for a, b in conf) + \
        sum(x[a] != x[b] for a, b in st)


# ---------------------------------------------------------------- launch forms

def test_results_independent_of_launch_shape(stream):
    L = synth.unit_disk_layout(30000, 3, seed=12, mean_deg=3.2, p_stitch=0.2)
    base = gpu_run(L, budget=4000, stream=stream.cuda_stream)
    for warps, slot in [(1, 0), (2, 0), (8, 0), (16, 0), (4, 1024), (4, 16)]:
        g = gpu_run(L, budget=4000, stream=stream.cuda_stream, warps=warps, slot=slot)
        assert np.array_equal(g["mask"], base["mask"]) and np.array_equal(g["nodes"], base["nodes"])


def test_plain_equals_batched_and_default_stream():
    L = synth.unit_disk_layout(6000, 4, seed=13, mean_deg=5.0, p_stitch=0.3)
    a = gpu_run(L, budget=2000, path="plain", stream=0)
    b = gpu_run(L, budget=2000, path="batch", stream=0)
    assert np.array_equal(a["mask"], b["mask"]) and np.array_equal(a["nodes"], b["nodes"])


def test_multi_problem_batch(stream):
    Ls = [synth.unit_disk_layout(3000 + 500 * i, 3 + (i % 2), seed=30 + i, mean_deg=4.0, p_stitch=0.2)
          for i in range(4)]
    probs = [mpld.mpld_build_matrix(L, None, stream.cuda_stream) for L in Ls]
    prm = mpld.make_params(node_budget=3000)
    rc, masks, ress = mpld.mpld_solve_batch(probs, prm, stream.cuda_stream)
    for L, m, r in zip(Ls, masks, ress):
        ref = oracle.decompose(L, budget=3000, nthreads=NTHREADS)
        assert np.array_equal(m, ref.mask) and r.nodes == ref.nodes and r.cost == ref.cost
    for p in probs:
        p.close()


def test_repeated_calls_and_graph_replay(stream):
    L = synth.unit_disk_layout(8000, 3, seed=14, mean_deg=3.0, p_stitch=0.2)
    prob = mpld.mpld_build_matrix(L, None, stream.cuda_stream)
    prm = mpld.make_params(node_budget=1000)
    outs = [mpld.mpld_solve_batch([prob], prm, stream.cuda_stream) for _ in range(3)]
    for rc, m, r in outs[1:]:
        assert np.array_equal(m[0], outs[0][1][0]) and r[0].nodes == outs[0][2][0].nodes
    # device-only search + fetch gives the same
    mpld.mpld_search_batch_async([prob], prm, stream.cuda_stream)
    rc, m, r = mpld.mpld_fetch(prob, stream.cuda_stream)
    assert np.array_equal(m, outs[0][1][0])
    prob.close()


def test_time_limit_stops_search(stream):
    # unlimited budget, 1 ms per instance: the search must stop by itself and
    # still return a consistent incumbent
    L, mode = synth.workload("k3_n400_p025_plain")
    g = gpu_run(L, flags=SINGLE, budget=0, time_limit_ms=1, stream=stream.cuda_stream)
    assert g["rc"] == mpld.MPLD_BUDGET
    assert g["status"][0] == mpld.MPLD_TIMEOUT
    conf, st = edges(L)
    x = g["mask"]
    assert g["res"].cost == 10 * sum(x[a] == x[b] for a, b in conf) + sum(x[a] != x[b] for a, b in st)


# ---------------------------------------------------------------- edge cases

def test_edge_cases(stream):
    s = stream.cuda_stream
    g = gpu_run(synth.graph_from_edges(0, 3, []), stream=s)
    assert g["res"].n_components == 0 and g["res"].cost == 0
    g = gpu_run(synth.graph_from_edges(5, 3, []), stream=s)          # all simplified away
    assert g["res"].n_removed_segments == 5 and np.all(g["mask"] == 0)
    g = gpu_run(synth.graph_from_edges(5, 3, []), flags=mpld.MPLD_NO_SIMPLIFY, stream=s)
    assert g["res"].n_components == 5 and g["res"].nodes == 10
    g = gpu_run(synth.graph_from_edges(1, 2, []), flags=SINGLE, stream=s)
    assert g["mask"].tolist() == [0] and g["res"].nodes == 2
    # even cycle, k = 2: bipartite, cost 0
    L = synth.graph_from_edges(10, 2, [(i, (i + 1) % 10) for i in range(10)])
    g = gpu_run(L, flags=SINGLE, stream=s)
    assert g["res"].cost == 0
    # duplicates merged
    a = gpu_run(synth.graph_from_edges(4, 3, [(0, 1), (1, 2), (0, 2), (2, 3)]), flags=SINGLE, stream=s)
    L = synth.graph_from_edges(4, 3, [(0, 1), (1, 2), (0, 2), (2, 3)])
    L.conf_u = np.concatenate([L.conf_u, [1, 2]]).astype(np.int32)
    L.conf_v = np.concatenate([L.conf_v, [0, 0]]).astype(np.int32)
    b = gpu_run(L, flags=SINGLE, stream=s)
    assert np.array_equal(a["mask"], b["mask"]) and a["res"].nodes == b["res"].nodes
    # a large k=8 instance exercises several words per lane
    L = synth.unit_disk_layout(700, 8, seed=3, mean_deg=9.0)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=20000)
    assert_same(gpu_run(L, flags=SINGLE, budget=20000, stream=s), ref, L)


# ------------------------------ density balance (a mask renaming after the search)

@pytest.mark.parametrize("n,k,deg,ps,seed", [(20000, 3, 3.0, 0.2, 2), (8000, 4, 5.0, 0.3, 3),
                                             (4000, 6, 7.0, 0.2, 9)])
def test_density_balance(n, k, deg, ps, seed, stream):
    L = synth.unit_disk_layout(n, k, seed=seed, mean_deg=deg, p_stitch=ps)
    DB = mpld.MPLD_DENSITY_BALANCE
    for sf, of in ((0, 0), (mpld.MPLD_SPLIT_BUDGET, oracle.SPLIT_BUDGET)):
        ref = oracle.decompose(L, flags=oracle.DENSITY_BALANCE | of, budget=4000, nthreads=NTHREADS)
        g = gpu_run(L, flags=DB, budget=4000, stream=stream.cuda_stream, search_flags=sf)
        assert_same(g, ref, L)
        counts = np.bincount(g["mask"], minlength=k)
        plain = oracle.decompose(L, flags=of, budget=4000, nthreads=NTHREADS)
        pc = np.bincount(plain.mask, minlength=k)
        assert counts.max() - counts.min() <= pc.max() - pc.min()
