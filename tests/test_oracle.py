"""Pins of the CPU oracle against things other than itself.

* brute force over all k^n assignments (Eq. 1) for the minimum cost;
* the bound-free canonical search tree (tests/graph_dfs.py, no dancing
  links) for the assignment = first minimum-cost leaf;
* an independent recursive restatement of the bounded search for node
  counts and the budget rule;
* closed forms: chromatic polynomials for exact-cover counts, pigeonhole
  optima of cliques and odd cycles;
* hand-derived traces and the Fig. 1 cases under tests/golden/;
* invariants of the EC matrix (Sec. 2.3) and of simplification/recovery.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from graph_dfs import bounded_search, brute_force, eq1_cost, first_min_leaf
from paper_2303_14335_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def edges(L):
    return list(zip(L.conf_u.tolist(), L.conf_v.tolist())), list(zip(L.st_u.tolist(), L.st_v.tolist()))


def clique(n):
    return [(a, b) for a in range(n) for b in range(a + 1, n)]


def cycle(n):
    return [(min(i, (i + 1) % n), max(i, (i + 1) % n)) for i in range(n)]


# ---------------------------------------------------------------- fixed cases

def test_golden_fig1():
    g = json.load(open(os.path.join(GOLDEN, "fig1_four_clique.json")))
    for c in g["cases"]:
        r = oracle.solve_instance(c["n"], c["k"], c["conf"], c["stitch"])
        assert r.cost == c["min_cost"]
        conf_n = sum(1 for a, b in c["conf"] if r.x[a] == r.x[b])
        st_n = sum(1 for a, b in c["stitch"] if r.x[a] != r.x[b])
        assert (conf_n, st_n) == (c["min_conflicts"], c["min_stitches"])


def test_golden_hand_traces():
    g = json.load(open(os.path.join(GOLDEN, "hand_traces.json")))
    for c in g["cases"]:
        r = oracle.solve_instance(c["n"], c["k"], c["conf"], c["stitch"])
        assert (r.cost, r.x.tolist(), r.nodes) == (c["cost"], c["x"], c["nodes"]), c["name"]
        # the same numbers from the recursion over the partial assignment
        cost, x, nodes, hit = bounded_search(c["n"], c["k"], c["conf"], c["stitch"])
        assert (cost, x, nodes, hit) == (c["cost"], c["x"], c["nodes"], False), c["name"]


@pytest.mark.parametrize("n,k,conf,cost,n_opt", [
    (3, 3, clique(3), 0, 6),        # triangle, k=3: 3! proper colourings
    (4, 3, clique(4), 10, 36),      # K4, k=3: C(4,2) mono pairs x 3 x 2 x 1
    (5, 2, cycle(5), 10, 10),       # C5, k=2: 5 mono edges x 2
    (5, 4, clique(5), 10, 240),     # K5, k=4: C(5,2) x 4!
])
def test_fixed_optima(n, k, conf, cost, n_opt):
    r = oracle.solve_instance(n, k, conf)
    assert r.cost == cost
    assert eq1_cost(r.x, conf, []) == cost
    m, cnt = brute_force(n, k, conf, [])
    assert (m, cnt) == (cost, n_opt)


def chromatic_cases():
    out = []
    for k in (2, 3, 4):
        for n in (3, 4, 5, 6):
            out.append(("cycle", n, k, cycle(n), (k - 1) ** n + (-1) ** n * (k - 1)))
            out.append(("clique", n, k, clique(n), math.perm(k, n) if n <= k else 0))
            path = [(i, i + 1) for i in range(n - 1)]
            out.append(("path", n, k, path, k * (k - 1) ** (n - 1)))
            out.append(("empty", n, k, [], k ** n))
            star = [(0, i) for i in range(1, n)]
            out.append(("star", n, k, star, k * (k - 1) ** (n - 1)))
    return out


@pytest.mark.parametrize("kind,n,k,conf,want", chromatic_cases())
def test_exact_cover_count_is_chromatic_polynomial(kind, n, k, conf, want):
    # With no stitches, exact covers of the EC matrix = proper k-colourings.
    assert oracle.count_exact_covers(n, k, conf) == want


def test_triangle_has_six_exact_covers():
    assert oracle.count_exact_covers(3, 3, clique(3)) == 6


# ---------------------------------------------------------------- EC matrix

def test_export_matrix_structure():
    L = synth.random_graph(6, 3, seed=2, p_edge=0.5)
    conf, _ = edges(L)
    M = oracle.export_matrix(6, 3, conf)
    n, k, ne = 6, 3, len(conf)
    assert M.shape == (n * k, 1 + n + k * ne)
    for v in range(n):
        for c in range(k):
            row = M[v * k + c]
            want = np.zeros_like(row)
            want[1 + v] = 1
            for e, (a, b) in enumerate(conf):
                if v in (a, b):
                    want[1 + n + e * k + c] = 1
            assert np.array_equal(row, want)


@pytest.mark.parametrize("seed", range(20))
def test_zero_cost_result_is_exact_cover(seed):
    L = synth.random_graph(7, 3, seed=100 + seed, p_edge=0.35)
    conf, _ = edges(L)
    r = oracle.solve_instance(7, 3, conf)
    M = oracle.export_matrix(7, 3, conf)
    chosen = M[[v * 3 + int(r.x[v]) for v in range(7)]]
    colsum = chosen.sum(axis=0)
    assert np.all(colsum[1:1 + 7] == 1)               # primary: exactly once
    if r.cost == 0:
        assert np.all(colsum[1 + 7:] <= 1)            # secondary: at most once
    else:
        # every doubly covered secondary column is a monochromatic conflict edge
        assert int((colsum[1 + 7:] == 2).sum()) * 10 == r.cost


# ---------------------------------------------------------------- search

def random_cases(count, nmax):
    out = []
    for s in range(count):
        rng = synth.uniform(999, np.arange(4 * s, 4 * s + 4, dtype=np.uint64))
        n = 2 + int(rng[0] * (nmax - 1))
        k = 2 + int(rng[1] * 3)
        while k ** n > 300_000:
            n -= 1
        p = 0.2 + 0.6 * rng[2]
        ns = int(rng[3] * 3)
        out.append((n, k, 1000 + s, p, ns))
    return out


@pytest.mark.parametrize("n,k,seed,p,ns", random_cases(60, 10))
def test_oracle_matches_brute_force_and_canonical_order(n, k, seed, p, ns):
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=ns)
    conf, st = edges(L)
    r = oracle.solve_instance(n, k, conf, st)
    m, _ = brute_force(n, k, conf, st)
    assert r.cost == m
    assert eq1_cost(r.x, conf, st) == r.cost
    if k ** n <= 20000:
        c, x = first_min_leaf(n, k, conf, st)
        assert (c, x) == (r.cost, r.x.tolist())
    c2, x2, nodes2, hit2 = bounded_search(n, k, conf, st)
    assert (c2, x2, nodes2) == (r.cost, r.x.tolist(), r.nodes)
    assert not hit2 and r.status == oracle.OK


@pytest.mark.parametrize("seed", range(8))
def test_costs_other_than_default(seed):
    L = synth.random_graph(8, 3, seed=40 + seed, p_edge=0.5, n_stitch=3)
    conf, st = edges(L)
    r = oracle.solve_instance(8, 3, conf, st, cost_conflict=3, cost_stitch=2)
    m, _ = brute_force(8, 3, conf, st, cc=3, cs=2)
    assert r.cost == m
    c2, x2, nodes2, _ = bounded_search(8, 3, conf, st, cc=3, cs=2)
    assert (c2, x2, nodes2) == (r.cost, r.x.tolist(), r.nodes)


@pytest.mark.parametrize("budget", [9, 10, 25, 60, 200])
def test_budget_rule(budget):
    L = synth.random_graph(11, 3, seed=77, p_edge=0.55, n_stitch=2)
    conf, st = edges(L)
    full = oracle.solve_instance(11, 3, conf, st)
    r = oracle.solve_instance(11, 3, conf, st, budget=budget)
    c2, x2, nodes2, hit2 = bounded_search(11, 3, conf, st, budget=budget)
    assert (r.cost, r.x.tolist(), r.nodes) == (c2, x2, nodes2)
    assert (r.status == oracle.BUDGET) == hit2
    if full.nodes > max(budget, 12):
        assert r.status == oracle.BUDGET and r.nodes == max(budget, 12)
        assert r.cost >= full.cost
    assert eq1_cost(r.x, conf, st) == r.cost


def test_budget_never_cuts_first_descent():
    # the first descent reaches a leaf after n+1 nodes even with budget 1
    L = synth.random_graph(9, 3, seed=5, p_edge=0.6)
    conf, _ = edges(L)
    r = oracle.solve_instance(9, 3, conf, budget=1)
    assert r.nodes == 10 and np.all(r.x >= 0)


def test_larger_instances_against_independent_search():
    for s in range(6):
        L = synth.unit_disk_layout(16, 3, seed=300 + s, mean_deg=4.5, p_stitch=0.25)
        conf, st = edges(L)
        r = oracle.solve_instance(L.n_seg, 3, conf, st, budget=20000)
        c2, x2, nodes2, hit2 = bounded_search(L.n_seg, 3, conf, st, budget=20000)
        assert (r.cost, r.x.tolist(), r.nodes, r.status == oracle.BUDGET) == (c2, x2, nodes2, hit2)


def test_invalid_inputs():
    with pytest.raises(ValueError):
        oracle.solve_instance(3, 3, [(0, 0)])
    with pytest.raises(ValueError):
        oracle.solve_instance(3, 3, [(0, 3)])
    with pytest.raises(ValueError):
        oracle.solve_instance(3, 9, [(0, 1)])
    with pytest.raises(ValueError):
        oracle.solve_instance(3, 1, [(0, 1)])


def test_duplicate_edges_are_merged():
    a = oracle.solve_instance(4, 3, clique(4))
    b = oracle.solve_instance(4, 3, clique(4) + [(1, 0), (3, 2)])
    assert (a.cost, a.x.tolist(), a.nodes) == (b.cost, b.x.tolist(), b.nodes)


# ---------------------------------------------------------------- layout flow

def kcore_ok(L, res):
    """Every remaining unit has >= k conflict edges to other remaining units."""
    unit = {}
    parent = list(range(L.n_seg))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a
    first = {}
    for s in range(L.n_seg):
        p = int(L.polygon_of[s])
        if p in first:
            ra, rb = find(first[p]), find(s)
            parent[max(ra, rb)] = min(ra, rb)
        else:
            first[p] = s
    for a, b in zip(L.st_u, L.st_v):
        ra, rb = find(int(a)), find(int(b))
        parent[max(ra, rb)] = min(ra, rb)
    for s in range(L.n_seg):
        unit[s] = find(s)
    deg = {}
    for a, b in zip(L.conf_u, L.conf_v):
        a, b = int(a), int(b)
        if res.comp_of[a] >= 0 and res.comp_of[b] >= 0 and unit[a] != unit[b]:
            deg[unit[a]] = deg.get(unit[a], 0) + 1
            deg[unit[b]] = deg.get(unit[b], 0) + 1
    for s in range(L.n_seg):
        if res.comp_of[s] >= 0 and deg.get(unit[s], 0) < L.k:
            return False
    return True


@pytest.mark.parametrize("seed", range(12))
def test_simplification_preserves_optimum(seed):
    # whole-layout brute force vs simplify + components + search + recover
    L = synth.unit_disk_layout(9, 3, seed=500 + seed, mean_deg=3.5, p_stitch=0.2)
    if 3 ** L.n_seg > 300_000:
        pytest.skip("too many segments for brute force")
    conf, st = edges(L)
    res = oracle.decompose(L)
    m, _ = brute_force(L.n_seg, 3, conf, st)
    assert res.cost == m
    assert eq1_cost(res.mask, conf, st) == res.cost
    assert res.component_cost_sum == res.cost
    assert res.n_conflicts * 10 + res.n_stitches == res.cost
    assert kcore_ok(L, res)


@pytest.mark.parametrize("k,deg,p", [(3, 3.0, 0.2), (4, 5.0, 0.3), (3, 4.0, 0.0)])
def test_decompose_invariants_midsize(k, deg, p):
    L = synth.unit_disk_layout(3000, k, seed=42, mean_deg=deg, p_stitch=p)
    conf, st = edges(L)
    res = oracle.decompose(L, budget=20000, nthreads=4)
    assert np.all((res.mask >= 0) & (res.mask < k))
    assert eq1_cost(res.mask, conf, st) == res.cost
    assert res.component_cost_sum == res.cost       # removed units cost nothing
    assert kcore_ok(L, res)
    # components are connected pieces with ascending ids by lowest segment
    firsts = [int(np.nonzero(res.comp_of == c)[0][0]) for c in range(res.n_components)]
    assert firsts == sorted(firsts)
    # each component result equals a stand-alone search of that component
    for c in range(min(res.n_components, 25)):
        segs = np.nonzero(res.comp_of == c)[0]
        loc = {int(s): i for i, s in enumerate(segs)}
        cc = [(loc[a], loc[b]) for a, b in conf if a in loc and b in loc]
        ss = [(loc[a], loc[b]) for a, b in st if a in loc and b in loc]
        r = oracle.solve_instance(len(segs), k, cc, ss, budget=20000)
        assert r.cost == res.comp_cost[c] and r.nodes == res.comp_nodes[c]
        assert np.array_equal(r.x, res.mask[segs])


def test_decompose_thread_count_does_not_change_results():
    L = synth.unit_disk_layout(4000, 3, seed=8, mean_deg=3.0, p_stitch=0.2)
    a = oracle.decompose(L, budget=5000, nthreads=1)
    b = oracle.decompose(L, budget=5000, nthreads=6)
    assert np.array_equal(a.mask, b.mask) and a.nodes == b.nodes and a.cost == b.cost


def test_single_instance_mode_matches_solve_instance():
    L, mode = synth.workload("k3_n24_plain")
    conf, st = edges(L)
    res = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE)
    r = oracle.solve_instance(L.n_seg, 3, conf, st)
    assert res.n_components == 1 and np.array_equal(res.mask, r.x) and res.nodes == r.nodes


def test_empty_and_isolated():
    L = synth.graph_from_edges(0, 3, [])
    res = oracle.decompose(L)
    assert res.n_components == 0 and res.cost == 0
    L = synth.graph_from_edges(5, 3, [])
    res = oracle.decompose(L)            # everything simplified away
    assert res.n_removed_segments == 5 and np.all(res.mask == 0)
    res = oracle.decompose(L, flags=oracle.NO_SIMPLIFY)
    assert res.n_components == 5 and res.nodes == 10 and np.all(res.mask == 0)


# ---------------------------------------------------------------- paper's column rule

def test_bfs_rank_hand_example():
    # path 0-1-2 plus stitch 0-3 and isolated 4: BFS from 0 visits 1, 3 (ascending), then 2
    from graph_dfs import bfs_rank
    assert bfs_rank(5, [(0, 1), (1, 2)], [(0, 3)]) == [0, 1, 3, 2, 4]


@pytest.mark.parametrize("n,k,seed,p,ns", random_cases(40, 10))
def test_paper_column_rule_matches_brute_force_and_independent_search(n, k, seed, p, ns):
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=ns)
    conf, st = edges(L)
    r = oracle.solve_instance(n, k, conf, st, rule=1)
    m, _ = brute_force(n, k, conf, st)
    assert r.cost == m and eq1_cost(r.x, conf, st) == m
    if k ** n <= 20000:
        assert first_min_leaf(n, k, conf, st, rule=1) == (r.cost, r.x.tolist())
    c2, x2, nodes2, _ = bounded_search(n, k, conf, st, rule=1)
    assert (c2, x2, nodes2) == (r.cost, r.x.tolist(), r.nodes)


@pytest.mark.parametrize("budget", [12, 50, 400])
def test_paper_column_rule_budget(budget):
    L = synth.unit_disk_layout(14, 3, seed=404, mean_deg=4.5, p_stitch=0.25)
    conf, st = edges(L)
    r = oracle.solve_instance(L.n_seg, 3, conf, st, budget=budget, rule=1)
    c2, x2, nodes2, hit2 = bounded_search(L.n_seg, 3, conf, st, budget=budget, rule=1)
    assert (r.cost, r.x.tolist(), r.nodes, r.status == oracle.BUDGET) == (c2, x2, nodes2, hit2)


def test_paper_column_rule_in_layout_flow():
    L = synth.unit_disk_layout(3000, 3, seed=21, mean_deg=3.5, p_stitch=0.2)
    a = oracle.decompose(L, budget=3000, flags=oracle.COLUMN_BFS, nthreads=4)
    conf, st = edges(L)
    assert eq1_cost(a.mask, conf, st) == a.cost == a.component_cost_sum
    for c in range(0, a.n_components, 9):
        segs = np.nonzero(a.comp_of == c)[0]
        loc = {int(s): i for i, s in enumerate(segs)}
        cc = [(loc[u], loc[v]) for u, v in conf if u in loc and v in loc]
        ss = [(loc[u], loc[v]) for u, v in st if u in loc and v in loc]
        r = oracle.solve_instance(len(segs), 3, cc, ss, budget=3000, rule=1)
        assert r.nodes == a.comp_nodes[c] and np.array_equal(r.x, a.mask[segs])
