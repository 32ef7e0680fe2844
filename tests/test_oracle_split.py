"""Pins of the oracle's budgeted split search (SPLIT_BUDGET).

The mode spends an instance's node budget B on a first search and then on
independent searches of the subtrees below a fixed cut depth, each with
ceil(B / (S + 1)) nodes and the first search's incumbent as its starting
bound (the task parallelism of Sec. 1 / Sec. 2.3 applied inside one
sub-graph; the definition is in the oracle's source).  It is checked
against things other than the oracle's dancing links:

* an independent restatement over the partial assignment
  (tests/graph_dfs.py: split_search), node counts included;
* when no subtree search runs out of budget, the answer is the first
  minimum-cost leaf of the whole tree (the bound-free enumeration of
  tests/graph_dfs.py), and its cost is the brute-force minimum of Eq. 1;
* with no budget it is the exhaustive search, node for node;
* on a layout, the flow (simplify, split, search, recover) gives each
  instance the mode's own answer for that instance;
* an instance above the size limit is searched once with the whole budget
  (the plain search's answer and node count).
"""
import numpy as np
import pytest

import oracle
from graph_dfs import (bounded_search, brute_force, eq1_cost, first_min_leaf, split_cut,
                       split_search)
from paper_2303_14335_gb300 import synth


def graph(seed, base=555, max_leaves=None):
    """A seeded random graph with stitches: k in 2..4, n in 6..12 (fewer
    segments when the bound-free tree, k^n leaves, must stay enumerable)."""
    d = synth.uniform(base, np.arange(3 * seed, 3 * seed + 3, dtype=np.uint64))
    k = 2 + int(d[0] * 3)
    n = 6 + int(d[1] * 7)
    while max_leaves and k ** n > max_leaves:
        n -= 1
    L = synth.random_graph(n, k, seed=3000 + seed, p_edge=0.3 + 0.4 * d[2], n_stitch=n // 4,
                           identity_polygons=False)
    conf = list(zip(L.conf_u.tolist(), L.conf_v.tolist()))
    st = list(zip(L.st_u.tolist(), L.st_v.tolist()))
    return n, k, conf, st


def test_cut_depths():
    # first depth with k^D >= 64, never below the leaves
    assert [split_cut(100, k) for k in range(2, 9)] == [
        (6, 64), (4, 81), (3, 64), (3, 125), (3, 216), (3, 343), (2, 64)]
    assert split_cut(3, 3) == (3, 27) and split_cut(0, 3) == (0, 1)


@pytest.mark.parametrize("seed", range(40))
def test_split_search_matches_restatement(seed):
    n, k, conf, st = graph(seed)
    lowest = brute_force(n, k, conf, st)[0] if k ** n <= 100000 else 0
    for B in (1, 50, 300, 2000):
        r = oracle.solve_instance(n, k, conf, st, budget=B, split=True)
        c, x, nodes, hit = split_search(n, k, conf, st, budget=B)
        assert (r.cost, r.x.tolist(), r.nodes, r.status == oracle.BUDGET) == (c, x, nodes, hit)
        assert r.cost == eq1_cost(r.x, conf, st)
        assert r.cost >= lowest


@pytest.mark.parametrize("seed", range(40, 60))
def test_split_search_column_rule_matches_restatement(seed):
    n, k, conf, st = graph(seed)
    for B in (30, 500, 5000):
        r = oracle.solve_instance(n, k, conf, st, budget=B, split=True, rule=1)
        c, x, nodes, hit = split_search(n, k, conf, st, budget=B, rule=1)
        assert (r.cost, r.x.tolist(), r.nodes, r.status == oracle.BUDGET) == (c, x, nodes, hit)


@pytest.mark.parametrize("seed", range(60, 90))
def test_subtrees_searched_to_the_end_give_the_first_minimum_leaf(seed):
    n, k, conf, st = graph(seed, max_leaves=60000)
    want_c, want_x = first_min_leaf(n, k, conf, st)
    assert want_c == brute_force(n, k, conf, st)[0]
    # a budget that stops the first search but no subtree search, when there is one
    seen_phase2 = False
    for B in (40, 100, 400, 1600, 6400, 25600):
        D, S = split_cut(n, k)
        b = (B + S) // (S + 1)
        if not bounded_search(n, k, conf, st, budget=b)[3]:
            continue
        r = oracle.solve_instance(n, k, conf, st, budget=B, split=True)
        if r.status == oracle.OK:
            seen_phase2 = True
            assert (r.cost, r.x.tolist()) == (want_c, want_x)
    if not seen_phase2:
        pytest.skip("no budget in the list stops only the first search")


@pytest.mark.parametrize("seed", range(90, 110))
def test_no_budget_is_the_exhaustive_search(seed):
    n, k, conf, st = graph(seed, max_leaves=60000)
    a = oracle.solve_instance(n, k, conf, st, budget=0, split=True)
    b = oracle.solve_instance(n, k, conf, st, budget=0)
    assert (a.cost, a.x.tolist(), a.nodes, a.status) == (b.cost, b.x.tolist(), b.nodes, b.status)
    assert (a.cost, a.x.tolist()) == first_min_leaf(n, k, conf, st)


def test_split_search_never_worse_than_its_first_search():
    worse = 0
    for seed in range(110, 150):
        n, k, conf, st = graph(seed)
        for B in (60, 600):
            D, S = split_cut(n, k)
            first = bounded_search(n, k, conf, st, budget=(B + S) // (S + 1))
            r = oracle.solve_instance(n, k, conf, st, budget=B, split=True)
            worse += r.cost > first[0]
    assert worse == 0


@pytest.mark.parametrize("k,deg", [(3, 3.0), (4, 4.5)])
def test_layout_instances_take_the_modes_answer(k, deg):
    L = synth.unit_disk_layout(1500, k, seed=41, mean_deg=deg, p_stitch=0.2)
    B = 3000
    r = oracle.decompose(L, flags=oracle.SPLIT_BUDGET, budget=B, nthreads=4)
    assert r.n_budget_components > 0
    conf = list(zip(L.conf_u.tolist(), L.conf_v.tolist()))
    st = list(zip(L.st_u.tolist(), L.st_v.tolist()))
    for c in range(r.n_components):
        seg = np.flatnonzero(r.comp_of == c)
        loc = {int(g): i for i, g in enumerate(seg)}
        cc = [(loc[a], loc[b]) for a, b in conf if a in loc and b in loc]
        ss = [(loc[a], loc[b]) for a, b in st if a in loc and b in loc]
        one = oracle.solve_instance(len(seg), k, cc, ss, budget=B, split=True)
        assert (one.cost, one.nodes) == (r.comp_cost[c], r.comp_nodes[c])
        assert np.array_equal(one.x, r.mask[seg])
    conf_n = sum(1 for a, b in conf if r.mask[a] == r.mask[b])
    st_n = sum(1 for a, b in st if r.mask[a] != r.mask[b])
    assert r.cost == 10 * conf_n + st_n


@pytest.mark.parametrize("n", [4096, 4097, 6000])
def test_instances_above_the_limit_are_not_split(n):
    # a ring at k = 2 with triangle chords (each forces a conflict), big
    # enough that the budget stops the search
    conf = [(i, (i + 1) % n) for i in range(n)] + [(i, i + 2) for i in range(0, n - 2, 97)]
    B = 3 * n
    split = oracle.solve_instance(n, 2, conf, budget=B, split=True)
    plain = oracle.solve_instance(n, 2, conf, budget=B)
    if n > 4096:
        assert (split.cost, split.nodes, split.x.tolist()) == (plain.cost, plain.nodes,
                                                               plain.x.tolist())
    else:
        # at the limit the instance is still split: the first search has a
        # share of the budget only
        D, S = split_cut(n, 2)
        first = oracle.solve_instance(n, 2, conf, budget=(B + S) // (S + 1))
        assert first.status == oracle.BUDGET and split.nodes > first.nodes
