"""Pins for the oracle's second bound mode (`oracle.CLIQUE_BOUND`).

Checked against things other than the oracle itself:
- the clique list equals a brute-force restatement (every (k+1)-subset in
  itertools order, taken when it is a clique sharing no edge with one taken
  before);
- node counts, assignments and costs equal an independent recursive search
  over the partial assignment with the same bound (tests/graph_dfs.py);
- an admissible bound cannot change the answer of an exhaustive search:
  the result equals the first minimum-cost leaf of the default search and
  the brute-force optimum, with no more nodes.
"""
import itertools

import numpy as np
import pytest

import oracle
from graph_dfs import bounded_search, brute_force, greedy_cliques
from paper_2303_14335_gb300 import synth


def edges(L):
    return list(zip(L.conf_u.tolist(), L.conf_v.tolist())), list(zip(L.st_u.tolist(), L.st_v.tolist()))


def cases(count, nmax, salt):
    out = []
    for s in range(count):
        d = synth.uniform(salt, np.arange(4 * s, 4 * s + 4, dtype=np.uint64))
        n = 4 + int(d[0] * (nmax - 3))
        k = 2 + int(d[1] * 3)
        out.append((n, k, 0.35 + 0.5 * d[2], int(d[3] * 3), salt + s))
    return out


@pytest.mark.parametrize("n,k,p,ns,seed", cases(40, 14, 6100))
def test_clique_list_is_the_greedy_lexicographic_packing(n, k, p, ns, seed):
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=ns)
    conf, _ = edges(L)
    assert oracle.cliques(n, k, conf) == greedy_cliques(n, k, conf)


def test_clique_list_small_fixtures():
    k4 = [(a, b) for a, b in itertools.combinations(range(4), 2)]
    assert oracle.cliques(4, 3, k4) == [[0, 1, 2, 3]]
    # two K4 sharing the edge (2,3): the second is not taken
    two = k4 + [(2, 4), (3, 4), (2, 5), (3, 5), (4, 5)]
    assert oracle.cliques(6, 3, two) == [[0, 1, 2, 3]]
    # k = 2: edge-disjoint triangles of K5 taken greedily
    k5 = [(a, b) for a, b in itertools.combinations(range(5), 2)]
    assert oracle.cliques(5, 2, k5) == [[0, 1, 2], [0, 3, 4]]


@pytest.mark.parametrize("n,k,p,ns,seed", cases(50, 10, 6300))
def test_clique_bound_search_matches_independent_search(n, k, p, ns, seed):
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=ns)
    conf, st = edges(L)
    for budget in (0, 7, 60):
        r = oracle.solve_instance(n, k, conf, st, budget=budget, clique_bound=True)
        c, x, nodes, hit = bounded_search(n, k, conf, st, budget=budget, clique_bound=True)
        assert (r.cost, r.x.tolist(), r.nodes) == (c, x, nodes)
        assert (r.status == oracle.BUDGET) == hit


@pytest.mark.parametrize("n,k,p,ns,seed", cases(50, 10, 6500))
def test_clique_bound_keeps_the_exhaustive_answer(n, k, p, ns, seed):
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=ns)
    conf, st = edges(L)
    a = oracle.solve_instance(n, k, conf, st)
    b = oracle.solve_instance(n, k, conf, st, clique_bound=True)
    assert (b.cost, b.x.tolist()) == (a.cost, a.x.tolist())
    assert b.nodes <= a.nodes
    if k ** n <= 300_000:
        assert b.cost == brute_force(n, k, conf, st)[0]


def test_clique_bound_in_the_flow():
    L = synth.unit_disk_layout(3000, 3, seed=44, mean_deg=4.5, p_stitch=0.2)
    conf, st = edges(L)
    r = oracle.decompose(L, flags=oracle.CLIQUE_BOUND, budget=4000, nthreads=4)
    d = oracle.decompose(L, budget=4000, nthreads=4)
    assert r.nodes < d.nodes
    assert r.component_cost_sum == r.cost
    for c in range(0, r.n_components, 37):
        segs = np.nonzero(r.comp_of == c)[0]
        loc = {int(s): i for i, s in enumerate(segs)}
        cc = [(loc[a], loc[b]) for a, b in conf if a in loc and b in loc]
        ss = [(loc[a], loc[b]) for a, b in st if a in loc and b in loc]
        s = oracle.solve_instance(len(segs), 3, cc, ss, budget=4000, clique_bound=True)
        assert s.cost == r.comp_cost[c] and s.nodes == r.comp_nodes[c]
        assert np.array_equal(s.x, r.mask[segs])
