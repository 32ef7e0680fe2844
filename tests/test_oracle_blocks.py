"""Pins for the oracle's biconnected-block split of the flow (`oracle.BICONNECTED`).

The split is checked against things other than the oracle itself:
- the blocks equal networkx's biconnected components (a library routine on
  the same graph), with lone segments as blocks of one;
- their order and attach segments equal an independent restatement, in
  Python, of the canonical breadth-first walk of the block-cut tree;
- with an exhaustive search, the split flow reaches the brute-force optimum
  of Eq. 1: every edge lies in exactly one block and renaming masks inside
  a block keeps its cost, so optimal blocks merge into an optimal layout;
- the merged masks cost exactly the sum of the block costs, and a block's
  merged masks are its own solution up to one transposition.
"""
import numpy as np
import pytest

import oracle
from graph_dfs import brute_force, eq1_cost
from paper_2303_14335_gb300 import synth

nx = pytest.importorskip("networkx")


def edges(L):
    return list(zip(L.conf_u.tolist(), L.conf_v.tolist())), list(zip(L.st_u.tolist(), L.st_v.tolist()))


def canonical_blocks(n, conf, stitch):
    """Blocks from networkx, put in the canonical order: components by lowest
    segment; in each, breadth-first over the block-cut tree from the
    lexicographically first block holding the lowest segment, a visited
    block's segments in ascending id, the unvisited blocks at a segment in
    lexicographic order."""
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from(conf)
    G.add_edges_from(stitch)
    out = []
    for comp in sorted((sorted(c) for c in nx.connected_components(G)), key=lambda c: c[0]):
        H = G.subgraph(comp)
        bl = sorted(sorted(b) for b in nx.biconnected_components(H)) if H.number_of_edges() else [[comp[0]]]
        at = {}
        for i, b in enumerate(bl):
            for v in b:
                at.setdefault(v, []).append(i)
        seen = {at[comp[0]][0]}
        queue = [(at[comp[0]][0], -1)]
        h = 0
        while h < len(queue):
            b, _ = queue[h]
            h += 1
            for v in bl[b]:
                for j in at[v]:
                    if j not in seen:
                        seen.add(j)
                        queue.append((j, v))
        out += [(bl[b], a) for b, a in queue]
    return out


def graph_cases():
    out = []
    for s in range(40):
        d = synth.uniform(2718, np.arange(3 * s, 3 * s + 3, dtype=np.uint64))
        n = 2 + int(d[0] * 40)
        out.append((n, 0.02 + 0.25 * d[1], int(d[2] * 6), 4400 + s))
    return out


@pytest.mark.parametrize("n,p,ns,seed", graph_cases())
def test_blocks_are_networkx_blocks_in_canonical_order(n, p, ns, seed):
    L = synth.random_graph(n, 3, seed=seed, p_edge=p, n_stitch=ns)
    conf, st = edges(L)
    got = oracle.blocks(n, conf, st)
    assert got == canonical_blocks(n, conf, st)


def test_bowtie_and_bridges():
    # two triangles sharing segment 2, a bridge to a pendant path
    conf = [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (2, 4), (4, 5), (5, 6)]
    assert oracle.blocks(7, conf) == [([0, 1, 2], -1), ([2, 3, 4], 2), ([4, 5], 4), ([5, 6], 5)]
    # at k = 2 each triangle forces one conflict; the path costs nothing
    L = synth.graph_from_edges(7, 2, conf)
    r = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.BICONNECTED)
    assert r.cost == 20 and r.n_components == 4
    assert eq1_cost(r.mask, conf, [], cc=10) == 20


def small_cases():
    out = []
    for s in range(60):
        d = synth.uniform(3141, np.arange(4 * s, 4 * s + 4, dtype=np.uint64))
        n = 3 + int(d[0] * 9)
        k = 2 + int(d[1] * 3)
        while k ** n > 300_000:
            n -= 1
        out.append((n, k, 0.15 + 0.45 * d[2], int(d[3] * 3), 5100 + s))
    return out


@pytest.mark.parametrize("n,k,p,ns,seed", small_cases())
def test_split_flow_is_exact(n, k, p, ns, seed):
    L = synth.random_graph(n, k, seed=seed, p_edge=p, n_stitch=ns, identity_polygons=False)
    conf, st = edges(L)
    m, _ = brute_force(n, k, conf, st)
    for flags in (oracle.NO_SIMPLIFY | oracle.BICONNECTED, oracle.BICONNECTED):
        r = oracle.decompose(L, flags=flags)
        assert r.cost == m
        assert eq1_cost(r.mask, conf, st) == r.cost == r.component_cost_sum


@pytest.mark.parametrize("k,deg,p", [(3, 3.2, 0.2), (4, 5.0, 0.3), (3, 4.5, 0.1)])
def test_split_flow_invariants(k, deg, p):
    L = synth.unit_disk_layout(3000, k, seed=77, mean_deg=deg, p_stitch=p)
    conf, st = edges(L)
    budget = 3000
    r = oracle.decompose(L, flags=oracle.BICONNECTED, budget=budget, nthreads=4)
    assert np.all((r.mask >= 0) & (r.mask < k))
    assert eq1_cost(r.mask, conf, st) == r.cost == r.component_cost_sum
    # the instances are the blocks of what simplification leaves
    keep = np.nonzero(r.comp_of >= 0)[0]
    sub = {int(s) for s in keep}
    kc = [(a, b) for a, b in conf if a in sub and b in sub]
    ks = [(a, b) for a, b in st if a in sub and b in sub]
    loc = {s: i for i, s in enumerate(sorted(sub))}
    want = canonical_blocks(len(sub), [(loc[a], loc[b]) for a, b in kc], [(loc[a], loc[b]) for a, b in ks])
    assert r.n_components == len(want)
    segs = sorted(sub)
    first = {}
    for i, (b, _) in enumerate(want):
        for v in b:
            first.setdefault(segs[v], i)
    assert all(r.comp_of[s] == first[s] for s in segs)
    # a block's merged masks are its stand-alone solution up to one transposition
    for i, (b, _) in enumerate(want[:40]):
        g = [segs[v] for v in b]
        lb = {s: j for j, s in enumerate(g)}
        cc = [(lb[x], lb[y]) for x, y in kc if x in lb and y in lb]
        ss = [(lb[x], lb[y]) for x, y in ks if x in lb and y in lb]
        s = oracle.solve_instance(len(g), k, cc, ss, budget=budget)
        assert s.cost == r.comp_cost[i] and s.nodes == r.comp_nodes[i]
        mp = {}
        for x, y in zip(s.x.tolist(), r.mask[g].tolist()):
            assert mp.setdefault(x, y) == y          # a function of the block's mask
        assert len(set(mp.values())) == len(mp)      # one to one
        moved = {x: y for x, y in mp.items() if x != y}
        assert len(moved) <= 2
        if len(moved) == 2:
            (a, b), = [(x, y) for x, y in moved.items() if x < y] or [(None, None)]
            assert moved == {a: b, b: a}


def test_split_with_single_instance_is_rejected():
    L = synth.graph_from_edges(3, 3, [(0, 1)])
    with pytest.raises(ValueError):
        oracle.decompose(L, flags=oracle.SINGLE_INSTANCE | oracle.BICONNECTED)
