"""Pins of the oracle's density-balance option (DENSITY_BALANCE).

Renaming the masks of one component keeps its cost, and a removed unit
recovered with any mask its coloured conflict neighbours leave free costs
nothing, so the option changes only which mask each segment gets.  Checked
against the rule written out over the plain decomposition (instances in
order, the greedy pairing of counts, the peel's removal order restated in
tests/graph_dfs.py), and against the invariants: the same cost, conflict
and stitch counts as without the option, each instance's masks a permutation
of its plain ones, and mask usage no less balanced.
"""
import numpy as np
import pytest

import oracle
from graph_dfs import density_balanced, peel_order, units_of
from paper_2303_14335_gb300 import synth


def edges(L):
    return list(zip(L.conf_u.tolist(), L.conf_v.tolist())), list(zip(L.st_u.tolist(), L.st_v.tolist()))


@pytest.mark.parametrize("n,k,deg,ps,seed", [
    (3000, 3, 3.0, 0.2, 2), (2000, 4, 5.0, 0.3, 3), (1500, 3, 2.4, 0.0, 5), (800, 2, 2.0, 0.3, 7),
    (1200, 5, 6.0, 0.2, 9)])
def test_balance_matches_the_rule_written_out(n, k, deg, ps, seed):
    L = synth.unit_disk_layout(n, k, seed=seed, mean_deg=deg, p_stitch=ps)
    plain = oracle.decompose(L, budget=3000, nthreads=4)
    bal = oracle.decompose(L, flags=oracle.DENSITY_BALANCE, budget=3000, nthreads=4)
    conf, st = edges(L)
    inst = np.where(plain.comp_of >= 0, plain.mask, -1)
    want = density_balanced(L.n_seg, k, conf, st, L.polygon_of, plain.comp_of.tolist(),
                            inst.tolist())
    assert bal.mask.tolist() == want
    # invariants
    assert (bal.cost, bal.n_conflicts, bal.n_stitches, bal.nodes) == \
        (plain.cost, plain.n_conflicts, plain.n_stitches, plain.nodes)
    assert np.array_equal(bal.comp_of, plain.comp_of)
    for c in range(plain.n_components):
        seg = plain.comp_of == c
        pairs = set(zip(plain.mask[seg].tolist(), bal.mask[seg].tolist()))
        assert len(pairs) == len({a for a, _ in pairs}) == len({b for _, b in pairs})
    cp, cb = np.bincount(plain.mask, minlength=k), np.bincount(bal.mask, minlength=k)
    assert cb.max() - cb.min() <= cp.max() - cp.min()


def test_peel_order_restatement_matches_the_removed_segments():
    L = synth.unit_disk_layout(3000, 3, seed=2, mean_deg=3.0, p_stitch=0.2)
    plain = oracle.decompose(L, budget=100, nthreads=4)
    conf, st = edges(L)
    unit = units_of(L.n_seg, L.polygon_of, st)
    order = peel_order(L.n_seg, 3, conf, unit)
    removed = {s for s in range(L.n_seg) if unit[s] in set(order)}
    assert removed == set(np.flatnonzero(plain.comp_of < 0).tolist())
    assert len(removed) == plain.n_removed_segments


def test_balance_refused_with_blocks():
    L = synth.unit_disk_layout(500, 3, seed=2, mean_deg=3.0, p_stitch=0.2)
    with pytest.raises(ValueError):
        oracle.decompose(L, flags=oracle.DENSITY_BALANCE | oracle.BICONNECTED)
