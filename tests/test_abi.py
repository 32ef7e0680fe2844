"""libmpld without a GPU: exported symbols and the host half of the flow.

The host-only build (MPLD_HOST_ONLY) runs the simplification, the sub-graph
split and the EC packing without touching the device, so they can be
checked here against the oracle's independent implementation.
"""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2303_14335_gb300 import mpld, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mpld.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpld_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["mpld_build_matrix", "mpld_solve", "mpld_solve_batch", "mpld_free"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = mpld.library()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_has_the_same_names():
    for name in declared_functions():
        assert callable(getattr(mpld, name)), name


def test_status_strings():
    assert mpld.mpld_status_string(0) == "ok"
    assert "too large" in mpld.mpld_status_string(mpld.MPLD_E_TOO_LARGE)


def host_only(layout, flags=0):
    return mpld.mpld_build_matrix(layout, mpld.make_params(flags=flags | mpld.MPLD_HOST_ONLY))


def edges(L):
    return list(zip(L.conf_u.tolist(), L.conf_v.tolist())), list(zip(L.st_u.tolist(), L.st_v.tolist()))


@pytest.mark.parametrize("k,deg,p,seed", [(3, 3.0, 0.2, 1), (4, 5.0, 0.3, 2), (3, 4.5, 0.25, 3),
                                          (5, 6.0, 0.1, 4), (2, 2.5, 0.2, 5)])
def test_host_split_matches_oracle(k, deg, p, seed):
    L = synth.unit_disk_layout(4000, k, seed=seed, mean_deg=deg, p_stitch=p)
    prob = host_only(L)
    info = mpld.mpld_problem_info(prob)
    _, _, _, comp_of = mpld.mpld_component_results(prob, results=False)
    ref = oracle.decompose(L, budget=50, nthreads=4)
    assert info.n_components == ref.n_components
    assert info.n_removed_segments == ref.n_removed_segments
    assert info.max_component == ref.max_component
    assert np.array_equal(comp_of, ref.comp_of)


@pytest.mark.parametrize("k,deg,p,seed", [(3, 3.0, 0.2, 1), (4, 5.0, 0.3, 2), (3, 4.5, 0.25, 3),
                                          (2, 2.5, 0.2, 5)])
def test_host_block_split_matches_oracle(k, deg, p, seed):
    # biconnected blocks as search instances: same count, order and sizes
    L = synth.unit_disk_layout(4000, k, seed=seed, mean_deg=deg, p_stitch=p)
    prob = host_only(L, mpld.MPLD_BICONNECTED)
    info = mpld.mpld_problem_info(prob)
    _, _, _, comp_of = mpld.mpld_component_results(prob, results=False)
    ref = oracle.decompose(L, flags=oracle.BICONNECTED, budget=50, nthreads=4)
    assert info.n_components == ref.n_components
    assert info.max_component == ref.max_component
    assert np.array_equal(comp_of, ref.comp_of)
    # each packed block is the EC matrix of that block's sub-graph
    keep = sorted(int(s) for s in np.nonzero(ref.comp_of >= 0)[0])
    conf, st = edges(L)
    sub = set(keep)
    loc = {s: i for i, s in enumerate(keep)}
    blocks = oracle.blocks(len(keep), [(loc[a], loc[b]) for a, b in conf if a in sub and b in sub],
                           [(loc[a], loc[b]) for a, b in st if a in sub and b in sub])
    assert len(blocks) == info.n_components
    for c in range(0, len(blocks), 11):
        g = [keep[v] for v in blocks[c][0]]
        lb = {s: j for j, s in enumerate(g)}
        cc = [(lb[a], lb[b]) for a, b in conf if a in lb and b in lb]
        assert np.array_equal(mpld.mpld_export_matrix(prob, c), oracle.export_matrix(len(g), k, cc))


def test_block_split_with_single_instance_rejected():
    with pytest.raises(mpld.MpldError) as e:
        host_only(synth.graph_from_edges(3, 3, [(0, 1)]),
                  mpld.MPLD_BICONNECTED | mpld.MPLD_SINGLE_INSTANCE)
    assert e.value.code == mpld.MPLD_E_INVALID


def test_host_single_instance_mode():
    L, mode = synth.workload("k3_n400_p025_plain")
    prob = host_only(L, mpld.MPLD_NO_SIMPLIFY | mpld.MPLD_SINGLE_INSTANCE)
    info = mpld.mpld_problem_info(prob)
    assert info.n_components == 1 and info.max_component == L.n_seg and info.n_removed_segments == 0


@pytest.mark.parametrize("seed", range(6))
def test_packed_matrix_is_the_ec_matrix(seed):
    # the packed block-sparse columns decode to exactly the oracle's DLX matrix
    L = synth.random_graph(9, 3 + seed % 3, seed=60 + seed, p_edge=0.45, n_stitch=2)
    prob = host_only(L, mpld.MPLD_NO_SIMPLIFY | mpld.MPLD_SINGLE_INSTANCE)
    conf, _ = edges(L)
    M = mpld.mpld_export_matrix(prob, 0)
    R = oracle.export_matrix(L.n_seg, L.k, conf)
    assert np.array_equal(M, R)


def test_packed_matrices_of_components():
    L = synth.unit_disk_layout(3000, 3, seed=17, mean_deg=3.0, p_stitch=0.2)
    prob = host_only(L)
    _, _, _, comp_of = mpld.mpld_component_results(prob, results=False)
    conf, _ = edges(L)
    for c in range(0, int(comp_of.max()) + 1, 7):
        segs = np.nonzero(comp_of == c)[0]
        loc = {int(s): i for i, s in enumerate(segs)}
        cc = [(loc[a], loc[b]) for a, b in conf if a in loc and b in loc]
        assert np.array_equal(mpld.mpld_export_matrix(prob, c), oracle.export_matrix(len(segs), 3, cc))


@pytest.mark.parametrize("seed", [1, 2])
def test_edge_order_and_duplicates_do_not_matter(seed):
    # sorted input takes a copy-only path; shuffled, reversed and repeated
    # edges go through the bucket sort: the built problems are the same
    import dataclasses
    L = synth.unit_disk_layout(3000, 3, seed=seed, mean_deg=3.5, p_stitch=0.3)
    rng = np.random.default_rng(seed)

    def scramble(u, v):
        u, v = u.copy(), v.copy()
        flip = rng.random(len(u)) < 0.5
        u[flip], v[flip] = v[flip].copy(), u[flip].copy()
        dup = rng.random(len(u)) < 0.1
        u, v = np.concatenate([u, v[dup]]), np.concatenate([v, u[dup]])
        perm = rng.permutation(len(u))
        return u[perm].astype(np.int32), v[perm].astype(np.int32)

    cu, cv = scramble(L.conf_u, L.conf_v)
    su, sv = scramble(L.st_u, L.st_v)
    M = dataclasses.replace(L, conf_u=cu, conf_v=cv, st_u=su, st_v=sv)
    a, b = host_only(L), host_only(M)
    ia, ib = mpld.mpld_problem_info(a), mpld.mpld_problem_info(b)
    assert (ia.n_components, ia.arena_bytes, ia.instance_segments) == \
        (ib.n_components, ib.arena_bytes, ib.instance_segments)
    assert np.array_equal(mpld.mpld_component_results(a, results=False)[3],
                          mpld.mpld_component_results(b, results=False)[3])
    for c in range(0, ia.n_components, max(1, ia.n_components // 25)):
        assert np.array_equal(mpld.mpld_export_matrix(a, c), mpld.mpld_export_matrix(b, c))
    a.close()
    b.close()


def test_invalid_inputs_rejected():
    bad = [synth.graph_from_edges(3, 3, [(0, 1)]), synth.graph_from_edges(3, 3, [(0, 1)])]
    bad[0].conf_v = np.array([0], dtype=np.int32)          # self-loop
    bad[1].conf_v = np.array([7], dtype=np.int32)          # out of range
    for L in bad:
        with pytest.raises(mpld.MpldError) as e:
            host_only(L)
        assert e.value.code == mpld.MPLD_E_INVALID
    for k in (1, 9):
        with pytest.raises(mpld.MpldError):
            host_only(synth.graph_from_edges(3, k, [(0, 1)]))
    L = synth.graph_from_edges(3, 3, [(0, 1)], cost_conflict=20000)
    with pytest.raises(mpld.MpldError):
        host_only(L)
    L = synth.graph_from_edges(3, 3, [(0, 1)], polygon_of=[0, 5, 1])
    with pytest.raises(mpld.MpldError):
        host_only(L)


def test_noalloc_entry_rejects_the_column_rule_before_any_device_work():
    # the allocation-free entry has no breadth-first ranks: the flag is an
    # argument error, reported before a pointer is followed or a device used
    prm = mpld.make_params(flags=mpld.MPLD_COLUMN_BFS)
    with pytest.raises(mpld.MpldError) as e:
        mpld.mpld_search_instance_noalloc(4, 3, 256, 512, 0, 768, 1024, 0, 1280, 1536, prm)
    assert e.value.code == mpld.MPLD_E_INVALID


def test_noalloc_entry_rejects_the_split_search():
    prm = mpld.make_params(flags=mpld.MPLD_PARALLEL_EXACT)
    with pytest.raises(mpld.MpldError) as e:
        mpld.mpld_search_instance_noalloc(4, 3, 256, 512, 0, 768, 1024, 0, 1280, 1536, prm)
    assert e.value.code == mpld.MPLD_E_INVALID


def test_split_search_needs_exact_mode():
    # the split search takes no node budget: an argument error before the
    # handle's state is looked at; without a budget the host-only handle
    # is the state error it always is
    prob = host_only(synth.graph_from_edges(3, 3, [(0, 1), (1, 2), (0, 2)]))
    for call in (lambda prm: mpld.mpld_solve(prob, prm),
                 lambda prm: mpld.mpld_solve_batch([prob, prob], prm),
                 lambda prm: mpld.mpld_search_batch_async([prob], prm)):
        with pytest.raises(mpld.MpldError) as e:
            call(mpld.make_params(node_budget=100, flags=mpld.MPLD_PARALLEL_EXACT))
        assert e.value.code == mpld.MPLD_E_INVALID
        with pytest.raises(mpld.MpldError) as e:
            call(mpld.make_params(flags=mpld.MPLD_PARALLEL_EXACT))
        assert e.value.code == mpld.MPLD_E_STATE


def test_too_large_instance_rejected():
    n = 70000
    L = synth.graph_from_edges(n, 3, [(i, i + 1) for i in range(n - 1)])
    with pytest.raises(mpld.MpldError) as e:
        host_only(L, mpld.MPLD_NO_SIMPLIFY)
    assert e.value.code == mpld.MPLD_E_TOO_LARGE


def test_solve_on_host_only_handle_is_a_state_error():
    prob = host_only(synth.graph_from_edges(3, 3, [(0, 1), (1, 2), (0, 2)]))
    with pytest.raises(mpld.MpldError) as e:
        mpld.mpld_solve(prob)
    assert e.value.code == mpld.MPLD_E_STATE
    with pytest.raises(mpld.MpldError) as e:
        mpld.mpld_fetch(prob)
    assert e.value.code == mpld.MPLD_E_STATE


def test_empty_layout():
    prob = host_only(synth.graph_from_edges(0, 3, []))
    assert mpld.mpld_problem_info(prob).n_components == 0


def test_builds_are_identical_alone_and_concurrent():
    # the host build uses a shared thread pool (parallel union-find, packing);
    # builds on several threads at once take the inline path: every build
    # must give the same instances, ids and packed matrices
    import threading
    L = synth.unit_disk_layout(20000, 3, seed=8, mean_deg=3.0, p_stitch=0.2)

    def digest(prob):
        info = mpld.mpld_problem_info(prob)
        comp_of = mpld.mpld_component_results(prob, results=False)[3]
        mats = [mpld.mpld_export_matrix(prob, c).tobytes()
                for c in range(0, info.n_components, max(1, info.n_components // 20))]
        return (info.n_components, info.arena_bytes, info.instance_segments,
                comp_of.tobytes(), tuple(mats))

    first = host_only(L)
    ref = digest(first)
    first.close()
    for _ in range(2):
        p = host_only(L)
        assert digest(p) == ref
        p.close()
    out, errs = [None] * 4, []

    def worker(i):
        try:
            p = host_only(L)
            out[i] = digest(p)
            p.close()
        except Exception as e:  # surfaced below
            errs.append(e)

    ts = [threading.Thread(target=worker, args=(i,)) for i in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs
    assert all(o == ref for o in out)


def test_instance_ids_are_valid_on_every_pooled_build():
    # the components' union-find runs on the host pool; its last pass stores
    # every segment's root.  Over repeated builds of a layout that keeps a
    # 12,000-segment component: every kept segment has an instance id, the
    # ids follow the instances' lowest segments, and the sizes agree
    L = synth.serving_request(2023, 9)
    ref = None
    for _ in range(12):
        p = host_only(L)
        info = mpld.mpld_problem_info(p)
        comp_of = mpld.mpld_component_results(p, results=False)[3]
        sizes = mpld.mpld_instance_sizes(p)
        p.close()
        C = info.n_components
        kept = comp_of >= 0
        assert np.all(comp_of < C)
        assert int(kept.sum()) == info.instance_segments == L.n_seg - info.n_removed_segments
        assert np.array_equal(np.bincount(comp_of[kept], minlength=C), sizes)
        first = np.full(C, L.n_seg)
        np.minimum.at(first, comp_of[kept], np.flatnonzero(kept))
        assert np.all(np.diff(first) > 0)
        if ref is None:
            ref = comp_of.copy()
        assert np.array_equal(comp_of, ref)


def test_density_balance_finish_on_the_host_matches_the_oracle():
    # host-only handle: the oracle's per-instance results go through the
    # library's own finish (scatter, balance, recovery, counts)
    import oracle
    for n, k, deg, ps, seed in ((3000, 3, 3.0, 0.2, 2), (1500, 4, 5.0, 0.3, 3), (1200, 5, 6.0, 0.2, 9)):
        L = synth.unit_disk_layout(n, k, seed=seed, mean_deg=deg, p_stitch=ps)
        plain = oracle.decompose(L, budget=3000, nthreads=4)
        want = oracle.decompose(L, flags=oracle.DENSITY_BALANCE, budget=3000, nthreads=4)
        prob = mpld.mpld_build_matrix(L, mpld.make_params(flags=mpld.MPLD_HOST_ONLY |
                                                          mpld.MPLD_DENSITY_BALANCE))
        try:
            _, _, _, comp_of = mpld.mpld_component_results(prob, results=False)
            assert np.array_equal(comp_of, plain.comp_of)
            sizes = mpld.mpld_instance_sizes(prob)
            masks = np.concatenate([plain.mask[comp_of == c] for c in range(len(sizes))] or
                                   [np.zeros(0, np.int8)])
            status = np.where(plain.comp_status == oracle.BUDGET, mpld.MPLD_BUDGET, mpld.MPLD_OK)
            rc, mask, res = mpld.mpld_finish_from(prob, plain.comp_nodes, plain.comp_cost, status,
                                                  masks)
        finally:
            prob.close()
        assert np.array_equal(mask, want.mask)
        assert (res.cost, res.n_conflicts, res.n_stitches) == (want.cost, want.n_conflicts,
                                                               want.n_stitches)


def test_density_balance_refused_with_blocks():
    L = synth.unit_disk_layout(500, 3, seed=2, mean_deg=3.0, p_stitch=0.2)
    with pytest.raises(mpld.MpldError) as e:
        mpld.mpld_build_matrix(L, mpld.make_params(flags=mpld.MPLD_HOST_ONLY | mpld.MPLD_BICONNECTED |
                                                   mpld.MPLD_DENSITY_BALANCE))
    assert e.value.code == mpld.MPLD_E_INVALID
