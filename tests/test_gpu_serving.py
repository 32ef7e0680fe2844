"""Serving loop: continuous batching of whole layouts (one batched launch per layout, streams).

Each request's result in the mix must equal its result alone (batched path,
same node budget) and the oracle's, bit for bit: masks, cost, node count.
"""
import os
import time

import numpy as np
import pytest

import oracle
from paper_2303_14335_gb300 import mpld, synth

pytestmark = pytest.mark.gpu

BUDGET = 3000
NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def requests(n, seed=77, n_max=20000):
    return [synth.serving_request(seed, i, n_min=500, n_max=n_max) for i in range(n)]


def alone(L, stream):
    prob = mpld.mpld_build_matrix(L, None, stream)
    rc, masks, res = mpld.mpld_solve_batch([prob], mpld.make_params(node_budget=BUDGET), stream)
    prob.close()
    return rc, masks[0], res[0]


def drain(server, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in mpld.mpld_server_poll(server):
            out[t] = mpld.mpld_server_result(server, t)
        if time.time() - t0 > timeout:
            st = mpld.mpld_server_stats_get(server).as_dict()
            raise TimeoutError(f"{len(out)}/{len(tickets)} requests finished; {st}")
        time.sleep(0.0005)
    return out


def test_mix_equals_alone_and_oracle(torch_cuda):
    stream = torch_cuda.cuda.Stream().cuda_stream
    Ls = requests(14)
    cfg = mpld.mpld_server_config(arena_bytes=6 << 20)   # forces waiting for device bytes
    with mpld.mpld_server_create(cfg, mpld.make_params(node_budget=BUDGET)) as srv:
        tickets = [mpld.mpld_server_submit(srv, L) for L in Ls]
        got = drain(srv, tickets)
        st = mpld.mpld_server_stats_get(srv)
    assert st.completed == len(Ls) and st.failed == 0
    assert st.arena_peak_bytes <= 6 << 20 and st.max_concurrent >= 2
    for t, L in zip(tickets, Ls):
        rc, mask, res = got[t]
        rc1, mask1, res1 = alone(L, stream)
        assert rc == rc1 and np.array_equal(mask, mask1)
        assert (res.cost, res.nodes, res.n_conflicts, res.n_stitches) == \
            (res1.cost, res1.nodes, res1.n_conflicts, res1.n_stitches)
    for t, L in list(zip(tickets, Ls))[:5]:
        ref = oracle.decompose(L, budget=BUDGET, nthreads=NTHREADS)
        rc, mask, res = got[t]
        assert np.array_equal(mask, ref.mask) and res.nodes == ref.nodes and res.cost == ref.cost


def test_staggered_arrivals_overlap(torch_cuda):
    stream = torch_cuda.cuda.Stream().cuda_stream
    Ls = requests(10, seed=78)
    with mpld.mpld_server_create(None, mpld.make_params(node_budget=BUDGET)) as srv:
        tickets, got = [], {}
        for L in Ls:                 # submit while earlier requests are in flight
            tickets.append(mpld.mpld_server_submit(srv, L))
            for t in mpld.mpld_server_poll(srv):
                got[t] = mpld.mpld_server_result(srv, t)
            time.sleep(0.002)
        rest = [t for t in tickets if t not in got]
        got.update(drain(srv, rest))
    for t, L in zip(tickets, Ls):
        rc, mask, res = got[t]
        rc1, mask1, res1 = alone(L, stream)
        assert np.array_equal(mask, mask1) and res.nodes == res1.nodes


def test_bad_and_oversized_requests_fail_alone(torch_cuda):
    good = requests(3, seed=79)
    bad = synth.graph_from_edges(4, 3, [(0, 1), (1, 2)])
    bad.conf_v = np.array([0, 2], dtype=np.int32)          # self-loop (0, 0)
    big = synth.unit_disk_layout(60000, 3, seed=5, mean_deg=4.5, p_stitch=0.2)
    cfg = mpld.mpld_server_config(arena_bytes=1 << 20)
    with mpld.mpld_server_create(cfg, mpld.make_params(node_budget=BUDGET)) as srv:
        tb = mpld.mpld_server_submit(srv, bad)
        tg = [mpld.mpld_server_submit(srv, L) for L in good]
        tl = mpld.mpld_server_submit(srv, big)
        got = drain(srv, [tb, tl] + tg)
    assert got[tb][0] == mpld.MPLD_E_INVALID
    assert got[tl][0] == mpld.MPLD_E_TOO_LARGE
    for t in tg:
        assert got[t][0] >= 0


def test_in_flight_limit_and_reuse(torch_cuda):
    stream = torch_cuda.cuda.Stream().cuda_stream
    Ls = requests(6, seed=80)
    cfg = mpld.mpld_server_config(max_in_flight=1, streams=2)
    with mpld.mpld_server_create(cfg, mpld.make_params(node_budget=BUDGET)) as srv:
        tickets = [mpld.mpld_server_submit(srv, L) for L in Ls]
        got = drain(srv, tickets)
        st = mpld.mpld_server_stats_get(srv)
    assert st.max_concurrent == 1 and st.completed == 6 and st.kernel_launches <= 6
    for t, L in zip(tickets, Ls):
        rc1, mask1, res1 = alone(L, stream)
        assert np.array_equal(got[t][1], mask1) and got[t][2].nodes == res1.nodes


def test_empty_and_fully_simplified_requests(torch_cuda):
    with mpld.mpld_server_create(None, mpld.make_params(node_budget=BUDGET)) as srv:
        t0 = mpld.mpld_server_submit(srv, synth.graph_from_edges(0, 3, []))
        t1 = mpld.mpld_server_submit(srv, synth.graph_from_edges(6, 3, [(0, 1), (2, 3)]))
        got = drain(srv, [t0, t1])
    assert got[t0][0] == 0 and got[t0][2].n_components == 0
    rc, mask, res = got[t1]
    assert rc == 0 and res.cost == 0 and res.n_removed_segments == 6 and np.all(mask >= 0)


def test_column_rule_flag_reaches_served_searches(torch_cuda):
    # a server created with the paper's column rule searches every request
    # with it: results equal the oracle's under the same rule
    Ls = requests(4, seed=81, n_max=8000)
    prm = mpld.make_params(node_budget=BUDGET, flags=mpld.MPLD_COLUMN_BFS)
    with mpld.mpld_server_create(None, prm) as srv:
        tickets = [mpld.mpld_server_submit(srv, L) for L in Ls]
        got = drain(srv, tickets)
    for t, L in zip(tickets, Ls):
        ref = oracle.decompose(L, flags=oracle.COLUMN_BFS, budget=BUDGET, nthreads=NTHREADS)
        rc, mask, res = got[t]
        assert np.array_equal(mask, ref.mask) and res.nodes == ref.nodes and res.cost == ref.cost


def test_block_split_requests(torch_cuda):
    # requests built with the biconnected split: results equal the oracle's
    Ls = requests(4, seed=83, n_max=8000)
    with mpld.mpld_server_create(None, mpld.make_params(node_budget=BUDGET)) as srv:
        tickets = [mpld.mpld_server_submit(srv, L, flags=mpld.MPLD_BICONNECTED) for L in Ls]
        got = drain(srv, tickets)
    for t, L in zip(tickets, Ls):
        ref = oracle.decompose(L, flags=oracle.BICONNECTED, budget=BUDGET, nthreads=NTHREADS)
        rc, mask, res = got[t]
        assert np.array_equal(mask, ref.mask) and res.nodes == ref.nodes and res.cost == ref.cost


def test_cta_team_threshold_reaches_served_searches(torch_cuda):
    # a server whose instances of 30+ segments go to whole-CTA teams
    Ls = requests(4, seed=85, n_max=8000)
    prm = mpld.make_params(node_budget=BUDGET, cta_segments=30)
    with mpld.mpld_server_create(None, prm) as srv:
        tickets = [mpld.mpld_server_submit(srv, L) for L in Ls]
        got = drain(srv, tickets)
    for t, L in zip(tickets, Ls):
        ref = oracle.decompose(L, budget=BUDGET, nthreads=NTHREADS)
        rc, mask, res = got[t]
        assert np.array_equal(mask, ref.mask) and res.nodes == ref.nodes and res.cost == ref.cost


def test_split_budget_served(torch_cuda):
    # a server with the budgeted split search: each layout's result equals
    # mpld_solve_batch's with the same flag and the oracle's split mode, in a
    # mix with a small arena (layouts wait for device bytes)
    stream = torch_cuda.cuda.Stream().cuda_stream
    Ls = requests(10, seed=91)
    prm = mpld.make_params(node_budget=BUDGET, flags=mpld.MPLD_SPLIT_BUDGET)
    cfg = mpld.mpld_server_config(arena_bytes=96 << 20)
    with mpld.mpld_server_create(cfg, prm) as srv:
        tickets = [mpld.mpld_server_submit(srv, L) for L in Ls]
        got = drain(srv, tickets)
        with pytest.raises(mpld.MpldError) as e:
            mpld.mpld_server_submit(srv, Ls[0], flags=mpld.MPLD_CLIQUE_BOUND)
        assert e.value.code == mpld.MPLD_E_INVALID
    for t, L in zip(tickets, Ls):
        rc, mask, res = got[t]
        prob = mpld.mpld_build_matrix(L, None, stream)
        rc2, masks2, res2 = mpld.mpld_solve_batch([prob], prm, stream)
        prob.close()
        ref = oracle.decompose(L, flags=oracle.SPLIT_BUDGET, budget=BUDGET, nthreads=NTHREADS)
        assert rc == rc2 and np.array_equal(mask, masks2[0]) and np.array_equal(mask, ref.mask)
        assert res.cost == res2[0].cost == ref.cost and res.nodes == res2[0].nodes == ref.nodes


def test_density_balance_served(torch_cuda):
    Ls = requests(6, seed=93)
    with mpld.mpld_server_create(None, mpld.make_params(node_budget=BUDGET)) as srv:
        tickets = [mpld.mpld_server_submit(srv, L, flags=mpld.MPLD_DENSITY_BALANCE) for L in Ls]
        got = drain(srv, tickets)
    for t, L in zip(tickets, Ls):
        rc, mask, res = got[t]
        ref = oracle.decompose(L, flags=oracle.DENSITY_BALANCE, budget=BUDGET, nthreads=NTHREADS)
        assert np.array_equal(mask, ref.mask) and res.cost == ref.cost and res.nodes == ref.nodes


def test_destroy_with_requests_in_every_state(torch_cuda):
    # a server destroyed while its layouts are queued, being built, on the
    # device and waiting to be finished frees each of them once; a server
    # created afterwards serves as before
    Ls = requests(12, seed=91, n_max=60000)
    for polls in (0, 3, 40):
        srv = mpld.mpld_server_create(
            mpld.mpld_server_config(max_in_flight=4, streams=2, worker_threads=2),
            mpld.make_params(node_budget=BUDGET, flags=mpld.MPLD_SPLIT_BUDGET))
        for L in Ls:
            mpld.mpld_server_submit(srv, L)
        for _ in range(polls):
            mpld.mpld_server_poll(srv)
            time.sleep(0.002)
        srv.close()
    with mpld.mpld_server_create(None, mpld.make_params(node_budget=BUDGET)) as srv:
        tickets = [mpld.mpld_server_submit(srv, L) for L in Ls[:3]]
        got = drain(srv, tickets)
    for t, L in zip(tickets, Ls[:3]):
        rc, mask, res = got[t]
        ref = oracle.decompose(L, budget=BUDGET, nthreads=NTHREADS)
        assert np.array_equal(mask, ref.mask) and res.cost == ref.cost
