"""The allocation-free entry point, mpld_search_instance_noalloc.

It serves callers that may not allocate GPU memory themselves (for example
a plug-in inside an application whose caching allocator owns the device
memory, or a caller that cannot afford the synchronisation an allocation
can cause): they hand over device buffers for the instance and the
outputs, and the library works in a fixed array of its own.  These tests
check its output against the allocating entry point, mpld_solve, on the
same graph, and against the CPU oracle's search of the graph as one
instance: masks, cost, node count and status must be identical, on two
calls in a row.  The kernel checks the caller's CSR before it searches; an
edge listed from one end only is reported as invalid input.  This file is
collected last so that a run that stops at the first failure has already run
every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2303_14335_gb300 import mpld, synth

pytestmark = pytest.mark.gpu

SINGLE = mpld.MPLD_NO_SIMPLIFY | mpld.MPLD_SINGLE_INSTANCE


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def csr(n, u, v):
    """Both directions of every edge, neighbours ascending."""
    a = np.concatenate([u, v]).astype(np.int64)
    b = np.concatenate([v, u]).astype(np.int64)
    order = np.lexsort((b, a))
    a, b = a[order], b[order]
    ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(ptr, a + 1, 1)
    return np.cumsum(ptr).astype(np.int32), b.astype(np.int32)


def split_status(word):
    """(status, device_error) from the third int64 of the result record."""
    w = int(np.int64(word).astype(np.uint64))
    lo, hi = w & 0xFFFFFFFF, w >> 32
    return (lo - (1 << 32) if lo >= 1 << 31 else lo), (hi - (1 << 32) if hi >= 1 << 31 else hi)


def run_noalloc(torch, cp, cn, sp, sn, n, k, budget, stream, cc=10, cs=1):
    outs = []
    # inputs and outputs are made and filled on the stream the kernel runs
    # on, so the fills are ordered before the kernel
    with torch.cuda.stream(stream):
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
        bufs = dict(cp=dev(cp), cn=dev(cn if len(cn) else np.zeros(1, np.int32)), sp=dev(sp),
                    sn=dev(sn if len(sn) else np.zeros(1, np.int32)))
        for _ in range(2):   # two calls in a row share the library's array
            mask = torch.full((n,), -7, dtype=torch.int8, device="cuda")
            res = torch.full((4,), -9, dtype=torch.int64, device="cuda")
            mpld.mpld_search_instance_noalloc(
                n, k, bufs["cp"].data_ptr(), bufs["cn"].data_ptr(), len(cn),
                bufs["sp"].data_ptr(), bufs["sn"].data_ptr(), len(sn), mask.data_ptr(),
                res.data_ptr(), mpld.make_params(node_budget=budget), stream.cuda_stream, cc, cs)
            outs.append((mask, res))
    stream.synchronize()
    result = []
    for mask, res in outs:
        r = res.cpu().numpy()
        status, derr = split_status(r[2])
        result.append((mask.cpu().numpy(), int(r[0]), int(r[1]), status, derr))
    return result


def run_layout(torch, L, budget, stream):
    cp, cn = csr(L.n_seg, L.conf_u, L.conf_v)
    sp, sn = csr(L.n_seg, L.st_u, L.st_v)
    return run_noalloc(torch, cp, cn, sp, sn, L.n_seg, L.k, budget, stream,
                       L.cost_conflict, L.cost_stitch)


def reference(L, budget, stream):
    prob = mpld.mpld_build_matrix(L, mpld.make_params(flags=SINGLE), stream.cuda_stream)
    rc, mask, res = mpld.mpld_solve(prob, mpld.make_params(node_budget=budget), stream.cuda_stream)
    nodes, cost, status, _ = mpld.mpld_component_results(prob)
    prob.close()
    return mask, int(cost[0]), int(nodes[0]), int(status[0])


CASES = [
    ("k3_small", lambda: synth.unit_disk_layout(60, 3, seed=5, mean_deg=4.5, p_stitch=0.25), 50000),
    ("k4_mid", lambda: synth.unit_disk_layout(300, 4, seed=6, mean_deg=5.0, p_stitch=0.3), 20000),
    ("k8", lambda: synth.unit_disk_layout(200, 8, seed=7, mean_deg=9.0, p_stitch=0.1), 20000),
    # too big for shared memory: the search state stays in the library's array
    ("k3_large", lambda: synth.unit_disk_layout(12000, 3, seed=8, mean_deg=3.5, p_stitch=0.2), 3000),
]


@pytest.mark.parametrize("name,make,budget", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_allocating_entry_point(torch_cuda, name, make, budget):
    stream = torch_cuda.cuda.Stream()
    L = make()
    want = reference(L, budget, stream)
    ref = oracle.decompose(L, flags=oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE, budget=budget)
    assert np.array_equal(ref.mask, want[0]) and (ref.comp_cost[0], ref.comp_nodes[0]) == want[1:3]
    got = run_layout(torch_cuda, L, budget, stream)
    for mask, cost, nodes, status, derr in got:
        assert np.array_equal(mask, want[0])
        assert (cost, nodes, status) == want[1:]
        # the oracle's search of the graph as one instance, element by element
        assert np.array_equal(mask, ref.mask)
        assert (cost, nodes) == (int(ref.comp_cost[0]), int(ref.comp_nodes[0]))
        assert status == (mpld.MPLD_BUDGET if ref.status == oracle.BUDGET else mpld.MPLD_OK)
        assert derr == 0


def test_noalloc_rejects_an_edge_listed_from_one_end(torch_cuda):
    stream = torch_cuda.cuda.Stream()
    # triangle 0-1-2 with 2 listing 0 but 0 not listing 2
    cp = np.array([0, 1, 3, 5], np.int32)
    cn = np.array([1, 0, 2, 0, 1], np.int32)
    sp = np.zeros(4, np.int32)
    for mask, cost, nodes, status, derr in run_noalloc(torch_cuda, cp, cn, sp, [], 3, 3, 0,
                                                       stream):
        assert status == mpld.MPLD_E_INVALID and nodes == 0
        assert (mask == -7).all()      # not written
    # the same triangle listed from both ends is searched
    cp = np.array([0, 2, 4, 6], np.int32)
    cn = np.array([1, 2, 0, 2, 0, 1], np.int32)
    for mask, cost, nodes, status, derr in run_noalloc(torch_cuda, cp, cn, sp, [], 3, 3, 0,
                                                       stream):
        assert (status, cost, nodes, derr) == (mpld.MPLD_OK, 0, 4, 0)
        assert mask.tolist() == [0, 1, 2]


def test_noalloc_rejects_too_large_instances(torch_cuda):
    n = 70000
    cp = torch_cuda.zeros(n + 1, dtype=torch_cuda.int32, device="cuda")
    mask = torch_cuda.zeros(n, dtype=torch_cuda.int8, device="cuda")
    res = torch_cuda.zeros(4, dtype=torch_cuda.int64, device="cuda")
    with pytest.raises(mpld.MpldError) as e:
        mpld.mpld_search_instance_noalloc(n, 3, cp.data_ptr(), 0, 0, cp.data_ptr(), 0, 0,
                                          mask.data_ptr(), res.data_ptr())
    assert e.value.code == mpld.MPLD_E_TOO_LARGE


def test_noalloc_reports_bad_neighbour_ids(torch_cuda):
    stream = torch_cuda.cuda.Stream()
    cp = np.array([0, 1, 2], np.int32)
    cn = np.array([1, 5], np.int32)   # 5 is out of range
    sp = np.zeros(3, np.int32)
    for mask, cost, nodes, status, derr in run_noalloc(torch_cuda, cp, cn, sp, [], 2, 3, 0,
                                                       stream):
        assert status == mpld.MPLD_E_INVALID and (mask == -7).all()


def test_noalloc_rejects_entry_counts_beyond_the_array(torch_cuda):
    # more adjacency entries than the array can hold are refused on the host,
    # before any layout arithmetic, with nothing launched
    n = 1000
    cp = torch_cuda.zeros(n + 1, dtype=torch_cuda.int32, device="cuda")
    mask = torch_cuda.zeros(n, dtype=torch_cuda.int8, device="cuda")
    res = torch_cuda.zeros(4, dtype=torch_cuda.int64, device="cuda")
    for ne2 in ((1 << 31) - 1, mpld.MPLD_NOALLOC_SCRATCH_BYTES // 2 + 1):
        with pytest.raises(mpld.MpldError) as e:
            mpld.mpld_search_instance_noalloc(n, 8, cp.data_ptr(), cp.data_ptr(), ne2, cp.data_ptr(),
                                              0, 0, mask.data_ptr(), res.data_ptr(), None, 0, 0, 1)
        assert e.value.code == mpld.MPLD_E_TOO_LARGE
