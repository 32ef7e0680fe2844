"""The allocation-free entry point, mpld_search_instance_noalloc.

It serves callers that may not allocate GPU memory themselves (for example
a plug-in inside an application whose caching allocator owns the device
memory, or a caller that cannot afford the synchronisation an allocation
can cause): they hand over device buffers for the instance and the
outputs, and the library works in a fixed array of its own.  These tests
check its output against the allocating entry point, mpld_solve, on the
same graph: masks, cost, node count and status must be identical, on two
calls in a row.  This file is collected last so that a run that stops at
the first failure has already run every other test.
"""
import numpy as np
import pytest

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


def run_noalloc(torch, L, budget, stream):
    cp, cn = csr(L.n_seg, L.conf_u, L.conf_v)
    sp, sn = csr(L.n_seg, L.st_u, L.st_v)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bufs = dict(cp=dev(cp), cn=dev(cn if len(cn) else np.zeros(1, np.int32)), sp=dev(sp),
                sn=dev(sn if len(sn) else np.zeros(1, np.int32)))
    outs = []
    for _ in range(2):   # two calls in a row share the library's array
        mask = torch.full((L.n_seg,), -7, dtype=torch.int8, device="cuda")
        res = torch.zeros(4, dtype=torch.int64, device="cuda")
        mpld.mpld_search_instance_noalloc(
            L.n_seg, L.k, bufs["cp"].data_ptr(), bufs["cn"].data_ptr(), len(cn),
            bufs["sp"].data_ptr(), bufs["sn"].data_ptr(), len(sn), mask.data_ptr(), res.data_ptr(),
            mpld.make_params(node_budget=budget), stream.cuda_stream,
            L.cost_conflict, L.cost_stitch)
        outs.append((mask, res))
    stream.synchronize()
    result = []
    for mask, res in outs:
        r = res.cpu().numpy()
        status = int(np.int64(r[2]).astype(np.uint64) & 0xFFFFFFFF)
        status = status - (1 << 32) if status >= 1 << 31 else status
        result.append((mask.cpu().numpy(), int(r[0]), int(r[1]), status))
    return result


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
    got = run_noalloc(torch_cuda, L, budget, stream)
    for mask, cost, nodes, status in got:
        assert np.array_equal(mask, want[0])
        assert (cost, nodes, status) == want[1:]


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
    cp = torch_cuda.tensor([0, 1, 2], dtype=torch_cuda.int32, device="cuda")
    cn = torch_cuda.tensor([1, 5], dtype=torch_cuda.int32, device="cuda")   # 5 is out of range
    sp = torch_cuda.zeros(3, dtype=torch_cuda.int32, device="cuda")
    mask = torch_cuda.zeros(2, dtype=torch_cuda.int8, device="cuda")
    res = torch_cuda.zeros(4, dtype=torch_cuda.int64, device="cuda")
    mpld.mpld_search_instance_noalloc(2, 3, cp.data_ptr(), cn.data_ptr(), 2, sp.data_ptr(), 0, 0,
                                      mask.data_ptr(), res.data_ptr(), None, stream.cuda_stream)
    stream.synchronize()
    assert int(res[2].item()) & 0xFFFFFFFF == (mpld.MPLD_E_INVALID & 0xFFFFFFFF)
