"""The seeded input generator (shared by the oracle tests and the CUDA path)."""
import numpy as np
import pytest

from paper_2303_14335_gb300 import synth


def test_splitmix64_published_vector():
    # First outputs of SplitMix64 from state 0 (Steele, Lea, Flood 2014;
    # the sequence used to seed xoshiro generators).
    z = synth.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_determinism():
    a = synth.uniform(7, np.arange(10000, dtype=np.uint64))
    b = synth.uniform(7, np.arange(10000, dtype=np.uint64))
    assert np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.02


def test_radius_formula_matches_mean_degree():
    # The border-corrected formula should give the requested mean degree.
    L = synth.unit_disk_layout(20000, 3, seed=11, mean_deg=4.0)
    deg = 2 * L.n_conf / L.n_poly
    assert abs(deg - 4.0) < 0.1


def test_edges_are_exactly_the_close_pairs():
    L = synth.unit_disk_layout(300, 3, seed=5, radius=0.08, p_stitch=0.0)
    p = L.points
    want = {(i, j) for i in range(300) for j in range(i + 1, 300)
            if (p[i, 0] - p[j, 0]) ** 2 + (p[i, 1] - p[j, 1]) ** 2 < 0.08 ** 2}
    got = set(zip(L.conf_u.tolist(), L.conf_v.tolist()))
    assert got == want


def test_stitch_split_structure():
    L = synth.unit_disk_layout(2000, 3, seed=9, mean_deg=4.0, p_stitch=0.3)
    poly = L.polygon_of
    # segments of a polygon are consecutive, split polygons have 2 segments
    assert np.all(np.diff(poly) >= 0)
    counts = np.bincount(poly, minlength=L.n_poly)
    assert set(np.unique(counts)) <= {1, 2}
    assert L.n_stitch == int((counts == 2).sum())
    assert abs(L.n_stitch / L.n_poly - 0.3) < 0.05
    assert np.all(poly[L.st_u] == poly[L.st_v]) and np.all(L.st_v == L.st_u + 1)
    # one segment-level edge per polygon-level edge, endpoints in different polygons
    assert np.all(poly[L.conf_u] != poly[L.conf_v])
    pairs = set(zip(poly[L.conf_u].tolist(), poly[L.conf_v].tolist()))
    assert len(pairs) == L.n_conf
    # sorted, normalised
    assert np.all(L.conf_u < L.conf_v)
    key = L.conf_u.astype(np.int64) * L.n_seg + L.conf_v
    assert np.all(np.diff(key) > 0)


def test_connected_resampling():
    L = synth.unit_disk_layout(24, 3, seed=0, radius=0.32, connected=True)
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    m = coo_matrix((np.ones(L.n_conf), (L.conf_u, L.conf_v)), shape=(24, 24))
    assert connected_components(m, directed=False)[0] == 1


@pytest.mark.parametrize("name", ["k3_n24_plain", "k3_n400_p025_plain"])
def test_workload_shapes(name):
    L, mode = synth.workload(name)
    assert mode == "single"
    if name == "k3_n24_plain":
        assert L.n_seg == 24 and L.n_stitch == 0 and L.k == 3
    else:
        assert 450 < L.n_seg < 560 and L.k == 3
        assert abs(2 * L.n_conf / L.n_poly - 4.5) < 0.6


def test_random_graph_polygons():
    L = synth.random_graph(8, 3, seed=3, p_edge=0.4, n_stitch=2, identity_polygons=False)
    for a, b in zip(L.st_u, L.st_v):
        assert L.polygon_of[a] == L.polygon_of[b]
    conf = set(zip(L.conf_u.tolist(), L.conf_v.tolist()))
    st = set(zip(L.st_u.tolist(), L.st_v.tolist()))
    assert not (conf & st)
