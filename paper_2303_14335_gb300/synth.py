"""Seeded synthetic layout graphs for the MPLD exact-cover search.

This module only draws inputs.  It holds none of the method's arithmetic (no
simplification, no exact-cover matrix, no search, no costs) so that both the
CUDA path and the CPU oracle can be fed from it without sharing any of the
code that is being checked.

The paper evaluates on ISCAS layouts (Sec. 3, Table 1), which are not
available here.  They are replaced by unit-disk conflict graphs shaped like
those layouts:

* polygons are points drawn uniformly in the unit square;
* two polygons conflict when their Euclidean distance is below ``r``, with
  ``r`` solved from the mean degree (boundary-corrected formula below);
* each polygon is split with probability ``p`` into two segments joined by a
  stitch edge (the stitch candidates of Sec. 1 / Fig. 1c); each conflict edge
  of a split polygon attaches to segment A or B by the sign of the
  neighbour's offset projected on a direction drawn for that polygon.

Random numbers come from SplitMix64 written out from its published
definition (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used as a counter-based stream: draw ``i`` of
stream ``seed`` is ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``.  A draw maps
to a double in [0, 1) as ``(z >> 11) * 2**-53``.  Only IEEE additions and
multiplications follow, so the same seed gives the same graph on x86 and
Arm.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx) -> np.ndarray:
    """Draws ``idx`` (array of counters) of the SplitMix64 stream ``seed``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, idx) -> np.ndarray:
    """Doubles in [0, 1) from draws ``idx`` of stream ``seed``."""
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Layout:
    """A layout conflict graph with stitch candidates (the input of Eq. 1).

    Segments are numbered ``0..n_seg-1``; the segments of one polygon are
    consecutive.  ``conf_u < conf_v`` and the conflict edges are sorted by
    ``(conf_u, conf_v)``; stitch edges likewise.
    """

    n_seg: int
    k: int
    conf_u: np.ndarray
    conf_v: np.ndarray
    st_u: np.ndarray
    st_v: np.ndarray
    polygon_of: np.ndarray
    n_poly: int
    cost_conflict: int = 10
    cost_stitch: int = 1
    name: str = ""
    points: np.ndarray | None = field(default=None, repr=False)

    @property
    def n_conf(self) -> int:
        return int(self.conf_u.shape[0])

    @property
    def n_stitch(self) -> int:
        return int(self.st_u.shape[0])


def radius_for_degree(n_poly: int, mean_deg: float) -> float:
    """Radius r with (N-1) * (pi r^2 - 8 r^3 / 3 + r^4 / 2) = mean_deg.

    The bracket is the expected fraction of the unit square within distance
    r of a uniform point (two uniform points in the unit square are closer
    than r with that probability), so it corrects for the square's border.
    Solved by bisection, which only uses + and *.
    """
    if n_poly < 2 or mean_deg <= 0:
        return 0.0
    target = mean_deg / (n_poly - 1)
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        f = math.pi * mid * mid - (8.0 / 3.0) * mid ** 3 + 0.5 * mid ** 4
        if f < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _pairs_within(points: np.ndarray, r: float) -> np.ndarray:
    """All index pairs (i < j) with squared distance < r*r, sorted."""
    from scipy.spatial import cKDTree

    n = points.shape[0]
    if n < 2 or r <= 0:
        return np.zeros((0, 2), dtype=np.int64)
    cand = cKDTree(points).query_pairs(r * (1.0 + 1e-6), output_type="ndarray")
    if cand.shape[0] == 0:
        return np.zeros((0, 2), dtype=np.int64)
    cand = np.sort(cand.astype(np.int64), axis=1)
    dx = points[cand[:, 0], 0] - points[cand[:, 1], 0]
    dy = points[cand[:, 0], 1] - points[cand[:, 1], 1]
    keep = dx * dx + dy * dy < r * r
    cand = cand[keep]
    order = np.lexsort((cand[:, 1], cand[:, 0]))
    return cand[order]


def _connected(n: int, pairs: np.ndarray) -> bool:
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    if n <= 1:
        return True
    m = coo_matrix((np.ones(pairs.shape[0]), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
    ncomp, _ = connected_components(m, directed=False)
    return ncomp == 1


def unit_disk_layout(n_poly: int, k: int, seed: int, *, mean_deg: float | None = None,
                     radius: float | None = None, p_stitch: float = 0.0,
                     connected: bool = False, name: str = "",
                     cost_conflict: int = 10, cost_stitch: int = 1,
                     max_attempts: int = 10000) -> Layout:
    """Unit-disk conflict graph with stitch splits.

    Draw order of stream ``seed``: attempt ``t`` takes draws
    ``[2Nt, 2N(t+1))`` as ``x_i = u(2Nt + 2i)``, ``y_i = u(2Nt + 2i + 1)``;
    when ``connected`` is set, attempts repeat until the polygon graph is
    connected.  After the accepted attempt, polygon ``i`` takes draws
    ``base + 3i`` (split test ``u < p_stitch``) and ``base + 3i + 1``,
    ``base + 3i + 2`` (split direction ``(u - 0.5, u - 0.5)``), with
    ``base = 2N(t+1)``.
    """
    if radius is None:
        radius = radius_for_degree(n_poly, mean_deg or 0.0)
    N = int(n_poly)
    t = 0
    while True:
        d = uniform(seed, np.arange(2 * N * t, 2 * N * (t + 1), dtype=np.uint64))
        pts = np.stack([d[0::2], d[1::2]], axis=1)
        pairs = _pairs_within(pts, radius)
        if not connected or _connected(N, pairs):
            break
        t += 1
        if t >= max_attempts:
            raise RuntimeError("no connected point set within max_attempts")
    base = 2 * N * (t + 1)
    dr = uniform(seed, np.arange(base, base + 3 * N, dtype=np.uint64)).reshape(N, 3) if N else np.zeros((0, 3))
    split = dr[:, 0] < p_stitch
    da = dr[:, 1] - 0.5
    db = dr[:, 2] - 0.5
    nseg_of = 1 + split.astype(np.int64)
    first = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(nseg_of, out=first[1:])
    n_seg = int(first[N])

    i = pairs[:, 0]
    j = pairs[:, 1]
    offx = pts[j, 0] - pts[i, 0]
    offy = pts[j, 1] - pts[i, 1]
    side_i = split[i] & (offx * da[i] + offy * db[i] > 0)
    side_j = split[j] & ((-offx) * da[j] + (-offy) * db[j] > 0)
    su = first[i] + side_i.astype(np.int64)
    sv = first[j] + side_j.astype(np.int64)
    cu = np.minimum(su, sv)
    cv = np.maximum(su, sv)
    order = np.lexsort((cv, cu))
    cu, cv = cu[order], cv[order]

    sp = np.nonzero(split)[0]
    st_u = first[sp]
    st_v = first[sp] + 1
    polygon_of = np.repeat(np.arange(N, dtype=np.int64), nseg_of)
    return Layout(n_seg=n_seg, k=int(k), conf_u=cu.astype(np.int32), conf_v=cv.astype(np.int32),
                  st_u=st_u.astype(np.int32), st_v=st_v.astype(np.int32),
                  polygon_of=polygon_of.astype(np.int32), n_poly=N,
                  cost_conflict=cost_conflict, cost_stitch=cost_stitch, name=name, points=pts)


def random_graph(n: int, k: int, seed: int, *, p_edge: float = 0.4, n_stitch: int = 0,
                 identity_polygons: bool = True) -> Layout:
    """Small Erdos-Renyi conflict graph plus stitch edges, for exhaustive tests.

    Pair ``(a, b)`` (``a < b``, row-major order, pair index ``q``) is a
    conflict edge when draw ``q`` < ``p_edge``.  Then ``n_stitch`` stitch
    edges are drawn as pairs ``(a, b)`` from the following draws; a pair
    already used by a conflict or stitch edge is skipped.  Every segment is
    its own polygon unless ``identity_polygons`` is False, in which case the
    endpoints of each stitch edge are merged into one polygon (the lower id's
    polygon) so that stitch edges join segments of one polygon.
    """
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    u = uniform(seed, np.arange(len(pairs), dtype=np.uint64)) if pairs else np.zeros(0)
    conf = [pairs[q] for q in range(len(pairs)) if u[q] < p_edge]
    used = set(conf)
    st = []
    pos = len(pairs)
    tries = 0
    while len(st) < n_stitch and len(pairs) > len(used) and tries < 1000:
        ab = uniform(seed, np.array([pos, pos + 1], dtype=np.uint64))
        pos += 2
        tries += 1
        a = int(ab[0] * n)
        b = int(ab[1] * n)
        if a == b:
            continue
        a, b = min(a, b), max(a, b)
        if (a, b) in used:
            continue
        used.add((a, b))
        st.append((a, b))
    st.sort()
    poly = np.arange(n, dtype=np.int32)
    if not identity_polygons:
        # union stitch-joined segments into one polygon each
        parent = list(range(n))

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        for a, b in st:
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
        poly = np.array([find(a) for a in range(n)], dtype=np.int32)
    cu = np.array([a for a, _ in conf], dtype=np.int32)
    cv = np.array([b for _, b in conf], dtype=np.int32)
    su = np.array([a for a, _ in st], dtype=np.int32)
    sv = np.array([b for _, b in st], dtype=np.int32)
    return Layout(n_seg=n, k=int(k), conf_u=cu, conf_v=cv, st_u=su, st_v=sv,
                  polygon_of=poly, n_poly=n, name=f"er{n}_k{k}_s{seed}")


def graph_from_edges(n: int, k: int, conf, stitch=(), polygon_of=None, name: str = "",
                     cost_conflict: int = 10, cost_stitch: int = 1) -> Layout:
    """Layout from explicit edge lists (edges are normalised and sorted)."""
    conf = sorted({(min(a, b), max(a, b)) for a, b in conf})
    stitch = sorted({(min(a, b), max(a, b)) for a, b in stitch})
    poly = np.arange(n, dtype=np.int32) if polygon_of is None else np.asarray(polygon_of, dtype=np.int32)
    return Layout(n_seg=n, k=int(k),
                  conf_u=np.array([a for a, _ in conf], dtype=np.int32),
                  conf_v=np.array([b for _, b in conf], dtype=np.int32),
                  st_u=np.array([a for a, _ in stitch], dtype=np.int32),
                  st_v=np.array([b for _, b in stitch], dtype=np.int32),
                  polygon_of=poly, n_poly=int(poly.max()) + 1 if n else 0, name=name,
                  cost_conflict=cost_conflict, cost_stitch=cost_stitch)


# Workloads shaped like the paper's layouts (Sec. 3).  ``flags`` names the
# decomposition mode: "single" = the whole graph is one search instance with
# no simplification; "batched" = simplification + one instance per connected
# component.
WORKLOADS = {
    "k3_n24_plain": dict(n_poly=24, k=3, seed=0, radius=0.32, p_stitch=0.0, connected=True,
                         mode="single"),
    "k3_n400_p025_plain": dict(n_poly=400, k=3, seed=1, mean_deg=4.5, p_stitch=0.25,
                               mode="single"),
    "k3_n200k_p02_batched": dict(n_poly=200_000, k=3, seed=2, mean_deg=3.0, p_stitch=0.2,
                                 mode="batched"),
    "k4_n100k_p03_batched": dict(n_poly=100_000, k=4, seed=3, mean_deg=5.0, p_stitch=0.3,
                                 mode="batched"),
}


def workload(name: str) -> tuple[Layout, str]:
    """The named workload's layout and its decomposition mode."""
    cfg = dict(WORKLOADS[name])
    mode = cfg.pop("mode")
    return unit_disk_layout(name=name, **cfg), mode


def serving_request(stream_seed: int, i: int, *, n_min: int = 1000, n_max: int = 200_000,
                    p_stitch: float = 0.2) -> Layout:
    """Request ``i`` of a serving stream: log-uniform size, k in {3,4}, degree U[3,5].

    Draws ``4i .. 4i+3`` of stream ``stream_seed`` give the size, k, degree
    and the request's own layout seed.
    """
    d = uniform(stream_seed, np.arange(4 * i, 4 * i + 4, dtype=np.uint64))
    n_poly = int(math.exp(math.log(n_min) + d[0] * (math.log(n_max) - math.log(n_min))))
    k = 3 if d[1] < 0.5 else 4
    deg = 3.0 + 2.0 * d[2]
    seed = int(splitmix64(stream_seed ^ 0x5EED, np.array([i], dtype=np.uint64))[0])
    return unit_disk_layout(n_poly, k, seed, mean_deg=deg, p_stitch=p_stitch,
                            name=f"req{i}")


def poisson_arrivals(stream_seed: int, n: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: exponential gaps from ``-ln(1-u)/rate``."""
    u = uniform(stream_seed ^ 0xA77, np.arange(n, dtype=np.uint64))
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)
