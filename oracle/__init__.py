"""CPU oracle for the exact-cover layout decomposition search.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product
library (``paper_2303_14335_gb300``) never imports it, and the two share no
code: the oracle is plain C dancing links (Knuth's Algorithm X, Sec. 2.3 and
Eq. 2 of the paper) written from the problem statement (Sec. 2.1, Eq. 1),
with its own simplification, component split and recovery (Sec. 2.2).

Every function here is pinned by the ``-m "not gpu"`` tests against things
other than itself: brute force over all k^n colourings, closed-form counts
of proper colourings (chromatic polynomials), hand-derived search traces and
an independent recursive graph search written in Python under ``tests/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpld_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmpld_oracle.so")

OK = 0
BUDGET = 1
E_INVALID = -1
E_OOM = -2
NO_SIMPLIFY = 1
SINGLE_INSTANCE = 2
COLUMN_BFS = 8      # the paper's column rule (single-row column, else BFS order)
BICONNECTED = 16    # search the biconnected blocks of each component, merge at cut segments
CLIQUE_BOUND = 32   # second bound mode: dead columns plus untouched edge-disjoint (k+1)-cliques
SPLIT_BUDGET = 64   # budgeted split search: the node budget spread over independent subtree searches
DENSITY_BALANCE = 128  # per-component mask permutations and recovery that balance mask usage
INF = (1 << 63) - 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no vector extensions)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-fPIC", "-shared", "-o", tmp, _SRC,
                           "-lpthread"])
    os.replace(tmp, _LIB)
    return _LIB


class _Totals(ctypes.Structure):
    _fields_ = [("n_components", ctypes.c_int64), ("n_removed_segments", ctypes.c_int64),
                ("n_conflicts", ctypes.c_int64), ("n_stitches", ctypes.c_int64),
                ("cost", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("component_cost_sum", ctypes.c_int64), ("n_budget_components", ctypes.c_int64),
                ("status", ctypes.c_int32), ("max_component", ctypes.c_int32),
                ("search_seconds", ctypes.c_double), ("instance_segments", ctypes.c_int64)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.oracle_solve_instance.argtypes = [i32, i32, i32, P, P, i32, P, P, i64, i64, i64, P, P, P]
        lib.oracle_solve_instance.restype = i32
        lib.oracle_solve_instance_rule.argtypes = [i32, i32, i32, P, P, i32, P, P, i64, i64, i64, i32,
                                                   P, P, P]
        lib.oracle_solve_instance_rule.restype = i32
        lib.oracle_count_exact_covers.argtypes = [i32, i32, i32, P, P, i64, P]
        lib.oracle_count_exact_covers.restype = i32
        lib.oracle_export_matrix.argtypes = [i32, i32, i32, P, P, P]
        lib.oracle_export_matrix.restype = i32
        lib.oracle_decompose.argtypes = [i32, i32, i32, P, P, i32, P, P, P, i64, i64, ctypes.c_uint32,
                                         i64, i32, P, P, P, P, P, ctypes.POINTER(_Totals)]
        lib.oracle_decompose.restype = i32
        lib.oracle_blocks.argtypes = [i32, i32, P, P, i32, P, P, P, P, P]
        lib.oracle_blocks.restype = i32
        lib.oracle_cliques.argtypes = [i32, i32, i32, P, P, i32, P]
        lib.oracle_cliques.restype = i32
        _lib = lib
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else ctypes.c_void_p(0)


@dataclass
class InstanceResult:
    status: int
    cost: int
    nodes: int
    x: np.ndarray


def solve_instance(n, k, conf, stitch=(), cost_conflict=10, cost_stitch=1, budget=0,
                   rule=0, clique_bound=False, split=False) -> InstanceResult:
    """Search one instance (the whole graph), Algorithm X with dancing links.

    rule 0: column with the fewest rows, lowest index on ties; rule 1: the
    paper's rule (a column with one row left, else breadth-first order).
    clique_bound: the second bound mode (dead columns plus untouched
    edge-disjoint (k+1)-cliques).  split: the budgeted split search (the
    node budget spent by a first search and then by independent searches of
    the subtrees below a fixed depth).
    """
    lib = _load()
    conf = np.asarray(conf, dtype=np.int32).reshape(-1, 2)
    stitch = np.asarray(stitch, dtype=np.int32).reshape(-1, 2)
    cu, cv = _i32(conf[:, 0]), _i32(conf[:, 1])
    su, sv = _i32(stitch[:, 0]), _i32(stitch[:, 1])
    x = np.full(max(n, 1), -1, dtype=np.int8)
    cost = ctypes.c_int64(0)
    nodes = ctypes.c_int64(0)
    rc = lib.oracle_solve_instance_rule(n, k, len(cu), _ptr(cu), _ptr(cv), len(su), _ptr(su),
                                        _ptr(sv), cost_conflict, cost_stitch, budget,
                                        rule | (2 if clique_bound else 0) | (4 if split else 0),
                                        _ptr(x),
                                        ctypes.byref(cost), ctypes.byref(nodes))
    if rc < 0:
        raise ValueError(f"oracle_solve_instance failed: {rc}")
    return InstanceResult(status=rc, cost=cost.value, nodes=nodes.value, x=x[:n].copy())


def cliques(n, k, conf) -> list:
    """The clique bound's cliques: greedy edge-disjoint (k+1)-cliques of the
    conflict graph in lexicographic order, each an ascending member list."""
    lib = _load()
    conf = np.asarray(conf, dtype=np.int32).reshape(-1, 2)
    cu, cv = _i32(conf[:, 0]), _i32(conf[:, 1])
    cap = max(1, len(cu))
    out = np.zeros(cap * (k + 1), dtype=np.int32)
    nq = lib.oracle_cliques(n, k, len(cu), _ptr(cu), _ptr(cv), cap, _ptr(out))
    if nq < 0:
        raise ValueError(f"oracle_cliques failed: {nq}")
    return [out[q * (k + 1):(q + 1) * (k + 1)].tolist() for q in range(nq)]


def count_exact_covers(n, k, conf, limit=1 << 62) -> int:
    """Exact covers of the EC matrix (textbook Algorithm X, active rows only)."""
    lib = _load()
    conf = np.asarray(conf, dtype=np.int32).reshape(-1, 2)
    cu, cv = _i32(conf[:, 0]), _i32(conf[:, 1])
    cnt = ctypes.c_int64(0)
    rc = lib.oracle_count_exact_covers(n, k, len(cu), _ptr(cu), _ptr(cv), limit, ctypes.byref(cnt))
    if rc < 0:
        raise ValueError(f"oracle_count_exact_covers failed: {rc}")
    return cnt.value


def export_matrix(n, k, conf) -> np.ndarray:
    """Dense 0/1 EC matrix [n*k, 1 + n + k*|E|] (column 0 is the root, all 0)."""
    lib = _load()
    conf = np.asarray(conf, dtype=np.int32).reshape(-1, 2)
    cu, cv = _i32(conf[:, 0]), _i32(conf[:, 1])
    ne = len({(min(a, b), max(a, b)) for a, b in conf.tolist()})
    out = np.zeros((n * k, 1 + n + k * ne), dtype=np.uint8)
    rc = lib.oracle_export_matrix(n, k, len(cu), _ptr(cu), _ptr(cv), _ptr(out))
    if rc < 0:
        raise ValueError(f"oracle_export_matrix failed: {rc}")
    return out


def blocks(n, conf, stitch=()):
    """Biconnected blocks of every component of the graph (no simplification),
    in the canonical order the flow searches them: list of (segments ascending,
    attach segment or -1)."""
    lib = _load()
    conf = np.asarray(conf, dtype=np.int32).reshape(-1, 2)
    stitch = np.asarray(stitch, dtype=np.int32).reshape(-1, 2)
    cu, cv = _i32(conf[:, 0]), _i32(conf[:, 1])
    su, sv = _i32(stitch[:, 0]), _i32(stitch[:, 1])
    cap = 2 * (n + len(cu) + len(su)) + 1
    ip = np.zeros(n + 2, dtype=np.int32)
    iseg = np.zeros(cap, dtype=np.int32)
    iatt = np.zeros(cap, dtype=np.int32)
    nb = lib.oracle_blocks(n, len(cu), _ptr(cu), _ptr(cv), len(su), _ptr(su), _ptr(sv), _ptr(ip),
                           _ptr(iseg), _ptr(iatt))
    if nb < 0:
        raise ValueError(f"oracle_blocks failed: {nb}")
    return [(iseg[ip[b]:ip[b + 1]].tolist(), int(iatt[b])) for b in range(nb)]


@dataclass
class LayoutResult:
    status: int
    mask: np.ndarray
    comp_of: np.ndarray
    comp_nodes: np.ndarray
    comp_cost: np.ndarray
    comp_status: np.ndarray
    n_components: int
    n_removed_segments: int
    n_conflicts: int
    n_stitches: int
    cost: int
    nodes: int
    component_cost_sum: int
    n_budget_components: int
    max_component: int
    search_seconds: float = 0.0    # wall time of the search phase alone (timing, not a result)
    instance_segments: int = 0     # segments inside search instances


def decompose(layout, *, flags: int = 0, budget: int = 0, nthreads: int = 1) -> LayoutResult:
    """Simplify, split into components, search each, recover, count (Sec. 2.2-2.3)."""
    lib = _load()
    n = int(layout.n_seg)
    cu, cv = _i32(layout.conf_u), _i32(layout.conf_v)
    su, sv = _i32(layout.st_u), _i32(layout.st_v)
    poly = _i32(layout.polygon_of) if layout.polygon_of is not None else None
    m = max(n, 1)
    mask = np.full(m, -1, dtype=np.int8)
    comp_of = np.full(m, -1, dtype=np.int32)
    cn = np.zeros(m, dtype=np.int64)
    cc = np.zeros(m, dtype=np.int64)
    cs = np.zeros(m, dtype=np.int32)
    tot = _Totals()
    rc = lib.oracle_decompose(n, int(layout.k), len(cu), _ptr(cu), _ptr(cv), len(su), _ptr(su), _ptr(sv),
                              _ptr(poly) if poly is not None else ctypes.c_void_p(0),
                              int(layout.cost_conflict), int(layout.cost_stitch), flags, budget,
                              nthreads, _ptr(mask), _ptr(comp_of), _ptr(cn), _ptr(cc), _ptr(cs),
                              ctypes.byref(tot))
    if rc < 0:
        raise ValueError(f"oracle_decompose failed: {rc}")
    nc = int(tot.n_components)
    return LayoutResult(status=rc, mask=mask[:n].copy(), comp_of=comp_of[:n].copy(),
                        comp_nodes=cn[:nc].copy(), comp_cost=cc[:nc].copy(), comp_status=cs[:nc].copy(),
                        n_components=nc, n_removed_segments=int(tot.n_removed_segments),
                        n_conflicts=int(tot.n_conflicts), n_stitches=int(tot.n_stitches),
                        cost=int(tot.cost), nodes=int(tot.nodes),
                        component_cost_sum=int(tot.component_cost_sum),
                        n_budget_components=int(tot.n_budget_components),
                        max_component=int(tot.max_component),
                        search_seconds=float(tot.search_seconds),
                        instance_segments=int(tot.instance_segments))
