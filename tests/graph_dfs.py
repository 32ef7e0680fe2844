"""Independent pure-Python restatements of the canonical search, used to pin the oracle.

Nothing here touches dancing links or bitsets: the state is the partial
assignment ``x`` itself.  A segment's "column size" is the number of masks
not used by an assigned conflict neighbour (the active rows of its primary
column in the EC matrix of Sec. 2.3); a row's added cost is the Eq. 1 cost of
its edges to assigned neighbours.  Only for tiny graphs.
"""
from __future__ import annotations

import itertools

import numpy as np


def adjacency(n, edges):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    return [sorted(set(l)) for l in adj]


def eq1_cost(x, conf, stitch, cc=10, cs=1):
    """Eq. 1 written out: Cc * #monochromatic conflict edges + Cs * #cut stitch edges."""
    return cc * sum(1 for a, b in conf if x[a] == x[b]) + cs * sum(1 for a, b in stitch if x[a] != x[b])


def brute_force(n, k, conf, stitch, cc=10, cs=1):
    """(min cost, number of optimal assignments) over all k^n assignments (numpy)."""
    if n == 0:
        return 0, 1
    X = np.array(list(itertools.product(range(k), repeat=n)), dtype=np.int8)
    cost = np.zeros(X.shape[0], dtype=np.int64)
    for a, b in conf:
        cost += cc * (X[:, a] == X[:, b])
    for a, b in stitch:
        cost += cs * (X[:, a] != X[:, b])
    m = int(cost.min())
    return m, int((cost == m).sum())


def bfs_rank(n, conf, stitch):
    """Breadth-first rank over conflict and stitch edges: roots in ascending
    id, each segment's neighbours (by either kind of edge) in ascending id."""
    nb = adjacency(n, list(conf) + list(stitch))
    rank = [-1] * n
    nxt = 0
    for r in range(n):
        if rank[r] >= 0:
            continue
        rank[r] = nxt
        nxt += 1
        queue = [r]
        while queue:
            u = queue.pop(0)
            for w in nb[u]:
                if rank[w] < 0:
                    rank[w] = nxt
                    nxt += 1
                    queue.append(w)
    return rank


def greedy_cliques(n, k, conf):
    """Edge-disjoint (k+1)-cliques: all of them in lexicographic order of
    their ascending member tuples (itertools.combinations order), each
    taken when it shares no edge with one taken before."""
    adj = [set(a) for a in adjacency(n, conf)]
    used, out = set(), []
    for t in itertools.combinations(range(n), k + 1):
        pairs = list(itertools.combinations(t, 2))
        if all(b in adj[a] for a, b in pairs) and not any(p in used for p in pairs):
            used.update(pairs)
            out.append(list(t))
    return out


class _Search:
    def __init__(self, n, k, conf, stitch, cc, cs, rule=0):
        self.n, self.k, self.cc, self.cs = n, k, cc, cs
        self.cadj = adjacency(n, conf)
        self.sadj = adjacency(n, stitch)
        self.x = [-1] * n
        self.rule = rule
        self.rank = bfs_rank(n, conf, stitch) if rule == 1 else None

    def avail(self, v):
        used = {self.x[u] for u in self.cadj[v] if self.x[u] >= 0}
        return self.k - len(used)

    def pick(self):
        """Column to branch on, and Z (uncovered segments with no available mask).

        rule 0: fewest available masks, lowest index on ties; rule 1: lowest
        index with exactly one available mask, else lowest breadth-first rank.
        """
        best_v, best_a, z = -1, None, 0
        single, by_rank = -1, -1
        for v in range(self.n):
            if self.x[v] >= 0:
                continue
            a = self.avail(v)
            if a == 0:
                z += 1
            if best_a is None or a < best_a:
                best_v, best_a = v, a
            if self.rule == 1:
                if a == 1 and single < 0:
                    single = v
                if by_rank < 0 or self.rank[v] < self.rank[by_rank]:
                    by_rank = v
        if self.rule == 1 and best_v >= 0:
            best_v = single if single >= 0 else by_rank
        return best_v, z

    def row_order(self, v):
        inc = []
        for c in range(self.k):
            t = self.cc * sum(1 for u in self.cadj[v] if self.x[u] == c)
            t += self.cs * sum(1 for u in self.sadj[v] if self.x[u] >= 0 and self.x[u] != c)
            inc.append(t)
        return sorted(range(self.k), key=lambda c: (inc[c], c)), inc


def canonical_leaves(n, k, conf, stitch, cc=10, cs=1, rule=0):
    """Every leaf of the bound-free canonical search tree, in depth-first order.

    Returns a list of (cost, x).  The method's answer is the first leaf of
    minimum cost in this list.
    """
    S = _Search(n, k, conf, stitch, cc, cs, rule)
    out = []

    def rec(g):
        v, _ = S.pick()
        if v < 0:
            out.append((g, list(S.x)))
            return
        order, inc = S.row_order(v)
        for c in order:
            S.x[v] = c
            rec(g + inc[c])
            S.x[v] = -1

    rec(0)
    return out


def first_min_leaf(n, k, conf, stitch, cc=10, cs=1, rule=0):
    leaves = canonical_leaves(n, k, conf, stitch, cc, cs, rule)
    m = min(c for c, _ in leaves)
    for c, x in leaves:
        if c == m:
            return c, x


def bounded_search(n, k, conf, stitch, cc=10, cs=1, budget=0, rule=0, clique_bound=False):
    """The canonical search with the dead-segment bound and node budget.

    node = one call; leaf with g < best is the new incumbent and best == 0
    stops; prune when g + cc * (#unassigned segments with no available mask)
    >= best; with clique_bound, the number of greedy cliques with no member
    assigned is added to that count; with budget B > 0, a call made when an
    incumbent exists and B nodes have been counted stops everything.
    Returns (cost, x, nodes, budget_hit).
    """
    S = _Search(n, k, conf, stitch, cc, cs, rule)
    cl = greedy_cliques(n, k, conf) if clique_bound else []
    st = dict(best=None, bestx=None, nodes=0, done=False, hit=False)

    def rec(g):
        if budget > 0 and st["best"] is not None and st["nodes"] >= budget:
            st["hit"] = True
            st["done"] = True
            return
        st["nodes"] += 1
        v, z = S.pick()
        if v < 0:
            if st["best"] is None or g < st["best"]:
                st["best"], st["bestx"] = g, list(S.x)
                if g == 0:
                    st["done"] = True
            return
        q = sum(1 for c in cl if all(S.x[v] < 0 for v in c))
        if st["best"] is not None and g + cc * (z + q) >= st["best"]:
            return
        order, inc = S.row_order(v)
        for c in order:
            if st["done"]:
                break
            S.x[v] = c
            rec(g + inc[c])
            S.x[v] = -1

    rec(0)
    return st["best"], st["bestx"], st["nodes"], st["hit"]


def _search_with_prefix(n, k, conf, stitch, cc, cs, budget, rule, prefix, init_best, track):
    """bounded_search with three additions for the budgeted split search:
    at level i < len(prefix) only the row at place prefix[i] of the row
    order is taken; the incumbent starts at ``init_best`` (None = no bound;
    a leaf must cost less than it to be taken); the row places of the
    incumbent leaf's path are kept for its first ``track`` levels.
    Returns (best, bestx, nodes, budget_hit, found, best_places)."""
    S = _Search(n, k, conf, stitch, cc, cs, rule)
    st = dict(best=init_best, bestx=None, nodes=0, done=False, hit=False, found=False,
              places=None)
    path = []

    def rec(g):
        if budget > 0 and st["best"] is not None and st["nodes"] >= budget:
            st["hit"] = True
            st["done"] = True
            return
        st["nodes"] += 1
        v, z = S.pick()
        if v < 0:
            if st["best"] is None or g < st["best"]:
                st["best"], st["bestx"], st["found"] = g, list(S.x), True
                st["places"] = list(path[:track])
                if g == 0:
                    st["done"] = True
            return
        if st["best"] is not None and g + cc * z >= st["best"]:
            return
        order, inc = S.row_order(v)
        level = len(path)
        for place, c in enumerate(order):
            if st["done"]:
                break
            if level < len(prefix) and place != prefix[level]:
                continue
            S.x[v] = c
            path.append(place)
            rec(g + inc[c])
            path.pop()
            S.x[v] = -1

    rec(0)
    return st["best"], st["bestx"], st["nodes"], st["hit"], st["found"], st["places"]


SPLIT_MAX_N = 4096   # larger instances are searched once with the whole budget


def split_cut(n, k, target=64):
    """Cut depth D (first depth with k^D >= target, at most n) and S = k^D."""
    D, S = 0, 1
    while S < target and D < n and D < 8:
        S *= k
        D += 1
    return D, S


def split_search(n, k, conf, stitch, cc=10, cs=1, budget=0, rule=0, target=64):
    """The budgeted split search, restated over the partial assignment.

    Every search gets b = ceil(budget / (S + 1)) nodes.  Phase 1 is the
    canonical search; if it ends on its own its answer stands.  Otherwise
    its incumbent (c1 in subtree s1, the number whose base-k digits are the
    row places of its leaf's first D levels) seeds one search per subtree s
    below the cut, each with the initial bound c1 + 1 if s < s1 else c1;
    the answer is the smallest (cost, subtree) among (c1, s1) and the
    subtrees' incumbents.  An instance of more than SPLIT_MAX_N segments is
    searched once with the whole budget.  Returns (cost, x, nodes,
    budget_hit).
    """
    if n > SPLIT_MAX_N:
        # not split: one search with the whole budget
        c, x, m, h = bounded_search(n, k, conf, stitch, cc, cs, budget=budget, rule=rule)
        return c, x, m, h
    D, S = split_cut(n, k, target)
    b = (budget + S) // (S + 1) if budget > 0 else 0
    c1, x1, nodes, hit, _, places = _search_with_prefix(n, k, conf, stitch, cc, cs, b, rule, (),
                                                        None, D)
    if not hit:
        return c1, x1, nodes, False
    s1 = 0
    for p in places:
        s1 = s1 * k + p
    win = (c1, s1, x1)
    any_hit = False
    for s in range(S):
        digits = []
        t = s
        for _ in range(D):
            digits.append(t % k)
            t //= k
        prefix = digits[::-1]
        c, x, m, h, found, _ = _search_with_prefix(n, k, conf, stitch, cc, cs, b, rule, prefix,
                                                   c1 + (1 if s < s1 else 0), 0)
        nodes += m
        any_hit = any_hit or h
        if found and (c, s) < win[:2]:
            win = (c, s, x)
    return win[0], win[2], nodes, any_hit


def units_of(n, polygon_of, stitch):
    """Unit of each segment: a polygon together with everything joined to it
    by stitch edges; a unit's id is its lowest segment."""
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    def unite(a, b):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)

    first = {}
    for s in range(n):
        p = polygon_of[s] if polygon_of is not None else s
        if p in first:
            unite(first[p], s)
        else:
            first[p] = s
    for a, b in stitch:
        unite(a, b)
    return [find(s) for s in range(n)]


def peel_order(n, k, conf, unit):
    """Removal order of the polygon-level k-core peel: FIFO queue seeded in
    ascending unit id; a unit with fewer than k conflict edges to remaining
    units is removed (its neighbours' counts drop and they join the queue when
    below k); a unit with a conflict edge inside itself is never removed."""
    edges = sorted({(min(a, b), max(a, b)) for a, b in conf if a != b})
    units = sorted(set(unit))
    deg = {u: 0 for u in units}
    selfc = set()
    for a, b in edges:
        ua, ub = unit[a], unit[b]
        if ua == ub:
            selfc.add(ua)
        else:
            deg[ua] += 1
            deg[ub] += 1
    cadj = adjacency(len(unit), edges)
    segs = {}
    for s_ in range(len(unit)):
        segs.setdefault(unit[s_], []).append(s_)
    queue = [u for u in units if u not in selfc and deg[u] < k]
    queued = set(queue)
    removed, order = set(), []
    h = 0
    while h < len(queue):
        u = queue[h]
        h += 1
        removed.add(u)
        order.append(u)
        # the unit's segments in ascending id, each one's neighbours ascending
        for s_ in segs[u]:
            for v in cadj[s_]:
                w = unit[v]
                if w == u or w in removed:
                    continue
                deg[w] -= 1
                if w not in queued and w not in selfc and deg[w] < k:
                    queue.append(w)
                    queued.add(w)
    return order


def density_balanced(n, k, conf, stitch, polygon_of, comp_of, inst_masks):
    """The density-balance rule written out: instances in order (ascending
    lowest segment) each take the mask permutation pairing their masks by
    decreasing segment count (lower mask first on ties) with the layout's
    masks so far by increasing count (lower first); then the removed units,
    in reverse removal order, take the least used of the masks their coloured
    conflict neighbours leave free (lowest on ties).  `inst_masks`: the
    search's masks on instance segments (-1 elsewhere)."""
    x = [-1] * n
    tot = [0] * k
    n_inst = max(comp_of) + 1 if len(comp_of) and max(comp_of) >= 0 else 0
    members = [[] for _ in range(n_inst)]
    for s in range(n):
        if comp_of[s] >= 0:
            members[comp_of[s]].append(s)
    for c in range(n_inst):
        cnt = [0] * k
        for s in members[c]:
            cnt[inst_masks[s]] += 1
        src = sorted(range(k), key=lambda m: (-cnt[m], m))
        dst = sorted(range(k), key=lambda m: (tot[m], m))
        perm = {src[i]: dst[i] for i in range(k)}
        for s in members[c]:
            x[s] = perm[inst_masks[s]]
        for m in range(k):
            tot[perm[m]] += cnt[m]
    unit = units_of(n, polygon_of, stitch)
    segs = {}
    for s in range(n):
        segs.setdefault(unit[s], []).append(s)
    cadj = adjacency(n, conf)
    for u in reversed(peel_order(n, k, conf, unit)):
        used = {x[w] for s in segs[u] for w in cadj[s] if x[w] >= 0}
        free = [m for m in range(k) if m not in used]
        c = min(free, key=lambda m: (tot[m], m))
        for s in segs[u]:
            x[s] = c
        tot[c] += len(segs[u])
    return x
