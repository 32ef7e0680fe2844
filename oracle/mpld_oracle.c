/*
 * mpld_oracle.c -- CPU oracle for the exact-cover (EC) layout decomposition
 * search of "GPU-Accelerated Matrix Cover Algorithm for Multiple Patterning
 * Layout Decomposition" (Chen, Yang, Yu).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never calls it and shares no code with it.
 *
 * What it computes
 * ----------------
 * Objective (Sec. 2.1, Eq. 1a-1d): for a graph with conflict edges CE and
 * stitch edges SE and k masks, minimise
 *     cost(x) = Cc * sum_{(i,j) in CE} [x_i == x_j] + Cs * sum_{(i,j) in SE} [x_i != x_j]
 * over x in {0..k-1}^n.  The paper writes the weights as 1 and alpha = 0.1;
 * integer weights Cc = 10, Cs = 1 are the same objective scaled by 10.
 *
 * Search (Sec. 2.3, Eq. 2, Algorithm 1): Knuth's Algorithm X with dancing
 * links over the EC matrix whose rows are (segment v, mask c), whose primary
 * column P_v must be covered exactly once and whose secondary column S_{e,c}
 * (conflict edge e, mask c) may be covered at most once.  Conflicts the
 * paper marks as "conflict candidates" (Algorithm 1, steps after the column
 * cover) are taken here as selectable inactive rows that pay their penalty,
 * which makes the search exact.  Stitch edges carry cost only; they have no
 * columns.
 *
 * Canonical order (the reading fixed here where the paper is silent):
 *   - node = one call of search(); the root counts;
 *   - leaf: every primary column covered; a leaf with cost g < best becomes
 *     the incumbent; best == 0 ends the search;
 *   - bound: Z = number of uncovered primary columns of size 0; prune when
 *     g + Cc * Z >= best (admissible: such a segment sees every mask taken by
 *     a distinct conflict neighbour, so it will pay at least Cc);
 *   - clique bound (optional, the second bound mode): the instance's
 *     (k+1)-cliques of conflict edges, enumerated in lexicographic order of
 *     their ascending member lists, are taken greedily when none of their
 *     edges is in a clique already taken.  Q = number of taken cliques whose
 *     members are all unassigned; prune when g + Cc * (Z + Q) >= best
 *     (admissible: k + 1 unassigned members of a clique must repeat a mask,
 *     on an edge between two unassigned segments, while Z's conflicts lie on
 *     edges to assigned segments, and taken cliques share no edge);
 *   - column, rule 0 (default): minimum size S, lowest segment index on
 *     ties (Knuth's S heuristic over a ring kept in index order);
 *   - column, rule 1 (the paper's rule, Algorithm 1: "a column with only
 *     one related row or in BFS order of G"): the lowest-index uncovered
 *     column with exactly one row left, else the uncovered column first in
 *     breadth-first order of the instance graph (conflict and stitch edges;
 *     roots in ascending id; neighbours in ascending id);
 *   - rows of the chosen segment v: all k masks, visited in ascending
 *     (inc(c), c) with inc(c) = Cc * #{conflict nbr u: x_u = c}
 *                            + Cs * #{stitch nbr u: x_u assigned, x_u != c};
 *   - node budget B > 0: once an incumbent exists and B nodes have been
 *     counted, the next call of search() stops the whole search (status
 *     BUDGET) and the incumbent is returned.  The first descent always
 *     reaches a leaf, so an incumbent always exists.
 * The answer is the first minimum-cost leaf in this depth-first order; no
 * admissible bound can change it, only the node count.
 *
 * Simplification (Sec. 2.2, the flow's simplify and recover steps; the
 * paper does not give the rule, this is the reading used): a unit is a
 * polygon together with every segment joined to it by a stitch edge.  Units
 * whose number of conflict edges to remaining units is below k are removed
 * in FIFO order (queue seeded in ascending unit id = lowest segment id; a
 * removal decrements its neighbours, which join the queue when they drop
 * below k).  A unit with a conflict edge inside itself is never removed.
 * Recovery walks the removal order backwards and gives all segments of a
 * unit the lowest mask not used by an already coloured conflict neighbour,
 * which costs nothing.  The remaining segments are split into connected
 * components (conflict + stitch edges), each searched on its own with
 * component-local ids in ascending global id.
 */
#define _POSIX_C_SOURCE 199309L   /* clock_gettime under -std=c11 */
#include <limits.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define OR_OK 0
#define OR_BUDGET 1
#define OR_E_INVALID (-1)
#define OR_E_OOM (-2)

#define OR_NO_SIMPLIFY 1u
#define OR_SINGLE_INSTANCE 2u
#define OR_COLUMN_BFS 8u
#define OR_BICONNECTED 16u
#define OR_CLIQUE_BOUND 32u
#define OR_SPLIT_BUDGET 64u
#define OR_DENSITY_BALANCE 128u

#define OR_INF INT64_MAX
#define OR_SPLIT_MAX_DEPTH 8

/* ------------------------------------------------------------------ */
/* Dancing-links matrix for one instance                                */
/* ------------------------------------------------------------------ */

typedef struct {
  int n, k, ne;
  int ncol;          /* 1 (root) + n primaries + k*ne secondaries */
  int nnode;
  int *L, *R, *U, *D, *C, *S;
  int *rownode;      /* node of row (v,c) in column P_v */
  char *covered;     /* secondary column covered flag */
  /* graph adjacency (for the row costs) */
  int *cptr, *cadj;  /* conflict neighbours */
  int *sptr, *sadj;  /* stitch neighbours */
  int64_t Cc, Cs;
  /* search state */
  signed char *x, *bestx;
  int64_t best, nodes, budget;
  int done, budget_hit;
  int *colstack;     /* columns covered by the rows on the current path */
  int coltop;
  int rule;          /* column rule: 0 fewest rows, 1 single row else BFS order */
  int *bfs_rank;     /* rule 1: breadth-first rank of each segment */
  int nq;            /* clique bound: taken cliques, k + 1 members each */
  int *qv;
  /* budgeted split search: the current call's level, the forced row places
   * of the levels above the cut, and the row places on the path of the
   * incumbent's leaf for the levels above `track` */
  int depth;
  int cut;
  int prefix[OR_SPLIT_MAX_DEPTH];
  int track;
  int path_pos[OR_SPLIT_MAX_DEPTH], best_pos[OR_SPLIT_MAX_DEPTH];
  int found;         /* a leaf became the incumbent in this search */
} dlx_t;

static void dlx_free(dlx_t *d) {
  free(d->L); free(d->R); free(d->U); free(d->D); free(d->C); free(d->S);
  free(d->rownode); free(d->covered);
  free(d->cptr); free(d->cadj); free(d->sptr); free(d->sadj);
  free(d->x); free(d->bestx); free(d->colstack); free(d->bfs_rank); free(d->qv);
  memset(d, 0, sizeof(*d));
}

/* CSR adjacency from an edge list (both directions), neighbours ascending. */
static int build_adj(int n, int m, const int *eu, const int *ev, int **ptr_out, int **adj_out) {
  int *ptr = calloc((size_t)n + 1, sizeof(int));
  int *adj = malloc(sizeof(int) * (size_t)(2 * m + 1));
  int *fill = calloc((size_t)n + 1, sizeof(int));
  if (!ptr || !adj || !fill) { free(ptr); free(adj); free(fill); return OR_E_OOM; }
  for (int e = 0; e < m; ++e) { ptr[eu[e] + 1]++; ptr[ev[e] + 1]++; }
  for (int v = 0; v < n; ++v) ptr[v + 1] += ptr[v];
  /* edges are sorted by (u, v) with u < v: scanning them in order and
   * appending gives each list in ascending neighbour order only for the
   * "v side"; sort each list afterwards (insertion sort, lists are short) */
  for (int e = 0; e < m; ++e) {
    adj[ptr[eu[e]] + fill[eu[e]]++] = ev[e];
    adj[ptr[ev[e]] + fill[ev[e]]++] = eu[e];
  }
  for (int v = 0; v < n; ++v) {
    for (int i = ptr[v] + 1; i < ptr[v + 1]; ++i) {
      int t = adj[i], j = i - 1;
      while (j >= ptr[v] && adj[j] > t) { adj[j + 1] = adj[j]; --j; }
      adj[j + 1] = t;
    }
  }
  free(fill);
  *ptr_out = ptr;
  *adj_out = adj;
  return OR_OK;
}

/* Breadth-first rank of every segment over conflict and stitch edges:
 * roots in ascending id, each segment's neighbours in ascending id (a
 * neighbour by both kinds of edge once). */
static int bfs_ranks(int n, const int *cptr, const int *cadj, const int *sptr, const int *sadj,
                     int **out) {
  int *rank = malloc(sizeof(int) * (size_t)(n + 1));
  int *queue = malloc(sizeof(int) * (size_t)(n + 1));
  if (!rank || !queue) { free(rank); free(queue); return OR_E_OOM; }
  for (int v = 0; v < n; ++v) rank[v] = -1;
  int next = 0;
  for (int r = 0; r < n; ++r) {
    if (rank[r] >= 0) continue;
    int qh = 0, qt = 0;
    rank[r] = next++;
    queue[qt++] = r;
    while (qh < qt) {
      const int u = queue[qh++];
      int i = cptr[u], j = sptr[u];
      while (i < cptr[u + 1] || j < sptr[u + 1]) {
        int w;
        if (j >= sptr[u + 1] || (i < cptr[u + 1] && cadj[i] <= sadj[j])) {
          w = cadj[i++];
          if (j < sptr[u + 1] && sadj[j] == w) ++j;
        } else {
          w = sadj[j++];
        }
        if (rank[w] < 0) { rank[w] = next++; queue[qt++] = w; }
      }
    }
  }
  free(queue);
  *out = rank;
  return OR_OK;
}

/* Build the EC matrix.  Columns: 0 = root, 1+v = P_v, 1+n+e*k+c = S_{e,c}.
 * Row (v,c) has a node in P_v and one in S_{e,c} for every conflict edge e
 * incident to v, in ascending e; rows are appended in ascending v*k+c, so
 * every column lists its rows in ascending row index. */
static int dlx_build(dlx_t *d, int n, int k, int ne, const int *eu, const int *ev,
                     int ns, const int *su, const int *sv, int64_t Cc, int64_t Cs) {
  memset(d, 0, sizeof(*d));
  d->n = n; d->k = k; d->ne = ne; d->Cc = Cc; d->Cs = Cs;
  d->ncol = 1 + n + k * ne;
  d->nnode = d->ncol + k * (n + 2 * ne);
  size_t nn = (size_t)d->nnode;
  d->L = malloc(nn * sizeof(int)); d->R = malloc(nn * sizeof(int));
  d->U = malloc(nn * sizeof(int)); d->D = malloc(nn * sizeof(int));
  d->C = malloc(nn * sizeof(int)); d->S = calloc((size_t)d->ncol, sizeof(int));
  d->rownode = malloc(sizeof(int) * (size_t)(n * k + 1));
  d->covered = calloc((size_t)d->ncol, 1);
  d->x = malloc((size_t)n + 1); d->bestx = malloc((size_t)n + 1);
  d->colstack = malloc(sizeof(int) * (size_t)(k * ne + 1));
  if (!d->L || !d->R || !d->U || !d->D || !d->C || !d->S || !d->rownode || !d->covered ||
      !d->x || !d->bestx || !d->colstack) { dlx_free(d); return OR_E_OOM; }
  if (build_adj(n, ne, eu, ev, &d->cptr, &d->cadj) != OR_OK ||
      build_adj(n, ns, su, sv, &d->sptr, &d->sadj) != OR_OK) { dlx_free(d); return OR_E_OOM; }

  /* headers */
  for (int c = 0; c < d->ncol; ++c) { d->U[c] = d->D[c] = c; d->C[c] = c; }
  /* ring: root and the primaries in index order */
  for (int c = 0; c <= n; ++c) { d->R[c] = (c == n) ? 0 : c + 1; d->L[c] = (c == 0) ? n : c - 1; }
  /* secondaries stay out of the ring */
  for (int c = n + 1; c < d->ncol; ++c) { d->L[c] = d->R[c] = c; }

  /* incident edge lists in ascending edge index */
  int *iptr = calloc((size_t)n + 1, sizeof(int));
  int *iedge = malloc(sizeof(int) * (size_t)(2 * ne + 1));
  int *ifill = calloc((size_t)n + 1, sizeof(int));
  if (!iptr || !iedge || !ifill) { free(iptr); free(iedge); free(ifill); dlx_free(d); return OR_E_OOM; }
  for (int e = 0; e < ne; ++e) { iptr[eu[e] + 1]++; iptr[ev[e] + 1]++; }
  for (int v = 0; v < n; ++v) iptr[v + 1] += iptr[v];
  for (int e = 0; e < ne; ++e) {
    iedge[iptr[eu[e]] + ifill[eu[e]]++] = e;
    iedge[iptr[ev[e]] + ifill[ev[e]]++] = e;
  }

  int next = d->ncol;
  for (int v = 0; v < n; ++v) {
    for (int c = 0; c < k; ++c) {
      int first = -1, prev = -1;
      int ncols_row = 1 + (iptr[v + 1] - iptr[v]);
      for (int t = 0; t < ncols_row; ++t) {
        int col = (t == 0) ? 1 + v : 1 + n + iedge[iptr[v] + t - 1] * k + c;
        int node = next++;
        d->C[node] = col;
        /* vertical: append at the bottom of the column */
        d->U[node] = d->U[col]; d->D[node] = col;
        d->D[d->U[col]] = node; d->U[col] = node;
        d->S[col]++;
        /* horizontal: append to the row's circular list */
        if (first < 0) { first = node; d->L[node] = d->R[node] = node; }
        else { d->L[node] = prev; d->R[node] = first; d->R[prev] = node; d->L[first] = node; }
        prev = node;
      }
      d->rownode[v * k + c] = first;
    }
  }
  free(iptr); free(iedge); free(ifill);
  for (int v = 0; v < n; ++v) d->x[v] = -1;
  d->best = OR_INF;
  return OR_OK;
}

/* Knuth's cover / uncover (Eq. 2). */
static void dlx_cover(dlx_t *d, int c) {
  int *L = d->L, *R = d->R, *U = d->U, *D = d->D, *C = d->C, *S = d->S;
  L[R[c]] = L[c];
  R[L[c]] = R[c];
  for (int i = D[c]; i != c; i = D[i])
    for (int j = R[i]; j != i; j = R[j]) {
      U[D[j]] = U[j];
      D[U[j]] = D[j];
      S[C[j]]--;
    }
}

static void dlx_uncover(dlx_t *d, int c) {
  int *L = d->L, *R = d->R, *U = d->U, *D = d->D, *C = d->C, *S = d->S;
  for (int i = U[c]; i != c; i = U[i])
    for (int j = L[i]; j != i; j = L[j]) {
      S[C[j]]++;
      U[D[j]] = j;
      D[U[j]] = j;
    }
  L[R[c]] = c;
  R[L[c]] = c;
}

/* Cost added by giving segment v mask c, against the current assignment. */
static int64_t row_inc(const dlx_t *d, int v, int c) {
  int64_t inc = 0;
  for (int i = d->cptr[v]; i < d->cptr[v + 1]; ++i)
    if (d->x[d->cadj[i]] == c) inc += d->Cc;
  for (int i = d->sptr[v]; i < d->sptr[v + 1]; ++i) {
    int xs = d->x[d->sadj[i]];
    if (xs >= 0 && xs != c) inc += d->Cs;
  }
  return inc;
}

static void dlx_search(dlx_t *d, int64_t g) {
  if (d->budget > 0 && d->best < OR_INF && d->nodes >= d->budget) {
    d->budget_hit = 1;
    d->done = 1;
    return;
  }
  d->nodes++;
  if (d->R[0] == 0) {                      /* every primary column covered */
    if (g < d->best) {
      d->best = g;
      d->found = 1;
      memcpy(d->bestx, d->x, (size_t)d->n);
      memcpy(d->best_pos, d->path_pos, sizeof(int) * (size_t)d->track);
      if (g == 0) d->done = 1;
    }
    return;
  }
  int64_t Z = 0;
  int cmin = 0, smin = INT_MAX;
  for (int c = d->R[0]; c != 0; c = d->R[c]) {
    if (d->S[c] == 0) Z++;
    if (d->rule == 0) {
      if (d->S[c] < smin) { smin = d->S[c]; cmin = c; }
    } else if (smin != 1) {
      /* first single-row column in index order, else lowest BFS rank */
      if (d->S[c] == 1) { smin = 1; cmin = c; }
      else if (cmin == 0 || d->bfs_rank[c - 1] < d->bfs_rank[cmin - 1]) cmin = c;
    }
  }
  int64_t Q = 0;                           /* taken cliques with no member assigned */
  for (int q = 0; q < d->nq; ++q) {
    int all = 1;
    for (int i = 0; i <= d->k && all; ++i) all = d->x[d->qv[q * (d->k + 1) + i]] < 0;
    Q += all;
  }
  if (g + d->Cc * (Z + Q) >= d->best) return;    /* admissible bound */

  const int v = cmin - 1, k = d->k;
  int64_t inc[8];
  int order[8];
  for (int c = 0; c < k; ++c) inc[c] = row_inc(d, v, c);
  for (int c = 0; c < k; ++c) {            /* insertion sort by (inc, c) */
    int j = c - 1;
    while (j >= 0 && inc[order[j]] > inc[c]) { order[j + 1] = order[j]; --j; }
    order[j + 1] = c;
  }

  dlx_cover(d, cmin);
  for (int t = 0; t < k && !d->done; ++t) {
    /* above the cut of a split search only the forced row is taken */
    if (d->depth < d->cut && t != d->prefix[d->depth]) continue;
    if (d->depth < d->track) d->path_pos[d->depth] = t;
    const int c = order[t];
    const int r = d->rownode[v * k + c];
    const int base = d->coltop;
    for (int j = d->R[r]; j != r; j = d->R[j]) {
      int col = d->C[j];
      if (!d->covered[col]) {              /* skip columns a neighbour took */
        dlx_cover(d, col);
        d->covered[col] = 1;
        d->colstack[d->coltop++] = col;
      }
    }
    d->x[v] = (signed char)c;
    d->depth++;
    dlx_search(d, g + inc[c]);
    d->depth--;
    d->x[v] = -1;
    while (d->coltop > base) {
      int col = d->colstack[--d->coltop];
      d->covered[col] = 0;
      dlx_uncover(d, col);
    }
  }
  dlx_uncover(d, cmin);
}

/* Textbook Algorithm X: count exact covers (active rows only). */
static void dlx_count(dlx_t *d, int64_t limit, int64_t *count) {
  if (*count >= limit) return;
  if (d->R[0] == 0) { (*count)++; return; }
  int cmin = 0, smin = INT_MAX;
  for (int c = d->R[0]; c != 0; c = d->R[c])
    if (d->S[c] < smin) { smin = d->S[c]; cmin = c; }
  if (smin == 0) return;
  dlx_cover(d, cmin);
  for (int r = d->D[cmin]; r != cmin; r = d->D[r]) {
    for (int j = d->R[r]; j != r; j = d->R[j]) dlx_cover(d, d->C[j]);
    dlx_count(d, limit, count);
    for (int j = d->L[r]; j != r; j = d->L[j]) dlx_uncover(d, d->C[j]);
  }
  dlx_uncover(d, cmin);
}

/* ------------------------------------------------------------------ */
/* Input validation and normalisation                                   */
/* ------------------------------------------------------------------ */

static int cmp_pair(const void *a, const void *b) {
  const int *p = a, *q = b;
  if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
  if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
  return 0;
}

/* (min,max)-normalised, sorted, de-duplicated copy of an edge list. */
static int norm_edges(int n, int m, const int *u, const int *v, int **ou, int **ov, int *om) {
  int *pairs = malloc(sizeof(int) * (size_t)(2 * m + 2));
  if (!pairs) return OR_E_OOM;
  for (int e = 0; e < m; ++e) {
    int a = u[e], b = v[e];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) { free(pairs); return OR_E_INVALID; }
    pairs[2 * e] = a < b ? a : b;
    pairs[2 * e + 1] = a < b ? b : a;
  }
  qsort(pairs, (size_t)m, 2 * sizeof(int), cmp_pair);
  int w = 0;
  for (int e = 0; e < m; ++e) {
    if (w > 0 && pairs[2 * (w - 1)] == pairs[2 * e] && pairs[2 * (w - 1) + 1] == pairs[2 * e + 1]) continue;
    pairs[2 * w] = pairs[2 * e];
    pairs[2 * w + 1] = pairs[2 * e + 1];
    ++w;
  }
  *ou = malloc(sizeof(int) * (size_t)(w + 1));
  *ov = malloc(sizeof(int) * (size_t)(w + 1));
  if (!*ou || !*ov) { free(pairs); free(*ou); free(*ov); return OR_E_OOM; }
  for (int e = 0; e < w; ++e) { (*ou)[e] = pairs[2 * e]; (*ov)[e] = pairs[2 * e + 1]; }
  *om = w;
  free(pairs);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Single-instance entry points                                         */
/* ------------------------------------------------------------------ */

/* Search one instance (the whole given graph, connected or not).
 * x_out: n masks; returns OR_OK / OR_BUDGET / error. */
/* Greedy edge-disjoint (k+1)-cliques of the conflict graph: every clique in
 * lexicographic order of its ascending member list, taken when none of its
 * edges is in a clique already taken. */
static int edge_slot(const dlx_t *d, int a, int b) {   /* adjacency entry of b in a's list */
  int lo = d->cptr[a], hi = d->cptr[a + 1];
  while (lo < hi) {
    int mid = lo + (hi - lo) / 2;
    if (d->cadj[mid] < b) lo = mid + 1;
    else hi = mid;
  }
  return (lo < d->cptr[a + 1] && d->cadj[lo] == b) ? lo : -1;
}
static int clique_extend(dlx_t *d, int *cur, int depth, char *used, int *cap) {
  const int K = d->k + 1;
  if (depth == K) {
    for (int i = 0; i < K; ++i)
      for (int j = i + 1; j < K; ++j)
        if (used[edge_slot(d, cur[i], cur[j])]) return OR_OK;
    for (int i = 0; i < K; ++i)
      for (int j = i + 1; j < K; ++j) {
        used[edge_slot(d, cur[i], cur[j])] = 1;
        used[edge_slot(d, cur[j], cur[i])] = 1;
      }
    if (d->nq == *cap) {
      int nc = *cap * 2 + 8;
      int *nv = realloc(d->qv, sizeof(int) * (size_t)nc * (size_t)K);
      if (!nv) return OR_E_OOM;
      d->qv = nv;
      *cap = nc;
    }
    memcpy(d->qv + (size_t)d->nq * (size_t)K, cur, sizeof(int) * (size_t)K);
    d->nq++;
    return OR_OK;
  }
  const int last = cur[depth - 1];
  for (int i = d->cptr[last]; i < d->cptr[last + 1]; ++i) {
    const int w = d->cadj[i];
    if (w <= last) continue;
    int ok = 1;
    for (int j = 0; j < depth - 1 && ok; ++j) ok = edge_slot(d, cur[j], w) >= 0;
    if (!ok) continue;
    cur[depth] = w;
    int rc = clique_extend(d, cur, depth + 1, used, cap);
    if (rc != OR_OK) return rc;
  }
  return OR_OK;
}
static int build_cliques(dlx_t *d) {
  char *used = calloc((size_t)d->cptr[d->n] + 1, 1);
  if (!used) return OR_E_OOM;
  int cur[9], cap = 0, rc = OR_OK;
  for (int v = 0; v < d->n && rc == OR_OK; ++v) {
    cur[0] = v;
    rc = clique_extend(d, cur, 1, used, &cap);
  }
  free(used);
  return rc;
}

/* Taken cliques of an instance (for tests): writes up to max_q * (k + 1)
 * member ids; returns the number of cliques. */
int oracle_cliques(int n, int k, int ne, const int *eu, const int *ev, int max_q, int *out) {
  if (n < 0 || k < 2 || k > 8 || ne < 0) return OR_E_INVALID;
  int *cu, *cv, mc, rc;
  if ((rc = norm_edges(n, ne, eu, ev, &cu, &cv, &mc)) != OR_OK) return rc;
  dlx_t d;
  rc = dlx_build(&d, n, k, mc, cu, cv, 0, NULL, NULL, 10, 1);
  free(cu); free(cv);
  if (rc != OR_OK) return rc;
  rc = build_cliques(&d);
  if (rc == OR_OK) {
    int m = d.nq < max_q ? d.nq : max_q;
    if (m > 0) memcpy(out, d.qv, sizeof(int) * (size_t)m * (size_t)(k + 1));
    rc = d.nq;
  }
  dlx_free(&d);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Budgeted split search                                                 */
/* ------------------------------------------------------------------ */

/* A node budget spent by one depth-first search is sequential: which nodes
 * the first B are depends on every node before them.  The split search
 * spends it on many independent searches instead (the paper's task
 * parallelism, Sec. 1 and Sec. 2.3, applied inside one sub-graph):
 *   - the canonical tree is cut at depth D, the first depth with
 *     k^D >= OR_SPLIT_TARGET (at most n); subtree s (0 <= s < S = k^D) is
 *     the set of nodes whose path takes, at level i < D, the row at place
 *     digit i of s in base k (most significant first) of the ascending
 *     (added cost, mask) order, so subtree numbers follow the depth-first
 *     order of the whole tree;
 *   - every search gets b = ceil(B / (S + 1)) nodes;
 *   - phase 1 is the canonical search with budget b.  If it ends on its
 *     own, its answer stands (the first minimum-cost leaf);
 *   - otherwise its incumbent (c1, at subtree s1) seeds S subtree searches.
 *     The search of subtree s is the canonical search restricted to s,
 *     counting the nodes on its forced path, with budget b and an initial
 *     bound of c1 + 1 if s < s1, else c1: a leaf of subtree s is taken
 *     when it beats (c1, s1) in the order (cost, subtree);
 *   - the answer is the smallest (cost, subtree) over (c1, s1) and the
 *     subtrees' incumbents, with that leaf's masks; the nodes are phase 1's
 *     plus every subtree's; the status is BUDGET if some subtree stopped on
 *     its budget.  When none did, every subtree was searched to the end
 *     and the answer is the first minimum-cost leaf of the whole tree, as
 *     an exhaustive search gives;
 *   - an instance of more than OR_SPLIT_MAX_N segments is not split: every
 *     subtree search would first descend through all its levels, so it is
 *     searched once with the whole budget B.
 * Each search depends on nothing but its own subtree and (c1, s1), so the
 * result does not depend on the order the searches run in. */
#ifndef OR_SPLIT_TARGET
#define OR_SPLIT_TARGET 64
#endif
#define OR_SPLIT_MAX_N 4096

static void split_cut(int n, int k, int *D_out, int64_t *S_out) {
  int D = 0;
  int64_t S = 1;
  while (S < OR_SPLIT_TARGET && D < n && D < OR_SPLIT_MAX_DEPTH) { S *= k; ++D; }
  *D_out = D;
  *S_out = S;
}

static int dlx_split_search(dlx_t *d, int64_t budget) {
  const int n = d->n, k = d->k;
  if (n > OR_SPLIT_MAX_N) {
    d->budget = budget;
    dlx_search(d, 0);
    return d->budget_hit ? OR_BUDGET : OR_OK;
  }
  int D;
  int64_t S;
  split_cut(n, k, &D, &S);
  const int64_t b = budget > 0 ? (budget + S) / (S + 1) : 0;   /* ceil(B / (S + 1)) */
  /* phase 1 */
  d->budget = b; d->cut = 0; d->track = D; d->depth = 0; d->found = 0;
  dlx_search(d, 0);
  int64_t nodes = d->nodes;
  if (!d->budget_hit) return OR_OK;
  const int64_t c1 = d->best;
  int64_t s1 = 0;
  for (int i = 0; i < D; ++i) s1 = s1 * k + d->best_pos[i];
  int64_t cw = c1, sw = s1;
  signed char *xw = malloc((size_t)n + 1);
  if (!xw) return OR_E_OOM;
  memcpy(xw, d->bestx, (size_t)n);
  int any_budget = 0;
  /* phase 2: the subtrees, each on its own */
  for (int64_t s = 0; s < S; ++s) {
    d->best = c1 + (s < s1 ? 1 : 0);
    d->found = 0; d->nodes = 0; d->done = 0; d->budget_hit = 0;
    d->budget = b; d->cut = D; d->track = 0; d->depth = 0;
    int64_t t = s;
    for (int i = D - 1; i >= 0; --i) { d->prefix[i] = (int)(t % k); t /= k; }
    dlx_search(d, 0);
    nodes += d->nodes;
    any_budget |= d->budget_hit;
    if (d->found && (d->best < cw || (d->best == cw && s < sw))) {
      cw = d->best;
      sw = s;
      memcpy(xw, d->bestx, (size_t)n);
    }
  }
  d->best = cw;
  memcpy(d->bestx, xw, (size_t)n);
  d->nodes = nodes;
  d->budget_hit = any_budget;
  d->cut = 0;
  free(xw);
  return any_budget ? OR_BUDGET : OR_OK;
}

int oracle_solve_instance_rule(int n, int k, int ne, const int *eu, const int *ev,
                               int ns, const int *su, const int *sv,
                               int64_t cost_conflict, int64_t cost_stitch, int64_t budget, int rule,
                               signed char *x_out, int64_t *cost_out, int64_t *nodes_out) {
  /* bit 0: column rule, bit 1: clique bound, bit 2: budgeted split search */
  if (rule < 0 || rule > 7) return OR_E_INVALID;
  if (n < 0 || k < 2 || k > 8 || ne < 0 || ns < 0) return OR_E_INVALID;
  int *cu, *cv, *tu, *tv, mc, ms, rc;
  if ((rc = norm_edges(n, ne, eu, ev, &cu, &cv, &mc)) != OR_OK) return rc;
  if ((rc = norm_edges(n, ns, su, sv, &tu, &tv, &ms)) != OR_OK) { free(cu); free(cv); return rc; }
  dlx_t d;
  rc = dlx_build(&d, n, k, mc, cu, cv, ms, tu, tv, cost_conflict, cost_stitch);
  free(cu); free(cv); free(tu); free(tv);
  if (rc != OR_OK) return rc;
  d.budget = budget;
  d.rule = rule & 1;
  if (d.rule == 1 && bfs_ranks(n, d.cptr, d.cadj, d.sptr, d.sadj, &d.bfs_rank) != OR_OK) {
    dlx_free(&d);
    return OR_E_OOM;
  }
  if ((rule & 2) && build_cliques(&d) != OR_OK) {
    dlx_free(&d);
    return OR_E_OOM;
  }
  if (rule & 4) {
    rc = dlx_split_search(&d, budget);
    if (rc < 0) { dlx_free(&d); return rc; }
  } else {
    dlx_search(&d, 0);
  }
  memcpy(x_out, d.bestx, (size_t)n);
  *cost_out = d.best;
  *nodes_out = d.nodes;
  rc = d.budget_hit ? OR_BUDGET : OR_OK;
  dlx_free(&d);
  return rc;
}

int oracle_solve_instance(int n, int k, int ne, const int *eu, const int *ev,
                          int ns, const int *su, const int *sv,
                          int64_t cost_conflict, int64_t cost_stitch, int64_t budget,
                          signed char *x_out, int64_t *cost_out, int64_t *nodes_out) {
  return oracle_solve_instance_rule(n, k, ne, eu, ev, ns, su, sv, cost_conflict, cost_stitch,
                                    budget, 0, x_out, cost_out, nodes_out);
}

/* Number of exact covers of the EC matrix (primary columns exactly once,
 * secondary columns at most once), stopping at `limit`. */
int oracle_count_exact_covers(int n, int k, int ne, const int *eu, const int *ev,
                              int64_t limit, int64_t *count_out) {
  if (n < 0 || k < 2 || k > 8 || ne < 0) return OR_E_INVALID;
  int *cu, *cv, mc, rc;
  if ((rc = norm_edges(n, ne, eu, ev, &cu, &cv, &mc)) != OR_OK) return rc;
  dlx_t d;
  rc = dlx_build(&d, n, k, mc, cu, cv, 0, NULL, NULL, 10, 1);
  free(cu); free(cv);
  if (rc != OR_OK) return rc;
  int64_t cnt = 0;
  dlx_count(&d, limit, &cnt);
  *count_out = cnt;
  dlx_free(&d);
  return OR_OK;
}

/* The EC matrix as a dense 0/1 array, row-major [n*k][1 + n + k*ne]
 * (column 0, the root, stays 0), read back from the dancing links. */
int oracle_export_matrix(int n, int k, int ne, const int *eu, const int *ev, unsigned char *dense) {
  if (n < 0 || k < 2 || k > 8 || ne < 0) return OR_E_INVALID;
  int *cu, *cv, mc, rc;
  if ((rc = norm_edges(n, ne, eu, ev, &cu, &cv, &mc)) != OR_OK) return rc;
  dlx_t d;
  rc = dlx_build(&d, n, k, mc, cu, cv, 0, NULL, NULL, 10, 1);
  free(cu); free(cv);
  if (rc != OR_OK) return rc;
  const size_t ncol = (size_t)d.ncol;
  memset(dense, 0, (size_t)n * (size_t)k * ncol);
  for (int row = 0; row < n * k; ++row) {
    int r = d.rownode[row];
    int j = r;
    do { dense[(size_t)row * ncol + (size_t)d.C[j]] = 1; j = d.R[j]; } while (j != r);
  }
  dlx_free(&d);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Whole-layout decomposition: simplify, split, search, recover          */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t n_components, n_removed_segments;
  int64_t n_conflicts, n_stitches, cost, nodes;
  int64_t component_cost_sum, n_budget_components;
  int32_t status, max_component;
  /* timing of the search phase alone (the instances' matrices built and
   * searched on the thread pool), for throughput figures; not part of the
   * result */
  double search_seconds;
  int64_t instance_segments;   /* segments inside search instances */
} oracle_totals;

static double wall_seconds(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

typedef struct {
  /* shared, read-only */
  int k, n_comp, rule;
  int64_t Cc, Cs, budget;
  const int *comp_ptr, *comp_seg;     /* segments of instance i, ascending */
  const int *cptr, *cadj, *sptr, *sadj; /* global adjacency */
  const int *work_order;              /* instances by descending size */
  /* outputs */
  signed char *imask;                 /* per instance entry (comp_ptr order) */
  int64_t *comp_cost, *comp_nodes;
  int32_t *comp_status;
  atomic_int next;
  atomic_int error;
} pool_t;

/* local id of global segment g in the sorted list seg[0..n), or -1 */
static int local_id(const int *seg, int n, int g) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = lo + (hi - lo) / 2;
    if (seg[mid] < g) lo = mid + 1;
    else hi = mid;
  }
  return (lo < n && seg[lo] == g) ? lo : -1;
}

/* Search instance ci: its segments are the sorted list comp_seg[a..b), its
 * edges every conflict / stitch edge with both ends among them. */
static void solve_component(pool_t *P, int ci) {
  const int a = P->comp_ptr[ci], b = P->comp_ptr[ci + 1], n = b - a;
  const int *seg = P->comp_seg + a;
  int ne = 0, ns = 0;
  for (int t = 0; t < n; ++t) {
    int g = seg[t];
    for (int i = P->cptr[g]; i < P->cptr[g + 1]; ++i)
      if (P->cadj[i] > g && local_id(seg, n, P->cadj[i]) >= 0) ne++;
    for (int i = P->sptr[g]; i < P->sptr[g + 1]; ++i)
      if (P->sadj[i] > g && local_id(seg, n, P->sadj[i]) >= 0) ns++;
  }
  int *eu = malloc(sizeof(int) * (size_t)(ne + 1)), *ev = malloc(sizeof(int) * (size_t)(ne + 1));
  int *su = malloc(sizeof(int) * (size_t)(ns + 1)), *sv = malloc(sizeof(int) * (size_t)(ns + 1));
  signed char *x = malloc((size_t)n + 1);
  if (!eu || !ev || !su || !sv || !x) { atomic_store(&P->error, OR_E_OOM); goto out; }
  ne = ns = 0;
  for (int t = 0; t < n; ++t) {
    int g = seg[t];
    for (int i = P->cptr[g]; i < P->cptr[g + 1]; ++i) {
      int l = P->cadj[i] > g ? local_id(seg, n, P->cadj[i]) : -1;
      if (l >= 0) { eu[ne] = t; ev[ne] = l; ne++; }
    }
    for (int i = P->sptr[g]; i < P->sptr[g + 1]; ++i) {
      int l = P->sadj[i] > g ? local_id(seg, n, P->sadj[i]) : -1;
      if (l >= 0) { su[ns] = t; sv[ns] = l; ns++; }
    }
  }
  int64_t cost = 0, nodes = 0;
  int rc = oracle_solve_instance_rule(n, P->k, ne, eu, ev, ns, su, sv, P->Cc, P->Cs, P->budget,
                                      P->rule, x, &cost, &nodes);
  if (rc < 0) { atomic_store(&P->error, rc); goto out; }
  memcpy(P->imask + a, x, (size_t)n);
  P->comp_cost[ci] = cost;
  P->comp_nodes[ci] = nodes;
  P->comp_status[ci] = rc;
out:
  free(eu); free(ev); free(su); free(sv); free(x);
}

static void *pool_worker(void *arg) {
  pool_t *P = arg;
  for (;;) {
    int i = atomic_fetch_add(&P->next, 1);
    if (i >= P->n_comp || atomic_load(&P->error)) break;
    solve_component(P, P->work_order[i]);
  }
  return NULL;
}

/* (size, id) pairs: larger components first, then ascending id */
static int cmp_comp(const void *a, const void *b) {
  const int *p = a, *q = b;
  if (p[0] != q[0]) return p[0] > q[0] ? -1 : 1;
  return p[1] < q[1] ? -1 : (p[1] > q[1]);
}

static int find_root(int *parent, int a) {
  while (parent[a] != a) { parent[a] = parent[parent[a]]; a = parent[a]; }
  return a;
}

/*
 * Decompose a whole layout.
 *   polygon_of: segment -> polygon id in [0, n_seg), or NULL (each segment
 *               its own polygon);
 *   flags: OR_NO_SIMPLIFY, OR_SINGLE_INSTANCE, OR_COLUMN_BFS (column rule 1);
 *   nthreads: worker threads for the per-component searches (>= 1);
 *   mask_out[n_seg]; comp_of_out[n_seg] (nullable): component of each
 *   segment, -1 if removed by simplification; comp_nodes_out /
 *   comp_cost_out / comp_status_out (nullable, n_seg entries each).
 */
/* ------------------------------------------------------------------ */
/* Biconnected blocks of one component (the flow's optional split)      */
/* ------------------------------------------------------------------ */

/* A block is a maximal 2-connected piece of the component's graph
 * (conflict and stitch edges together); a bridge is a block of two, and a
 * component without edges is one block of one segment.  Computed from a
 * plain characterisation: two edges (v, a) and (v, b) at a vertex v lie in
 * one block exactly when a and b are still connected once v is removed;
 * blocks are the classes of the transitive closure of that relation.
 *
 * Canonical order: the blocks are visited breadth-first over the
 * block-cut tree.  The first is, among the blocks holding the component's
 * lowest segment, the one whose ascending segment list is lexicographically
 * smallest.  From a visited block, its segments are taken in ascending id,
 * and each unvisited block holding that segment is visited next (blocks in
 * lexicographic order of their segment lists), attached at that segment.
 * The merge gives a block's solution the transposition of masks that makes
 * its attach segment agree with the mask it already has; cost is unchanged
 * by renaming masks, and each edge lies in exactly one block. */

typedef struct { int *v; int n; } vlist_t;

static int lex_cmp(const vlist_t *x, const vlist_t *y) {
  int m = x->n < y->n ? x->n : y->n;
  for (int i = 0; i < m; ++i)
    if (x->v[i] != y->v[i]) return x->v[i] < y->v[i] ? -1 : 1;
  return x->n < y->n ? -1 : x->n > y->n ? 1 : 0;
}
static int find_uf(int *p, int a) {
  while (p[a] != a) { p[a] = p[p[a]]; a = p[a]; }
  return a;
}

/* Append the blocks of component seg[0..n) (ascending global ids) in
 * canonical order: segments to *out_seg (grown), block boundaries to
 * *out_ptr, attach segments (global id, -1 for the first) to *out_att. */
static int component_blocks(const int *seg, int n, const int *cptr, const int *cadj,
                            const int *sptr, const int *sadj, int **out_ptr, int **out_seg,
                            int **out_att, int *n_out, int *cap_blocks, int *len_seg,
                            int *cap_seg) {
  int rc = OR_E_OOM;
  /* local adjacency: union of conflict and stitch neighbours inside */
  int *deg = calloc((size_t)n + 1, sizeof(int)), *lptr = NULL, *ladj = NULL;
  int *eid = NULL, *ea = NULL, *eb = NULL, *uf = NULL, *lab = NULL, *stack = NULL;
  int *bid = NULL, *mark = NULL, *bcount = NULL, *order = NULL, *visited = NULL, *queue = NULL;
  int *attach = NULL, *vb_ptr = NULL, *vb = NULL;
  vlist_t *blocks = NULL;
  int nb = 0, ne = 0;
  if (!deg) goto done;
  for (int t = 0; t < n; ++t) {
    int g = seg[t], i = cptr[g], j = sptr[g];
    while (i < cptr[g + 1] || j < sptr[g + 1]) {
      int w;
      if (j >= sptr[g + 1] || (i < cptr[g + 1] && cadj[i] <= sadj[j])) {
        w = cadj[i++];
        if (j < sptr[g + 1] && sadj[j] == w) ++j;
      } else w = sadj[j++];
      if (local_id(seg, n, w) >= 0) deg[t]++;
    }
  }
  lptr = calloc((size_t)n + 1, sizeof(int));
  if (!lptr) goto done;
  for (int t = 0; t < n; ++t) lptr[t + 1] = lptr[t] + deg[t];
  ladj = malloc(sizeof(int) * (size_t)(lptr[n] + 1));
  eid = malloc(sizeof(int) * (size_t)(lptr[n] + 1));
  if (!ladj || !eid) goto done;
  for (int t = 0, f = 0; t < n; ++t) {
    int g = seg[t], i = cptr[g], j = sptr[g];
    while (i < cptr[g + 1] || j < sptr[g + 1]) {
      int w;
      if (j >= sptr[g + 1] || (i < cptr[g + 1] && cadj[i] <= sadj[j])) {
        w = cadj[i++];
        if (j < sptr[g + 1] && sadj[j] == w) ++j;
      } else w = sadj[j++];
      int l = local_id(seg, n, w);
      if (l >= 0) ladj[f++] = l;
    }
  }
  /* edge ids: edge (t, l) with t < l gets the next id; the reverse entry shares it */
  ne = lptr[n] / 2;
  ea = malloc(sizeof(int) * (size_t)(ne + 1));
  eb = malloc(sizeof(int) * (size_t)(ne + 1));
  uf = malloc(sizeof(int) * (size_t)(ne + 1));
  if (!ea || !eb || !uf) goto done;
  for (int t = 0, e = 0; t < n; ++t)
    for (int i = lptr[t]; i < lptr[t + 1]; ++i)
      if (ladj[i] > t) { eid[i] = e; ea[e] = t; eb[e] = ladj[i]; uf[e] = e; ++e; }
  for (int t = 0; t < n; ++t)
    for (int i = lptr[t]; i < lptr[t + 1]; ++i)
      if (ladj[i] < t) {
        int u = ladj[i];
        for (int j = lptr[u]; j < lptr[u + 1]; ++j)
          if (ladj[j] == t) { eid[i] = eid[j]; break; }
      }
  /* for every v: components of the graph without v; join v's edges whose
   * other ends share one */
  lab = malloc(sizeof(int) * (size_t)(n + 1));
  stack = malloc(sizeof(int) * (size_t)(n + 1));
  if (!lab || !stack) goto done;
  for (int v = 0; v < n; ++v) {
    if (lptr[v + 1] - lptr[v] < 2) continue;
    for (int t = 0; t < n; ++t) lab[t] = -1;
    int nl = 0;
    for (int s0 = 0; s0 < n; ++s0) {
      if (s0 == v || lab[s0] >= 0) continue;
      int top = 0;
      stack[top++] = s0;
      lab[s0] = nl;
      while (top) {
        int u = stack[--top];
        for (int i = lptr[u]; i < lptr[u + 1]; ++i) {
          int w = ladj[i];
          if (w != v && lab[w] < 0) { lab[w] = nl; stack[top++] = w; }
        }
      }
      ++nl;
    }
    for (int i = lptr[v]; i < lptr[v + 1]; ++i)
      for (int j = i + 1; j < lptr[v + 1]; ++j)
        if (lab[ladj[i]] == lab[ladj[j]]) {
          int ra = find_uf(uf, eid[i]), rb = find_uf(uf, eid[j]);
          if (ra != rb) uf[ra > rb ? ra : rb] = ra < rb ? ra : rb;
        }
  }
  /* blocks: one per edge class, or the lone segment */
  bid = malloc(sizeof(int) * (size_t)(ne + 1));
  mark = malloc(sizeof(int) * (size_t)(n + 1));
  if (!bid || !mark) goto done;
  for (int e = 0; e < ne; ++e) bid[e] = -1;
  for (int e = 0; e < ne; ++e) {
    int r = find_uf(uf, e);
    if (bid[r] < 0) bid[r] = nb++;
    bid[e] = bid[r];
  }
  if (ne == 0) nb = 1;
  blocks = calloc((size_t)nb, sizeof(vlist_t));
  if (!blocks) goto done;
  if (ne == 0) {
    blocks[0].v = malloc(sizeof(int));
    if (!blocks[0].v) goto done;
    blocks[0].v[0] = 0;
    blocks[0].n = 1;
  } else {
    for (int b = 0; b < nb; ++b) {
      for (int t = 0; t < n; ++t) mark[t] = 0;
      int cnt = 0;
      for (int e = 0; e < ne; ++e)
        if (bid[e] == b) {
          if (!mark[ea[e]]) { mark[ea[e]] = 1; ++cnt; }
          if (!mark[eb[e]]) { mark[eb[e]] = 1; ++cnt; }
        }
      blocks[b].v = malloc(sizeof(int) * (size_t)cnt);
      if (!blocks[b].v) goto done;
      for (int t = 0; t < n; ++t) if (mark[t]) blocks[b].v[blocks[b].n++] = t;
    }
  }
  /* blocks of each segment, in lexicographic order of their lists */
  vb_ptr = calloc((size_t)n + 1, sizeof(int));
  if (!vb_ptr) goto done;
  for (int b = 0; b < nb; ++b) for (int i = 0; i < blocks[b].n; ++i) vb_ptr[blocks[b].v[i] + 1]++;
  for (int t = 0; t < n; ++t) vb_ptr[t + 1] += vb_ptr[t];
  vb = malloc(sizeof(int) * (size_t)(vb_ptr[n] + 1));
  bcount = calloc((size_t)n + 1, sizeof(int));
  if (!vb || !bcount) goto done;
  for (int b = 0; b < nb; ++b)
    for (int i = 0; i < blocks[b].n; ++i) {
      int t = blocks[b].v[i];
      vb[vb_ptr[t] + bcount[t]++] = b;
    }
  for (int t = 0; t < n; ++t)   /* insertion sort by segment list */
    for (int i = vb_ptr[t] + 1; i < vb_ptr[t + 1]; ++i) {
      int x = vb[i], j = i - 1;
      while (j >= vb_ptr[t] && lex_cmp(&blocks[vb[j]], &blocks[x]) > 0) { vb[j + 1] = vb[j]; --j; }
      vb[j + 1] = x;
    }
  /* breadth-first over the block-cut tree from the first block of segment 0 */
  order = malloc(sizeof(int) * (size_t)nb);
  attach = malloc(sizeof(int) * (size_t)nb);
  visited = calloc((size_t)nb, sizeof(int));
  if (!order || !attach || !visited) goto done;
  int qn = 0;
  order[qn] = vb[vb_ptr[0]];
  attach[qn] = -1;
  visited[order[qn]] = 1;
  ++qn;
  for (int h = 0; h < qn; ++h) {
    const vlist_t *B = &blocks[order[h]];
    for (int i = 0; i < B->n; ++i) {
      int t = B->v[i];
      for (int j = vb_ptr[t]; j < vb_ptr[t + 1]; ++j)
        if (!visited[vb[j]]) {
          visited[vb[j]] = 1;
          order[qn] = vb[j];
          attach[qn] = seg[t];
          ++qn;
        }
    }
  }
  if (qn != nb) { rc = OR_E_INVALID; goto done; }   /* a component is connected */
  for (int q = 0; q < nb; ++q) {
    const vlist_t *B = &blocks[order[q]];
    if (*n_out + 1 >= *cap_blocks) {
      int nc = *cap_blocks * 2 + 16;
      int *np = realloc(*out_ptr, sizeof(int) * (size_t)(nc + 1));
      if (!np) goto done;
      *out_ptr = np;
      int *na = realloc(*out_att, sizeof(int) * (size_t)(nc + 1));
      if (!na) goto done;
      *out_att = na;
      *cap_blocks = nc;
    }
    if (*len_seg + B->n > *cap_seg) {
      int nc = (*cap_seg + B->n) * 2 + 16;
      int *ns = realloc(*out_seg, sizeof(int) * (size_t)nc);
      if (!ns) goto done;
      *out_seg = ns;
      *cap_seg = nc;
    }
    for (int i = 0; i < B->n; ++i) (*out_seg)[*len_seg + i] = seg[B->v[i]];
    *len_seg += B->n;
    (*out_att)[*n_out] = attach[q];
    (*out_ptr)[*n_out + 1] = *len_seg;
    *n_out += 1;
  }
  rc = OR_OK;
done:
  if (blocks) for (int b = 0; b < nb; ++b) free(blocks[b].v);
  free(blocks); free(deg); free(lptr); free(ladj); free(eid); free(ea); free(eb); free(uf);
  free(lab); free(stack); free(bid); free(mark); free(bcount); free(order); free(visited);
  free(queue); free(attach); free(vb_ptr); free(vb);
  return rc;
}

/* Components (conflict and stitch edges, numbered by lowest segment) and
 * their blocks in canonical order, for the given graph as it stands (no
 * simplification).  inst_ptr has room for n + 1 entries, inst_seg and
 * inst_att for 2 * (n + ne + ns) + 1; returns the number of blocks. */
int oracle_blocks(int n, int ne, const int *eu, const int *ev, int ns, const int *su,
                  const int *sv, int *inst_ptr_out, int *inst_seg_out, int *inst_att_out) {
  if (n < 0 || ne < 0 || ns < 0) return OR_E_INVALID;
  int rc, *cu = NULL, *cv = NULL, *tu = NULL, *tv = NULL, mc = 0, ms = 0;
  int *cptr = NULL, *cadj = NULL, *sptr = NULL, *sadj = NULL, *parent = NULL, *cid = NULL;
  int *cseg = NULL, *cp = NULL, *ip = NULL, *is = NULL, *ia = NULL;
  int n_inst = 0, cap_b = 16, cap_s = 16, len = 0;
  if ((rc = norm_edges(n, ne, eu, ev, &cu, &cv, &mc)) != OR_OK) goto done;
  if ((rc = norm_edges(n, ns, su, sv, &tu, &tv, &ms)) != OR_OK) goto done;
  if ((rc = build_adj(n, mc, cu, cv, &cptr, &cadj)) != OR_OK) goto done;
  if ((rc = build_adj(n, ms, tu, tv, &sptr, &sadj)) != OR_OK) goto done;
  rc = OR_E_OOM;
  parent = malloc(sizeof(int) * (size_t)(n + 1));
  cid = malloc(sizeof(int) * (size_t)(n + 1));
  cseg = malloc(sizeof(int) * (size_t)(n + 1));
  cp = calloc((size_t)n + 2, sizeof(int));
  ip = malloc(sizeof(int) * (size_t)(cap_b + 1));
  ia = malloc(sizeof(int) * (size_t)(cap_b + 1));
  is = malloc(sizeof(int) * (size_t)cap_s);
  if (!parent || !cid || !cseg || !cp || !ip || !ia || !is) goto done;
  for (int s = 0; s < n; ++s) parent[s] = s;
  for (int e = 0; e < mc; ++e) {
    int ra = find_root(parent, cu[e]), rb = find_root(parent, cv[e]);
    if (ra != rb) parent[ra > rb ? ra : rb] = ra < rb ? ra : rb;
  }
  for (int e = 0; e < ms; ++e) {
    int ra = find_root(parent, tu[e]), rb = find_root(parent, tv[e]);
    if (ra != rb) parent[ra > rb ? ra : rb] = ra < rb ? ra : rb;
  }
  int nc = 0;
  for (int s = 0; s < n; ++s) cid[s] = -1;
  for (int s = 0; s < n; ++s) {
    int r = find_root(parent, s);
    if (cid[r] < 0) cid[r] = nc++;
    cid[s] = cid[r];
  }
  for (int s = 0; s < n; ++s) cp[cid[s] + 1]++;
  for (int c = 0; c < nc; ++c) cp[c + 1] += cp[c];
  {
    int *fill = calloc((size_t)nc + 1, sizeof(int));
    if (!fill) goto done;
    for (int s = 0; s < n; ++s) cseg[cp[cid[s]] + fill[cid[s]]++] = s;
    free(fill);
  }
  ip[0] = 0;
  for (int c = 0; c < nc; ++c)
    if ((rc = component_blocks(cseg + cp[c], cp[c + 1] - cp[c], cptr, cadj, sptr, sadj, &ip, &is,
                               &ia, &n_inst, &cap_b, &len, &cap_s)) != OR_OK)
      goto done;
  memcpy(inst_ptr_out, ip, sizeof(int) * (size_t)(n_inst + 1));
  memcpy(inst_seg_out, is, sizeof(int) * (size_t)len);
  memcpy(inst_att_out, ia, sizeof(int) * (size_t)n_inst);
  rc = n_inst;
done:
  free(cu); free(cv); free(tu); free(tv); free(cptr); free(cadj); free(sptr); free(sadj);
  free(parent); free(cid); free(cseg); free(cp); free(ip); free(is); free(ia);
  return rc;
}

int oracle_decompose(int n_seg, int k, int n_conf, const int *conf_u, const int *conf_v,
                     int n_st, const int *st_u, const int *st_v, const int *polygon_of,
                     int64_t cost_conflict, int64_t cost_stitch, uint32_t flags, int64_t budget,
                     int nthreads, signed char *mask_out, int32_t *comp_of_out,
                     int64_t *comp_nodes_out, int64_t *comp_cost_out, int32_t *comp_status_out,
                     oracle_totals *tot) {
  if (n_seg < 0 || k < 2 || k > 8 || n_conf < 0 || n_st < 0 || nthreads < 1) return OR_E_INVALID;
  if ((flags & OR_BICONNECTED) && (flags & OR_SINGLE_INSTANCE)) return OR_E_INVALID;
  if ((flags & OR_BICONNECTED) && (flags & OR_DENSITY_BALANCE)) return OR_E_INVALID;
  if (polygon_of)
    for (int s = 0; s < n_seg; ++s)
      if (polygon_of[s] < 0 || polygon_of[s] >= n_seg) return OR_E_INVALID;
  int rc;
  int *cu = NULL, *cv = NULL, *tu = NULL, *tv = NULL, mc = 0, ms = 0;
  int *cptr = NULL, *cadj = NULL, *sptr = NULL, *sadj = NULL;
  int *unit = NULL, *udeg = NULL, *queue = NULL, *removed_order = NULL, *uptr = NULL, *useg = NULL;
  char *removed = NULL, *queued = NULL, *selfc = NULL;
  int *parent = NULL, *comp_of = NULL, *comp_ptr = NULL, *comp_seg = NULL, *local_of = NULL, *order = NULL;
  int *inst_ptr = NULL, *inst_seg = NULL, *inst_att = NULL;
  signed char *imask = NULL;
  int64_t *ccost = NULL, *cnodes = NULL;
  int32_t *cstat = NULL;
  memset(tot, 0, sizeof(*tot));

  if ((rc = norm_edges(n_seg, n_conf, conf_u, conf_v, &cu, &cv, &mc)) != OR_OK) goto done;
  if ((rc = norm_edges(n_seg, n_st, st_u, st_v, &tu, &tv, &ms)) != OR_OK) goto done;
  if ((rc = build_adj(n_seg, mc, cu, cv, &cptr, &cadj)) != OR_OK) goto done;
  if ((rc = build_adj(n_seg, ms, tu, tv, &sptr, &sadj)) != OR_OK) goto done;
  rc = OR_E_OOM;

  /* units: polygons merged along stitch edges; unit id = lowest segment */
  parent = malloc(sizeof(int) * (size_t)(n_seg + 1));
  unit = malloc(sizeof(int) * (size_t)(n_seg + 1));
  if (!parent || !unit) goto done;
  for (int s = 0; s < n_seg; ++s) parent[s] = s;
  {
    int *first_of_poly = malloc(sizeof(int) * (size_t)(n_seg + 1));
    if (!first_of_poly) goto done;
    for (int p = 0; p < n_seg; ++p) first_of_poly[p] = -1;
    for (int s = 0; s < n_seg; ++s) {
      int p = polygon_of ? polygon_of[s] : s;
      if (first_of_poly[p] < 0) first_of_poly[p] = s;
      else {
        int ra = find_root(parent, first_of_poly[p]), rb = find_root(parent, s);
        if (ra != rb) parent[ra > rb ? ra : rb] = ra < rb ? ra : rb;
      }
    }
    free(first_of_poly);
  }
  for (int e = 0; e < ms; ++e) {
    int ra = find_root(parent, tu[e]), rb = find_root(parent, tv[e]);
    if (ra != rb) parent[ra > rb ? ra : rb] = ra < rb ? ra : rb;
  }
  for (int s = 0; s < n_seg; ++s) unit[s] = find_root(parent, s);

  /* unit member lists (segments ascending) */
  uptr = calloc((size_t)n_seg + 1, sizeof(int));
  useg = malloc(sizeof(int) * (size_t)(n_seg + 1));
  if (!uptr || !useg) goto done;
  for (int s = 0; s < n_seg; ++s) uptr[unit[s] + 1]++;
  for (int u = 0; u < n_seg; ++u) uptr[u + 1] += uptr[u];
  {
    int *fill = calloc((size_t)n_seg + 1, sizeof(int));
    if (!fill) goto done;
    for (int s = 0; s < n_seg; ++s) useg[uptr[unit[s]] + fill[unit[s]]++] = s;
    free(fill);
  }

  removed = calloc((size_t)n_seg + 1, 1);
  queued = calloc((size_t)n_seg + 1, 1);
  selfc = calloc((size_t)n_seg + 1, 1);
  udeg = calloc((size_t)n_seg + 1, sizeof(int));
  queue = malloc(sizeof(int) * (size_t)(n_seg + 1));
  removed_order = malloc(sizeof(int) * (size_t)(n_seg + 1));
  if (!removed || !queued || !selfc || !udeg || !queue || !removed_order) goto done;
  int n_removed_units = 0;
  if (!(flags & OR_NO_SIMPLIFY)) {
    for (int e = 0; e < mc; ++e) {
      int ua = unit[cu[e]], ub = unit[cv[e]];
      if (ua == ub) selfc[ua] = 1;
      else { udeg[ua]++; udeg[ub]++; }
    }
    int qh = 0, qt = 0;
    for (int u = 0; u < n_seg; ++u)
      if (unit[u] == u && !selfc[u] && udeg[u] < k) { queue[qt++] = u; queued[u] = 1; }
    while (qh < qt) {
      int u = queue[qh++];
      removed[u] = 1;
      removed_order[n_removed_units++] = u;
      for (int t = uptr[u]; t < uptr[u + 1]; ++t) {
        int s = useg[t];
        for (int i = cptr[s]; i < cptr[s + 1]; ++i) {
          int w = unit[cadj[i]];
          if (w == u || removed[w]) continue;
          udeg[w]--;
          if (!queued[w] && !selfc[w] && udeg[w] < k) { queue[qt++] = w; queued[w] = 1; }
        }
      }
    }
  }

  /* components of the remaining segments */
  comp_of = malloc(sizeof(int) * (size_t)(n_seg + 1));
  local_of = malloc(sizeof(int) * (size_t)(n_seg + 1));
  if (!comp_of || !local_of) goto done;
  for (int s = 0; s < n_seg; ++s) parent[s] = s;
  if (!(flags & OR_SINGLE_INSTANCE)) {
    for (int e = 0; e < mc; ++e)
      if (!removed[unit[cu[e]]] && !removed[unit[cv[e]]]) {
        int ra = find_root(parent, cu[e]), rb = find_root(parent, cv[e]);
        if (ra != rb) parent[ra > rb ? ra : rb] = ra < rb ? ra : rb;
      }
    for (int e = 0; e < ms; ++e)
      if (!removed[unit[tu[e]]]) {
        int ra = find_root(parent, tu[e]), rb = find_root(parent, tv[e]);
        if (ra != rb) parent[ra > rb ? ra : rb] = ra < rb ? ra : rb;
      }
  }
  int n_comp = 0;
  {
    int *id_of_root = malloc(sizeof(int) * (size_t)(n_seg + 1));
    if (!id_of_root) goto done;
    for (int s = 0; s < n_seg; ++s) id_of_root[s] = -1;
    int single_id = -1;
    for (int s = 0; s < n_seg; ++s) {
      if (removed[unit[s]]) { comp_of[s] = -1; continue; }
      if (flags & OR_SINGLE_INSTANCE) {
        if (single_id < 0) single_id = n_comp++;
        comp_of[s] = single_id;
      } else {
        int r = find_root(parent, s);   /* roots are the lowest segment */
        if (id_of_root[r] < 0) id_of_root[r] = n_comp++;
        comp_of[s] = id_of_root[r];
      }
    }
    free(id_of_root);
  }
  comp_ptr = calloc((size_t)n_comp + 2, sizeof(int));
  comp_seg = malloc(sizeof(int) * (size_t)(n_seg + 1));
  if (!comp_ptr || !comp_seg) goto done;
  for (int s = 0; s < n_seg; ++s) if (comp_of[s] >= 0) comp_ptr[comp_of[s] + 1]++;
  for (int c = 0; c < n_comp; ++c) comp_ptr[c + 1] += comp_ptr[c];
  {
    int *fill = calloc((size_t)n_comp + 1, sizeof(int));
    if (!fill) goto done;
    for (int s = 0; s < n_seg; ++s)
      if (comp_of[s] >= 0) {
        int c = comp_of[s];
        local_of[s] = fill[c];
        comp_seg[comp_ptr[c] + fill[c]++] = s;
      } else local_of[s] = -1;
    free(fill);
  }

  /* search instances: the components, or their biconnected blocks */
  int n_inst = 0, len_seg = 0;
  if (flags & OR_BICONNECTED) {
    int cap_b = 16, cap_s = 16;
    inst_ptr = malloc(sizeof(int) * (size_t)(cap_b + 1));
    inst_att = malloc(sizeof(int) * (size_t)(cap_b + 1));
    inst_seg = malloc(sizeof(int) * (size_t)cap_s);
    if (!inst_ptr || !inst_att || !inst_seg) goto done;
    inst_ptr[0] = 0;
    for (int c = 0; c < n_comp; ++c) {
      rc = component_blocks(comp_seg + comp_ptr[c], comp_ptr[c + 1] - comp_ptr[c], cptr, cadj,
                            sptr, sadj, &inst_ptr, &inst_seg, &inst_att, &n_inst, &cap_b,
                            &len_seg, &cap_s);
      if (rc != OR_OK) goto done;
    }
    rc = OR_E_OOM;
  } else {
    n_inst = n_comp;
    len_seg = comp_ptr[n_comp];
    inst_ptr = malloc(sizeof(int) * (size_t)(n_comp + 1));
    inst_att = malloc(sizeof(int) * (size_t)(n_comp + 1));
    inst_seg = malloc(sizeof(int) * (size_t)(len_seg + 1));
    if (!inst_ptr || !inst_att || !inst_seg) goto done;
    memcpy(inst_ptr, comp_ptr, sizeof(int) * (size_t)(n_comp + 1));
    memcpy(inst_seg, comp_seg, sizeof(int) * (size_t)len_seg);
    for (int c = 0; c < n_comp; ++c) inst_att[c] = -1;
  }
  order = malloc(sizeof(int) * (size_t)(n_inst + 1));
  ccost = calloc((size_t)n_inst + 1, sizeof(int64_t));
  cnodes = calloc((size_t)n_inst + 1, sizeof(int64_t));
  cstat = calloc((size_t)n_inst + 1, sizeof(int32_t));
  imask = malloc((size_t)len_seg + 1);
  if (!order || !ccost || !cnodes || !cstat || !imask) goto done;
  {
    int *keys = malloc(sizeof(int) * (size_t)(2 * n_inst + 2));
    if (!keys) goto done;
    for (int c = 0; c < n_inst; ++c) { keys[2 * c] = inst_ptr[c + 1] - inst_ptr[c]; keys[2 * c + 1] = c; }
    qsort(keys, (size_t)n_inst, 2 * sizeof(int), cmp_comp);
    for (int c = 0; c < n_inst; ++c) order[c] = keys[2 * c + 1];
    free(keys);
  }

  for (int s = 0; s < n_seg; ++s) mask_out[s] = -1;
  {
    pool_t P;
    memset(&P, 0, sizeof(P));
    P.k = k; P.n_comp = n_inst; P.Cc = cost_conflict; P.Cs = cost_stitch; P.budget = budget;
    P.rule = ((flags & OR_COLUMN_BFS) ? 1 : 0) | ((flags & OR_CLIQUE_BOUND) ? 2 : 0) |
             ((flags & OR_SPLIT_BUDGET) ? 4 : 0);
    P.comp_ptr = inst_ptr; P.comp_seg = inst_seg;
    P.cptr = cptr; P.cadj = cadj; P.sptr = sptr; P.sadj = sadj; P.work_order = order;
    P.imask = imask; P.comp_cost = ccost; P.comp_nodes = cnodes; P.comp_status = cstat;
    atomic_init(&P.next, 0);
    atomic_init(&P.error, 0);
    int nt = nthreads < n_inst ? nthreads : (n_inst > 0 ? n_inst : 1);
    pthread_t *th = malloc(sizeof(pthread_t) * (size_t)nt);
    if (!th) goto done;
    pthread_attr_t attr;
    pthread_attr_init(&attr);
    pthread_attr_setstacksize(&attr, (size_t)256 << 20);   /* deep recursion */
    int started = 0;
    const double t_search = wall_seconds();
    for (int t = 0; t < nt; ++t)
      if (pthread_create(&th[t], &attr, pool_worker, &P) == 0) started++;
      else break;
    pthread_attr_destroy(&attr);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    tot->search_seconds = wall_seconds() - t_search;
    tot->instance_segments = len_seg;
    free(th);
    if (started == 0) goto done;
    if (atomic_load(&P.error)) { rc = atomic_load(&P.error); goto done; }
  }
  /* instance masks into the layout, in instance order: a block attached at
   * segment a takes the transposition of masks that keeps a's mask */
  for (int c = 0; c < n_inst; ++c) {
    const int a = inst_ptr[c], b = inst_ptr[c + 1];
    int from = -1, to = -1;
    if (inst_att[c] >= 0) {
      int l = local_id(inst_seg + a, b - a, inst_att[c]);
      if (l < 0 || mask_out[inst_att[c]] < 0) { rc = OR_E_INVALID; goto done; }
      from = imask[a + l];
      to = mask_out[inst_att[c]];
    }
    for (int t = a; t < b; ++t) {
      int m = imask[t];
      if (from >= 0) m = m == from ? to : m == to ? from : m;
      mask_out[inst_seg[t]] = (signed char)m;
    }
  }
  /* density balance (a reading; the paper names the rule only in passing):
   * permuting the masks of one component keeps its cost, so each instance in
   * instance order gets the permutation that pairs its masks, by decreasing
   * segment count (lower mask first on ties), with the masks of the layout so
   * far by increasing segment count (lower mask first); recovery below then
   * gives a removed unit the least used of the masks its coloured conflict
   * neighbours leave free (lowest on ties) */
  int64_t tot_mask[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (flags & OR_DENSITY_BALANCE) {
    for (int c = 0; c < n_inst; ++c) {
      int64_t x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int t = inst_ptr[c]; t < inst_ptr[c + 1]; ++t) x[mask_out[inst_seg[t]]]++;
      int src[8], dst[8], perm[8];
      for (int m = 0; m < k; ++m) { src[m] = m; dst[m] = m; }
      /* insertion sorts: src by (x desc, m asc), dst by (tot asc, m asc) */
      for (int i = 1; i < k; ++i)
        for (int j = i; j > 0 && x[src[j]] > x[src[j - 1]]; --j) {
          int t = src[j]; src[j] = src[j - 1]; src[j - 1] = t;
        }
      for (int i = 1; i < k; ++i)
        for (int j = i; j > 0 && tot_mask[dst[j]] < tot_mask[dst[j - 1]]; --j) {
          int t = dst[j]; dst[j] = dst[j - 1]; dst[j - 1] = t;
        }
      for (int i = 0; i < k; ++i) perm[src[i]] = dst[i];
      for (int t = inst_ptr[c]; t < inst_ptr[c + 1]; ++t)
        mask_out[inst_seg[t]] = (signed char)perm[mask_out[inst_seg[t]]];
      for (int m = 0; m < k; ++m) tot_mask[perm[m]] += x[m];
    }
  }
  /* instance of each segment: the first one holding it */
  for (int s = 0; s < n_seg; ++s) comp_of[s] = -1;
  for (int c = n_inst - 1; c >= 0; --c)
    for (int t = inst_ptr[c]; t < inst_ptr[c + 1]; ++t) comp_of[inst_seg[t]] = c;

  /* recovery: reverse removal order, lowest mask unused by coloured nbrs */
  for (int t = n_removed_units - 1; t >= 0; --t) {
    int u = removed_order[t];
    unsigned used = 0;
    for (int q = uptr[u]; q < uptr[u + 1]; ++q) {
      int s = useg[q];
      for (int i = cptr[s]; i < cptr[s + 1]; ++i) {
        int m = mask_out[cadj[i]];
        if (m >= 0) used |= 1u << m;
      }
    }
    int c = 0;
    if (flags & OR_DENSITY_BALANCE) {
      c = -1;
      for (int m = 0; m < k; ++m)
        if (!((used >> m) & 1u) && (c < 0 || tot_mask[m] < tot_mask[c])) c = m;
      if (c < 0) c = k;
    } else {
      while (c < k && (used >> c) & 1u) ++c;
    }
    if (c == k) { rc = OR_E_INVALID; goto done; }   /* cannot happen for a k-core peel */
    for (int q = uptr[u]; q < uptr[u + 1]; ++q) mask_out[useg[q]] = (signed char)c;
    tot_mask[c] += uptr[u + 1] - uptr[u];
    tot->n_removed_segments += uptr[u + 1] - uptr[u];
  }

  /* totals over the whole layout (Eq. 1) */
  for (int e = 0; e < mc; ++e) if (mask_out[cu[e]] == mask_out[cv[e]]) tot->n_conflicts++;
  for (int e = 0; e < ms; ++e) if (mask_out[tu[e]] != mask_out[tv[e]]) tot->n_stitches++;
  tot->cost = cost_conflict * tot->n_conflicts + cost_stitch * tot->n_stitches;
  tot->n_components = n_inst;
  tot->status = OR_OK;
  for (int c = 0; c < n_inst; ++c) {
    tot->nodes += cnodes[c];
    tot->component_cost_sum += ccost[c];
    if (cstat[c] == OR_BUDGET) { tot->n_budget_components++; tot->status = OR_BUDGET; }
    int sz = inst_ptr[c + 1] - inst_ptr[c];
    if (sz > tot->max_component) tot->max_component = sz;
    if (comp_nodes_out) comp_nodes_out[c] = cnodes[c];
    if (comp_cost_out) comp_cost_out[c] = ccost[c];
    if (comp_status_out) comp_status_out[c] = cstat[c];
  }
  if (comp_of_out) for (int s = 0; s < n_seg; ++s) comp_of_out[s] = comp_of[s];
  rc = tot->status;

done:
  free(cu); free(cv); free(tu); free(tv); free(cptr); free(cadj); free(sptr); free(sadj);
  free(unit); free(udeg); free(queue); free(removed_order); free(uptr); free(useg);
  free(removed); free(queued); free(selfc); free(parent); free(comp_of); free(comp_ptr);
  free(comp_seg); free(local_of); free(order); free(ccost); free(cnodes); free(cstat);
  free(inst_ptr); free(inst_seg); free(inst_att); free(imask);
  return rc;
}
