// mpld_host.cpp -- host half of libmpld: input checks, simplification and
// sub-graph split (Sec. 2.2; Algorithm 1 steps that split the DG), EC matrix
// packing (Sec. 2.3), launches of the search kernels, copy back, recovery of
// removed nodes (Sec. 2.2) and the conflict / stitch counts (Eq. 1).
//
// Simplification rule (the paper names the step but not its rule): a unit is
// a polygon together with every segment joined to it by a stitch edge.  A
// unit with fewer than k conflict edges to remaining units is removed; the
// queue is FIFO, seeded in ascending unit id (its lowest segment), and a
// removal decrements its neighbours, which join the queue when they drop
// below k.  A unit with a conflict edge inside itself is never removed.
// Recovery walks the removal order backwards and gives every segment of a
// unit the lowest mask unused by its coloured conflict neighbours, which
// costs nothing, so the layout optimum equals the sum of instance optima.
#include <cuda_runtime.h>

#include <algorithm>
#include <limits>
#include <memory>
#include <deque>
#include <condition_variable>
#include <thread>
#include <atomic>
#include <functional>
#include <chrono>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "../../include/mpld.h"
#include "mpld_internal.h"
#include "mpld_problem.h"

using mpld::InstDesc;
using mpld::InstResult;

namespace {

constexpr int MAX_COST = 10000;
constexpr int64_t DEFAULT_TIME_LIMIT_MS = 60000;
constexpr int DEFAULT_CTA_SEGMENTS = 4096;   // instances this large get a whole CTA
constexpr int CTA_TEAM_WARPS = 8;            // least CTA size when some instance does

using mpld::GraphKey;

struct Shape {
  int nw, slot, ctas;
};

}  // namespace

namespace {

// ---------------------------------------------------------------- helpers

int find_root(std::vector<int32_t> &parent, int a) {
  while (parent[a] != a) {
    parent[a] = parent[parent[a]];
    a = parent[a];
  }
  return a;
}

void unite_min(std::vector<int32_t> &parent, int a, int b) {
  int ra = find_root(parent, a), rb = find_root(parent, b);
  if (ra == rb) return;
  if (ra < rb) parent[rb] = ra;
  else parent[ra] = rb;
}

// The same forest shared by threads: a link hangs the larger root under the
// smaller with a compare-and-swap, so parent[x] <= x always and every root is
// its set's lowest element whatever the order of the unions; finds halve
// paths (a parent only ever moves to an ancestor).
int pfind(int32_t *par, int x) {
  for (;;) {
    const int px = __atomic_load_n(par + x, __ATOMIC_RELAXED);
    if (px == x) return x;
    const int gx = __atomic_load_n(par + px, __ATOMIC_RELAXED);
    if (gx != px) __atomic_store_n(par + x, gx, __ATOMIC_RELAXED);
    x = gx;
  }
}
// The root of x once every union is done, without writing on the way: run
// by every thread at once to store each entry's root, it never stores
// anything but a root, so no entry can lose its root to another thread's
// path halving (which would store a grandparent over it).
int proot(const int32_t *par, int x) {
  for (;;) {
    const int px = __atomic_load_n(par + x, __ATOMIC_RELAXED);
    if (px == x) return x;
    x = px;
  }
}
void punite(int32_t *par, int a, int b) {
  for (;;) {
    a = pfind(par, a);
    b = pfind(par, b);
    if (a == b) return;
    if (a > b) std::swap(a, b);
    int expect = b;
    if (__atomic_compare_exchange_n(par + b, &expect, a, false, __ATOMIC_RELAXED, __ATOMIC_RELAXED))
      return;
  }
}

// Biconnected blocks of one component (MPLD_BICONNECTED), appended in the
// canonical order: breadth-first over the block-cut tree, starting from the
// lexicographically first block (ascending segment list) that holds the
// component's lowest segment; from a block, its segments in ascending id,
// and at each the blocks not yet taken in lexicographic order, attached at
// that segment.  Blocks come from one iterative depth-first search with
// discovery times and low points over conflict and stitch edges together;
// a component without edges is one block of one segment.
//   seg:  the component's segments, ascending; loc: scratch, -1 on entry
//   and on return (global segment -> index in seg)
//   iptr / iseg / iatt: block boundaries, segments, attach index within the
//   block (-1 for the first block)
void component_blocks(const std::vector<int32_t> &seg, const std::vector<int32_t> &cptr,
                      const std::vector<int32_t> &cadj, const std::vector<int32_t> &sptr,
                      const std::vector<int32_t> &sadj, std::vector<int32_t> &loc,
                      std::vector<int32_t> &iptr, std::vector<int32_t> &iseg,
                      std::vector<int32_t> &iatt) {
  const int n = (int)seg.size();
  for (int i = 0; i < n; ++i) loc[seg[i]] = i;
  // union adjacency, local ids ascending
  std::vector<int32_t> lptr((size_t)n + 1, 0), ladj;
  for (int i = 0; i < n; ++i) {
    const int g = seg[i];
    int a = cptr[g], b = sptr[g];
    while (a < cptr[g + 1] || b < sptr[g + 1]) {
      int w;
      if (b >= sptr[g + 1] || (a < cptr[g + 1] && cadj[a] <= sadj[b])) {
        w = cadj[a++];
        if (b < sptr[g + 1] && sadj[b] == w) ++b;
      } else {
        w = sadj[b++];
      }
      if (loc[w] >= 0) ladj.push_back(loc[w]);
    }
    lptr[i + 1] = (int32_t)ladj.size();
  }
  std::vector<std::vector<int32_t>> blocks;
  if (ladj.empty()) {
    blocks.push_back({0});
  } else {
    std::vector<int32_t> disc((size_t)n, -1), low((size_t)n, 0), mark((size_t)n, -1);
    struct Frame { int v, parent, it; };
    std::vector<Frame> st;
    std::vector<std::pair<int32_t, int32_t>> es;
    int timer = 0;
    disc[0] = low[0] = timer++;
    st.push_back({0, -1, lptr[0]});
    while (!st.empty()) {
      Frame &f = st.back();
      const int v = f.v;
      if (f.it < lptr[v + 1]) {
        const int w = ladj[f.it++];
        if (disc[w] < 0) {
          es.emplace_back(v, w);
          disc[w] = low[w] = timer++;
          st.push_back({w, v, lptr[w]});
        } else if (w != f.parent && disc[w] < disc[v]) {
          es.emplace_back(v, w);
          low[v] = std::min(low[v], disc[w]);
        }
        continue;
      }
      st.pop_back();
      if (st.empty()) break;
      const int u = st.back().v;
      low[u] = std::min(low[u], low[v]);
      if (low[v] >= disc[u]) {
        // u separates v's subtree: its edges since (u, v) form a block
        std::vector<int32_t> b;
        const int id = (int)blocks.size();
        for (;;) {
          const auto e = es.back();
          es.pop_back();
          for (int x : {e.first, e.second})
            if (mark[x] != id) { mark[x] = id; b.push_back(x); }
          if (e.first == u && e.second == v) break;
        }
        std::sort(b.begin(), b.end());
        blocks.push_back(std::move(b));
      }
    }
  }
  // blocks at each segment, lexicographic; breadth-first from segment 0's first
  std::vector<std::vector<int32_t>> at((size_t)n);
  for (int b = 0; b < (int)blocks.size(); ++b)
    for (int x : blocks[b]) at[x].push_back(b);
  for (auto &l : at)
    std::sort(l.begin(), l.end(), [&](int x, int y) { return blocks[x] < blocks[y]; });
  std::vector<uint8_t> taken(blocks.size(), 0);
  std::vector<std::pair<int32_t, int32_t>> queue;   // block, attach segment (local) or -1
  queue.emplace_back(at[0][0], -1);
  taken[at[0][0]] = 1;
  for (size_t h = 0; h < queue.size(); ++h)
    for (int x : blocks[queue[h].first])
      for (int b : at[x])
        if (!taken[b]) {
          taken[b] = 1;
          queue.emplace_back(b, x);
        }
  for (const auto &q : queue) {
    const auto &b = blocks[q.first];
    int att = -1;
    for (size_t i = 0; i < b.size(); ++i) {
      if (b[i] == q.second) att = (int)i;
      iseg.push_back(seg[b[i]]);
    }
    iatt.push_back(att);
    iptr.push_back((int32_t)iseg.size());
  }
  for (int i = 0; i < n; ++i) loc[seg[i]] = -1;
}

// Cliques of the second bound mode (MPLD_CLIQUE_BOUND) of one instance:
// every (k+1)-clique of its conflict graph, in lexicographic order of the
// ascending member lists, is taken when it shares no edge with a clique
// taken before.  lp / la: the instance's conflict adjacency, local ids,
// ascending.  Returns the members of the taken cliques, k + 1 each.
std::vector<uint16_t> greedy_cliques(int n, int K, const std::vector<int32_t> &lp,
                                     const std::vector<int32_t> &la) {
  std::vector<uint8_t> used(la.size(), 0);
  auto slot = [&](int a, int b) -> int {
    const auto first = la.begin() + lp[a], last = la.begin() + lp[a + 1];
    const auto it = std::lower_bound(first, last, b);
    return (it != last && *it == b) ? (int)(it - la.begin()) : -1;
  };
  std::vector<uint16_t> out;
  int cur[9];
  std::function<void(int)> extend = [&](int depth) {
    if (depth == K) {
      for (int i = 0; i < K; ++i)
        for (int j = i + 1; j < K; ++j)
          if (used[slot(cur[i], cur[j])]) return;
      for (int i = 0; i < K; ++i)
        for (int j = i + 1; j < K; ++j) {
          used[slot(cur[i], cur[j])] = 1;
          used[slot(cur[j], cur[i])] = 1;
        }
      for (int i = 0; i < K; ++i) out.push_back((uint16_t)cur[i]);
      return;
    }
    const int last = cur[depth - 1];
    for (int i = lp[last]; i < lp[last + 1]; ++i) {
      const int w = la[i];
      if (w <= last) continue;
      bool ok = true;
      for (int j = 0; j < depth - 1 && ok; ++j) ok = slot(cur[j], w) >= 0;
      if (!ok) continue;
      cur[depth] = w;
      extend(depth + 1);
    }
  };
  for (int v = 0; v < n; ++v) {
    cur[0] = v;
    extend(1);
  }
  return out;
}

// Host worker pool for the build and the result counting: up to 15 threads
// started on first use and kept for the life of the process.  A parallel
// loop puts helper tasks on the queue and works through its chunks on the
// calling thread as well; it returns when every chunk is done, not when
// every helper ran (a helper that starts late finds no chunk left and only
// touches the loop's shared, reference-counted state).
class HostPool {
 public:
  static HostPool &get() {
    static HostPool pool;
    return pool;
  }
  int helpers() const { return (int)th_.size(); }
  void post(std::function<void()> task) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      q_.push_back(std::move(task));
      pending_.fetch_add(1, std::memory_order_relaxed);
    }
    cv_.notify_one();
  }
  // tasks posted and not yet started (another parallel loop is filling the
  // pool), and whether the calling thread is one of the helpers
  int pending() const { return pending_.load(std::memory_order_relaxed); }
  static bool on_helper() { return helper_flag(); }

 private:
  HostPool() {
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int n = std::min(hw, 16) - 1;
    for (int i = 0; i < n; ++i) th_.emplace_back([this] { loop(); });
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto &t : th_) t.join();
  }
  static bool &helper_flag() {
    static thread_local bool flag = false;
    return flag;
  }
  void loop() {
    helper_flag() = true;
    for (;;) {
      std::function<void()> task;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || !q_.empty(); });
        if (stop_ && q_.empty()) return;
        task = std::move(q_.front());
        q_.pop_front();
        pending_.fetch_sub(1, std::memory_order_relaxed);
      }
      task();
    }
  }
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<std::function<void()>> q_;
  std::vector<std::thread> th_;
  std::atomic<int> pending_{0};
  bool stop_ = false;
};

// f(i) for i in [0, count), in chunks of `grain`, on the calling thread and
// the host pool.  An exception in f (out of memory) is rethrown as
// std::bad_alloc once every chunk has finished.
template <typename F>
void parallel_for(int count, int grain, F f) {
  const int chunks = (count + grain - 1) / grain;
  HostPool &pool = HostPool::get();
  // inline when nested in a pool task or when other loops already fill the
  // pool (concurrent layout builds): their threads are busy anyway
  const bool busy = HostPool::on_helper() || pool.pending() > 0;
  const int nh = busy ? 0 : std::min(pool.helpers(), chunks - 1);
  if (nh <= 0) {
    for (int i = 0; i < count; ++i) f(i);
    return;
  }
  struct State {
    std::atomic<int> next{0}, done{0};
    std::atomic<bool> failed{false};
    std::mutex mu;
    std::condition_variable cv;
  };
  auto st = std::make_shared<State>();
  F *fp = &f;
  auto work = [st, fp, count, grain, chunks] {
    for (;;) {
      const int q = st->next.fetch_add(1);
      if (q >= chunks) return;
      try {
        if (!st->failed.load())
          for (int i = q * grain, e = std::min(count, (q + 1) * grain); i < e; ++i) (*fp)(i);
      } catch (...) {
        st->failed = true;
      }
      if (st->done.fetch_add(1) + 1 == chunks) {
        std::lock_guard<std::mutex> lk(st->mu);
        st->cv.notify_all();
      }
    }
  };
  for (int t = 0; t < nh; ++t) pool.post(work);
  work();
  {
    std::unique_lock<std::mutex> lk(st->mu);
    st->cv.wait(lk, [&] { return st->done.load() == chunks; });
  }
  if (st->failed) throw std::bad_alloc();
}

// f(j) for j in [0, count) over `lanes` tasks, task q taking j = q, q + lanes,
// ...: the first `lanes` jobs (the largest instances, in a largest-first
// order) start at once on different threads, and the many small ones share
// few claims of the work counter.
template <typename F>
void parallel_strided(int count, int lanes, F f) {
  lanes = std::max(1, std::min(lanes, count));
  parallel_for(lanes, 1, [&](int q) {
    for (int j = q; j < count; j += lanes) f(j);
  });
}

// ---- steps of the host build, each on the host pool with the same result
// as one thread would give

// (min,max)-normalised, sorted, unique edges; returns false on a bad edge.
// Input already in that form (u < v, strictly ascending pairs) is checked
// and copied in chunks.  Otherwise the larger endpoints are bucketed by the
// smaller one (a counting sort), then each (short) bucket is sorted and
// deduplicated.
bool normalise(int n, int m, const int32_t *u, const int32_t *v, std::vector<int32_t> &ou,
               std::vector<int32_t> &ov) {
  constexpr int G = 1 << 15;
  const int chunks = (m + G - 1) / G;
  std::atomic<bool> sorted{true};
  parallel_for(chunks, 1, [&](int q) {
    for (int e = q * G, end = std::min(m, (q + 1) * G); e < end; ++e) {
      const int a = u[e], b = v[e];
      if (!(a >= 0 && a < b && b < n &&
            (e == 0 || a > u[e - 1] || (a == u[e - 1] && b > v[e - 1])))) {
        sorted.store(false, std::memory_order_relaxed);
        return;
      }
    }
  });
  if (sorted.load()) {
    ou.resize((size_t)m);
    ov.resize((size_t)m);
    parallel_for(chunks, 1, [&](int q) {
      const size_t e0 = (size_t)q * G, e1 = std::min((size_t)m, e0 + G);
      std::memcpy(ou.data() + e0, u + e0, (e1 - e0) * sizeof(int32_t));
      std::memcpy(ov.data() + e0, v + e0, (e1 - e0) * sizeof(int32_t));
    });
    return true;
  }
  std::vector<int32_t> start((size_t)n + 1, 0);
  for (int e = 0; e < m; ++e) {
    const int a = u[e], b = v[e];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) return false;
    start[std::min(a, b) + 1]++;
  }
  for (int i = 0; i < n; ++i) start[i + 1] += start[i];
  std::vector<int32_t> hi((size_t)m), fill(start.begin(), start.end() - 1);
  for (int e = 0; e < m; ++e) hi[fill[std::min(u[e], v[e])]++] = std::max(u[e], v[e]);
  ou.clear();
  ov.clear();
  ou.reserve((size_t)m);
  ov.reserve((size_t)m);
  for (int a = 0; a < n; ++a) {
    const auto first = hi.begin() + start[a], last = hi.begin() + start[a + 1];
    if (first == last) continue;
    std::sort(first, last);
    for (auto it = first; it != last; ++it)
      if (it == first || *it != *(it - 1)) {
        ou.push_back(a);
        ov.push_back(*it);
      }
  }
  return true;
}

// Adjacency with neighbours ascending (edges come sorted by (min,max)).
void csr(int n, const std::vector<int32_t> &u, const std::vector<int32_t> &v,
         std::vector<int32_t> &ptr, std::vector<int32_t> &adj) {
  ptr.assign((size_t)n + 1, 0);
  for (size_t e = 0; e < u.size(); ++e) { ptr[u[e] + 1]++; ptr[v[e] + 1]++; }
  for (int i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
  adj.resize(2 * u.size());
  std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
  // smaller neighbours of x arrive (as u of edges (u,x)) in ascending u, then
  // larger ones (as v of edges (x,v)) in ascending v -- but interleaved in
  // edge order; two passes keep each list sorted.
  for (size_t e = 0; e < u.size(); ++e) adj[fill[v[e]]++] = u[e];
  for (size_t e = 0; e < u.size(); ++e) adj[fill[u[e]]++] = v[e];
}

int cuda_ok(cudaError_t e) { return e == cudaSuccess ? MPLD_OK : MPLD_E_CUDA; }

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, mpld_tune> g_tune_cache;

// Process-wide cache key of a problem set: k and a coarse size histogram.
// Tuned launch shapes are kept per (k, size histogram, search mode): the
// budgeted split search's first launch is much shorter than a whole search.
std::tuple<int, int, int, int, int> tune_key(mpld_problem *const *ps, int n,
                                             const mpld_params *prm) {
  int kmax = 0;
  int64_t inst = 0;
  uint32_t fmax = 0;
  int64_t fsum = 0;
  for (int i = 0; i < n; ++i) {
    kmax = std::max(kmax, ps[i]->k);
    inst += ps[i]->n_comp;
    for (uint32_t f : ps[i]->footprint) { fmax = std::max(fmax, f); fsum += f; }
  }
  auto lg = [](int64_t x) { int b = 0; while (x > 1) { x >>= 1; ++b; } return b; };
  const int mode = (prm && (prm->flags & MPLD_SPLIT_BUDGET)) ? 1 : 0;
  return {kmax, lg(inst), lg(fmax), lg(inst ? fsum / inst : 0), mode};
}

}  // namespace

// ================================================================= build

extern "C" int mpld_build_matrix(const mpld_graph *g, const mpld_params *params, void *stream,
                                 mpld_problem **out) {
  if (!g || !out) return MPLD_E_INVALID;
  *out = nullptr;
  const int n = g->n_seg, k = g->k;
  if (n < 0 || k < 2 || k > 8 || g->n_conf < 0 || g->n_stitch < 0) return MPLD_E_INVALID;
  if ((g->n_conf > 0 && (!g->conf_u || !g->conf_v)) ||
      (g->n_stitch > 0 && (!g->st_u || !g->st_v)))
    return MPLD_E_INVALID;
  if (g->cost_conflict < 0 || g->cost_conflict > MAX_COST || g->cost_stitch < 0 ||
      g->cost_stitch > MAX_COST)
    return MPLD_E_INVALID;
  if (g->polygon_of)
    for (int s = 0; s < n; ++s)
      if (g->polygon_of[s] < 0 || g->polygon_of[s] >= n) return MPLD_E_INVALID;

  if (params && (params->flags & MPLD_BICONNECTED) && (params->flags & MPLD_SINGLE_INSTANCE))
    return MPLD_E_INVALID;
  // a block's masks are tied to its attach segment: no renaming for balance
  if (params && (params->flags & MPLD_BICONNECTED) && (params->flags & MPLD_DENSITY_BALANCE))
    return MPLD_E_INVALID;
  mpld_problem *p = new (std::nothrow) mpld_problem();
  if (!p) return MPLD_E_OOM;
  p->n_seg = n;
  p->k = k;
  p->Cc = g->cost_conflict;
  p->Cs = g->cost_stitch;
  p->flags = params ? params->flags : 0u;
  try {
    // the conflict edges normalised (checked and copied in chunks when they
    // come sorted); then their CSR form on one thread while another
    // normalises the stitch edges, puts them in CSR form and builds the
    // units (polygons merged along stitch edges, id = lowest segment), which
    // need nothing else
    std::vector<int32_t> sptr, sadj;
    std::vector<int32_t> parent((size_t)n);
    bool ok[2] = {true, true};
    ok[0] = normalise(n, g->n_conf, g->conf_u, g->conf_v, p->cu, p->cv);
    if (ok[0]) parallel_for(2, 1, [&](int which) {
      if (which == 0) {
        csr(n, p->cu, p->cv, p->cptr, p->cadj);
        return;
      }
      ok[1] = normalise(n, g->n_stitch, g->st_u, g->st_v, p->su, p->sv);
      if (!ok[1]) return;
      csr(n, p->su, p->sv, sptr, sadj);
      std::iota(parent.begin(), parent.end(), 0);
      {
        std::vector<int32_t> first_of((size_t)n, -1);
        for (int s = 0; s < n; ++s) {
          const int poly = g->polygon_of ? g->polygon_of[s] : s;
          if (first_of[poly] < 0) first_of[poly] = s;
          else unite_min(parent, first_of[poly], s);
        }
      }
      for (size_t e = 0; e < p->su.size(); ++e) unite_min(parent, p->su[e], p->sv[e]);
      p->unit_of.resize((size_t)n);
      for (int s = 0; s < n; ++s) p->unit_of[s] = find_root(parent, s);
      p->uptr.assign((size_t)n + 1, 0);
      for (int s = 0; s < n; ++s) p->uptr[p->unit_of[s] + 1]++;
      for (int u = 0; u < n; ++u) p->uptr[u + 1] += p->uptr[u];
      p->useg.resize((size_t)n);
      std::vector<int32_t> fill(p->uptr.begin(), p->uptr.end() - 1);
      for (int s = 0; s < n; ++s) p->useg[fill[p->unit_of[s]]++] = s;
    });
    if (!ok[0] || !ok[1]) {
      delete p;
      return MPLD_E_INVALID;
    }

    // ---- simplification: FIFO peel of units with < k external conflict edges
    std::vector<uint8_t> removed((size_t)n, 0);
    if (!(p->flags & MPLD_NO_SIMPLIFY)) {
      // per unit: external conflict degree, and a bit saying it may still
      // join the queue (not queued yet, no conflict edge inside)
      constexpr int32_t CAN = 1 << 30, DEG = CAN - 1;
      // the conflict adjacency with each neighbour replaced by its unit
      std::vector<int32_t> uadj(p->cadj.size());
      parallel_for((int)p->cadj.size(), 1 << 16, [&](int i) { uadj[i] = p->unit_of[p->cadj[i]]; });
      // each unit's state from its own segments (units in parallel), and
      // whether it starts in the queue
      std::vector<int32_t> st((size_t)n, CAN);
      std::vector<uint8_t> first((size_t)n, 0);
      parallel_for(n, 1 << 14, [&](int u) {
        int32_t x = CAN;
        for (int t = p->uptr[u]; t < p->uptr[u + 1]; ++t) {
          const int s = p->useg[t];
          for (int i = p->cptr[s]; i < p->cptr[s + 1]; ++i) {
            if (uadj[i] == u) x &= ~CAN;   // a conflict edge inside the unit
            else x++;
          }
        }
        const bool q = p->uptr[u + 1] > p->uptr[u] && (x & CAN) && (x & DEG) < k;
        st[u] = q ? x & ~CAN : x;
        first[u] = q ? 1 : 0;
      });
      std::vector<int32_t> &queue = p->removed_order;
      queue.reserve((size_t)n);
      for (int u = 0; u < n; ++u)
        if (first[u]) queue.push_back(u);
      // the queue is the removal order; a removed unit's degree is never
      // read again, so its neighbours may still decrement it
      // the walk is bound by memory latency: the units a few places ahead in
      // the queue have their ranges, segments and neighbour states fetched
      // early, one level per distance
      const int32_t *uptr = p->uptr.data(), *useg = p->useg.data(), *cptr = p->cptr.data();
      for (size_t h = 0; h < queue.size(); ++h) {
        const size_t qn = queue.size();
        if (h + 12 < qn) __builtin_prefetch(uptr + queue[h + 12]);
        if (h + 8 < qn) __builtin_prefetch(useg + uptr[queue[h + 8]]);
        if (h + 4 < qn) __builtin_prefetch(cptr + useg[uptr[queue[h + 4]]]);
        if (h + 2 < qn) {
          const int s2 = useg[uptr[queue[h + 2]]];
          for (int i = cptr[s2], e = std::min(cptr[s2 + 1], cptr[s2] + 8); i < e; ++i)
            __builtin_prefetch(st.data() + uadj[i]);
        }
        const int u = queue[h];
        removed[u] = 1;
        for (int t = p->uptr[u]; t < p->uptr[u + 1]; ++t) {
          const int s = p->useg[t];
          for (int i = p->cptr[s]; i < p->cptr[s + 1]; ++i) {
            const int w = uadj[i];
            const int32_t x = --st[w];
            if ((x & CAN) && (x & DEG) < k) {
              queue.push_back(w);
              st[w] = x & ~CAN;
            }
          }
        }
      }
    }

    // ---- sub-graphs: connected components of what remains.  Edges are
    // united in parallel; a link always hangs the larger root under the
    // smaller, so every root is its component's lowest segment whatever the
    // order, and ids follow the lowest segments ascending.
    std::iota(parent.begin(), parent.end(), 0);
    const bool single = (p->flags & MPLD_SINGLE_INSTANCE) != 0;
    std::vector<uint8_t> alive((size_t)n);
    parallel_for(n, 1 << 15, [&](int s) { alive[s] = removed[p->unit_of[s]] ? 0 : 1; });
    if (!single) {
      int32_t *par = parent.data();
      const int mc = (int)p->cu.size(), ms = (int)p->su.size();
      parallel_for(mc + ms, 1 << 14, [&](int e) {
        if (e < mc) {
          if (alive[p->cu[e]] && alive[p->cv[e]]) punite(par, p->cu[e], p->cv[e]);
        } else if (alive[p->su[e - mc]]) {
          punite(par, p->su[e - mc], p->sv[e - mc]);
        }
      });
      // every entry its root
      parallel_for(n, 1 << 15, [&](int x) { __atomic_store_n(par + x, proot(par, x), __ATOMIC_RELAXED); });
    }
    p->comp_of.assign((size_t)n, -1);
    {
      // ids: the roots (lowest alive segments) in ascending order, counted
      // per chunk and numbered from each chunk's offset
      constexpr int G = 1 << 15;
      const int chunks = (n + G - 1) / G;
      std::vector<int32_t> roots((size_t)chunks + 1, 0), live((size_t)chunks + 1, 0);
      parallel_for(chunks, 1, [&](int q) {
        int r = 0, a = 0;
        for (int s = q * G, e = std::min(n, (q + 1) * G); s < e; ++s) {
          if (!alive[s]) continue;
          ++a;
          r += parent[s] == s;
        }
        roots[q + 1] = r;
        live[q + 1] = a;
      });
      for (int q = 0; q < chunks; ++q) {
        roots[q + 1] += roots[q];
        live[q + 1] += live[q];
      }
      const int n_alive = live[chunks];
      p->n_comp = single ? (n_alive > 0 ? 1 : 0) : roots[chunks];
      // every segment is either in a removed unit or in an instance
      p->n_removed_segments = n - n_alive;
      std::vector<int32_t> id_of(single ? 0 : (size_t)n, -1);
      if (!single)
        parallel_for(chunks, 1, [&](int q) {
          int id = roots[q];
          for (int s = q * G, e = std::min(n, (q + 1) * G); s < e; ++s)
            if (alive[s] && parent[s] == s) id_of[s] = id++;
        });
      parallel_for(n, 1 << 15, [&](int s) {
        if (alive[s]) p->comp_of[s] = single ? 0 : id_of[parent[s]];
      });
      // each instance's segments ascending: in order per chunk for a single
      // instance, else one pass in segment order (one counter per instance:
      // a giant instance would have every thread increment the same one)
      const int C0 = p->n_comp;
      p->comp_ptr.assign((size_t)C0 + 1, 0);
      p->comp_seg.resize((size_t)n_alive);
      if (single) {
        if (C0) p->comp_ptr[1] = n_alive;
        parallel_for(chunks, 1, [&](int q) {
          int t = live[q];
          for (int s = q * G, e = std::min(n, (q + 1) * G); s < e; ++s)
            if (alive[s]) p->comp_seg[t++] = s;
        });
      } else {
        for (int s = 0; s < n; ++s)
          if (alive[s]) p->comp_ptr[p->comp_of[s] + 1]++;
        for (int c = 0; c < C0; ++c) p->comp_ptr[c + 1] += p->comp_ptr[c];
        std::vector<int32_t> fill(p->comp_ptr.begin(), p->comp_ptr.end() - 1);
        for (int s = 0; s < n; ++s)
          if (alive[s]) p->comp_seg[fill[p->comp_of[s]]++] = s;
      }
    }
    int C = p->n_comp;
    if (p->flags & MPLD_BICONNECTED) {
      // the search instances become the biconnected blocks of each component
      std::vector<int32_t> iptr{0}, iseg, iatt, loc((size_t)n, -1);
      for (int c = 0; c < C; ++c) {
        const std::vector<int32_t> seg(p->comp_seg.begin() + p->comp_ptr[c],
                                       p->comp_seg.begin() + p->comp_ptr[c + 1]);
        component_blocks(seg, p->cptr, p->cadj, sptr, sadj, loc, iptr, iseg, iatt);
      }
      p->n_comp = (int)iatt.size();
      p->comp_ptr = std::move(iptr);
      p->comp_seg = std::move(iseg);
      p->inst_attach = std::move(iatt);
      std::fill(p->comp_of.begin(), p->comp_of.end(), -1);
      for (int c = p->n_comp - 1; c >= 0; --c)
        for (int t = p->comp_ptr[c]; t < p->comp_ptr[c + 1]; ++t) p->comp_of[p->comp_seg[t]] = c;
    }
    C = p->n_comp;
    for (int c = 0; c < C; ++c) {
      const int sz = p->comp_ptr[c + 1] - p->comp_ptr[c];
      p->max_component = std::max(p->max_component, sz);
      if (sz > MPLD_MAX_INSTANCE_SEGMENTS) { delete p; return MPLD_E_TOO_LARGE; }
    }
    p->instance_segments = p->comp_ptr[C];
    // ---- pack each instance: read-only block + descriptor.  Instances are
    // packed in parallel; a segment's local id in an instance is found by
    // binary search in the instance's ascending segment list (a segment may
    // sit in several blocks).
    // when the instances are whole components each segment has one, and its
    // local id is looked up directly
    const bool blocks = !p->inst_attach.empty();
    std::vector<int32_t> lid_of;
    if (!blocks) {
      lid_of.assign((size_t)n, -1);
      parallel_for(C, 1 << 10, [&](int c) {
        for (int t = p->comp_ptr[c]; t < p->comp_ptr[c + 1]; ++t)
          lid_of[p->comp_seg[t]] = t - p->comp_ptr[c];
      });
    }
    auto local_of = [&](int c, int g) -> int {
      if (!blocks) return p->comp_of[g] == c ? lid_of[g] : -1;
      const int32_t *first = p->comp_seg.data() + p->comp_ptr[c];
      const int32_t *last = p->comp_seg.data() + p->comp_ptr[c + 1];
      const int32_t *it = std::lower_bound(first, last, g);
      return (it != last && *it == g) ? (int)(it - first) : -1;
    };
    // instances are packed largest first, one per task, so that the few
    // large ones start at once on different threads
    std::vector<int32_t> by_size((size_t)C);
    std::iota(by_size.begin(), by_size.end(), 0);
    std::stable_sort(by_size.begin(), by_size.end(), [&](int x, int y) {
      return p->comp_ptr[x + 1] - p->comp_ptr[x] > p->comp_ptr[y + 1] - p->comp_ptr[y];
    });
    p->ro_off.resize((size_t)C);
    p->footprint.resize((size_t)C);
    p->inst_nq.assign((size_t)C, 0);
    p->inst_ne2.resize((size_t)C);
    p->h_desc.resize((size_t)C);
    std::vector<int32_t> ns2v((size_t)C), mask_off((size_t)C), maxdeg((size_t)C);
    std::vector<int64_t> maxinc((size_t)C);
    uint64_t arena = 0, scratch = 0;
    std::vector<uint64_t> scratch_off((size_t)C);
    const bool cliques = (p->flags & MPLD_CLIQUE_BOUND) != 0;
    std::vector<std::vector<uint16_t>> inst_q((size_t)(cliques ? C : 0));
    // pass 1: sizes, degrees, cliques
    parallel_strided(C, 256, [&](int job) {
      const int c = by_size[job];
      const int a = p->comp_ptr[c], b = p->comp_ptr[c + 1], nc = b - a;
      int ne2 = 0, ns2 = 0, mdc = 0, mds = 0;
      int64_t max_inc = 0;
      std::vector<int32_t> lp, la;
      if (cliques) lp.assign((size_t)nc + 1, 0);
      for (int t = a; t < b; ++t) {
        const int s = p->comp_seg[t];
        int dc = 0, ds = 0;
        for (int i = p->cptr[s]; i < p->cptr[s + 1]; ++i) {
          const int l = local_of(c, p->cadj[i]);
          if (l < 0) continue;
          ++dc;
          if (cliques) la.push_back(l);
        }
        for (int i = sptr[s]; i < sptr[s + 1]; ++i) ds += local_of(c, sadj[i]) >= 0;
        if (cliques) lp[t - a + 1] = (int32_t)la.size();
        ne2 += dc;
        ns2 += ds;
        mdc = std::max(mdc, dc);
        mds = std::max(mds, ds);
        max_inc = std::max(max_inc, p->Cc * dc + p->Cs * ds);
      }
      if (cliques) inst_q[c] = greedy_cliques(nc, k + 1, lp, la);
      p->inst_ne2[c] = ne2;
      ns2v[c] = ns2;
      maxdeg[c] = std::min(mdc, 0xFFFF) | (std::min(mds, 0x7FFF) << 16);
      maxinc[c] = max_inc;
    });
    for (int c = 0; c < C; ++c) {
      const int nc = p->comp_ptr[c + 1] - p->comp_ptr[c];
      const int ne2 = p->inst_ne2[c], ns2 = ns2v[c];
      // the kernel orders a segment's rows by 32-bit keys (added cost << 3 |
      // mask) and keeps path costs in 32 bits
      if (maxinc[c] >= (int64_t)1 << 28 ||
          p->Cc * (ne2 / 2) + p->Cs * (ns2 / 2) >= ((int64_t)1 << 31) - 1 ||
          (cliques && inst_q[c].size() / (size_t)(k + 1) > 65535)) {
        delete p;
        return MPLD_E_TOO_LARGE;
      }
      const int nq = cliques ? (int)(inst_q[c].size() / (size_t)(k + 1)) : 0;
      const mpld::RoLayout R = mpld::ro_layout(nc, ne2, ns2, nq * (k + 1));
      p->ro_off[c] = arena;
      arena += R.bytes;
      scratch_off[c] = scratch;
      scratch += mpld::search_state_bytes(nc, ne2, k, nq);
      p->footprint[c] = mpld::search_footprint(nc, ne2, ns2, k, nq);
      p->inst_nq[c] = nq;
      mask_off[c] = p->comp_ptr[c];
    }
    p->arena_bytes = (size_t)arena;
    p->scratch_bytes = (size_t)scratch;
    p->h_arena.assign((size_t)arena, 0);
    // pass 2: the read-only blocks
    parallel_strided(C, 256, [&](int job) {
      const int c = by_size[job];
      const int a = p->comp_ptr[c], b = p->comp_ptr[c + 1], nc = b - a;
      const int nq = p->inst_nq[c];
      const mpld::RoLayout R = mpld::ro_layout(nc, p->inst_ne2[c], ns2v[c], nq * (k + 1));
      uint8_t *blk = p->h_arena.data() + p->ro_off[c];
      if (nq > 0) {
        // each segment's cliques, in clique order
        int32_t *qptr = (int32_t *)(blk + R.qptr);
        uint16_t *qlist = (uint16_t *)(blk + R.qlist);
        std::vector<int32_t> cnt((size_t)nc + 1, 0);
        for (uint16_t m : inst_q[c]) cnt[m + 1]++;
        for (int v = 0; v < nc; ++v) cnt[v + 1] += cnt[v];
        for (int v = 0; v <= nc; ++v) qptr[v] = cnt[v];
        for (int q = 0; q < nq; ++q)
          for (int i = 0; i <= k; ++i) qlist[cnt[inst_q[c][q * (k + 1) + i]]++] = (uint16_t)q;
      }
      int32_t *ptr = (int32_t *)(blk + R.ptr);   // {conflict, stitch} offset pairs
      uint16_t *cn = (uint16_t *)(blk + R.cnbr);
      uint16_t *sn = (uint16_t *)(blk + R.snbr);
      int ci = 0, si = 0;
      for (int t = a; t < b; ++t) {
        const int s = p->comp_seg[t];
        ptr[2 * (t - a)] = ci;
        ptr[2 * (t - a) + 1] = si;
        for (int i = p->cptr[s]; i < p->cptr[s + 1]; ++i) {
          const int l = local_of(c, p->cadj[i]);
          if (l >= 0) cn[ci++] = (uint16_t)l;
        }
        for (int i = sptr[s]; i < sptr[s + 1]; ++i) {
          const int l = local_of(c, sadj[i]);
          if (l >= 0) sn[si++] = (uint16_t)l;
        }
      }
      ptr[2 * nc] = ci;
      ptr[2 * nc + 1] = si;
      if (nc <= mpld::LANE_MAX_N) {
        // the neighbours of each segment as bit masks (the per-lane search)
        uint64_t *bits = (uint64_t *)(blk + R.bits);
        for (int v = 0; v < nc; ++v) {
          uint64_t cm = 0, sm = 0;
          for (int i = ptr[2 * v]; i < ptr[2 * v + 2]; ++i) cm |= 1ull << cn[i];
          for (int i = ptr[2 * v + 1]; i < ptr[2 * v + 3]; ++i) sm |= 1ull << sn[i];
          bits[v] = cm;
          bits[nc + v] = sm;
        }
      }
      // breadth-first ranks over conflict and stitch edges (local ids):
      // roots ascending, each segment's neighbours ascending, once each
      uint16_t *rank = (uint16_t *)(blk + R.rank);
      uint16_t *order = (uint16_t *)(blk + R.order);
      std::vector<uint8_t> seen((size_t)nc, 0);
      int nxt = 0, qh = 0;
      for (int r = 0; r < nc; ++r) {
        if (seen[r]) continue;
        seen[r] = 1;
        rank[r] = (uint16_t)nxt;
        order[nxt++] = (uint16_t)r;
        qh = nxt - 1;
        while (qh < nxt) {
          const int u = order[qh++];
          int i = ptr[2 * u], j = ptr[2 * u + 1];
          const int ie = ptr[2 * u + 2], je = ptr[2 * u + 3];
          while (i < ie || j < je) {
            int w;
            if (j >= je || (i < ie && cn[i] <= sn[j])) {
              w = cn[i++];
              if (j < je && sn[j] == w) ++j;
            } else {
              w = sn[j++];
            }
            if (!seen[w]) {
              seen[w] = 1;
              rank[w] = (uint16_t)nxt;
              order[nxt++] = (uint16_t)w;
            }
          }
        }
      }
    });
    // largest first (ties: lower instance id first)
    p->h_order.resize((size_t)C);
    std::iota(p->h_order.begin(), p->h_order.end(), 0);
    std::stable_sort(p->h_order.begin(), p->h_order.end(), [&](int x, int y) {
      const int sx = p->comp_ptr[x + 1] - p->comp_ptr[x], sy = p->comp_ptr[y + 1] - p->comp_ptr[y];
      if (sx != sy) return sx > sy;
      return p->inst_ne2[x] > p->inst_ne2[y];
    });

    for (int c = 0; c < C; ++c) {
      InstDesc &d = p->h_desc[c];
      std::memset(&d, 0, sizeof(d));
      const int nc = p->comp_ptr[c + 1] - p->comp_ptr[c];
      d.n = nc;
      d.maxdeg = maxdeg[c];
      d.ne2 = p->inst_ne2[c];
      d.ns2 = ns2v[c];
      d.nq = p->inst_nq[c];
      d.ro_bytes = (int32_t)mpld::ro_layout(nc, d.ne2, d.ns2, d.nq * (k + 1)).bytes;
      d.state_bytes = (int32_t)mpld::search_state_bytes(nc, d.ne2, k, d.nq);
      d.k = k;
      d.cost_conflict = (int32_t)p->Cc;
      d.cost_stitch = (int32_t)p->Cs;
      d.idx = c;
    }
    if (p->flags & MPLD_HOST_ONLY) {
      *out = p;
      return MPLD_OK;
    }
    // ---- device memory: one allocation, 256-byte aligned sections
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    p->mask_bytes = (size_t)std::max<int64_t>(p->instance_segments, 1);
    const size_t o_arena = 0;
    const size_t o_scratch = al(o_arena + std::max<size_t>(p->arena_bytes, 16));
    const size_t o_desc = al(o_scratch + std::max<size_t>(p->scratch_bytes, 16));
    const size_t o_order = al(o_desc + sizeof(InstDesc) * (size_t)std::max(C, 1));
    const size_t o_res = al(o_order + sizeof(int32_t) * (size_t)std::max(C, 1));
    const size_t o_masks = al(o_res + sizeof(InstResult) * (size_t)std::max(C, 1));
    const size_t o_queue = al(o_masks + p->mask_bytes);
    const size_t total = al(o_queue + 256);
    const cudaError_t me = cudaMalloc((void **)&p->d_base, total);
    if (me != cudaSuccess) {
      cudaGetLastError();
      delete p;
      return me == cudaErrorMemoryAllocation ? MPLD_E_OOM : MPLD_E_CUDA;
    }
    p->d_bytes = total;
    p->d_arena = p->d_base + o_arena;
    p->d_scratch = p->d_base + o_scratch;
    p->d_desc = (InstDesc *)(p->d_base + o_desc);
    p->d_order = (int32_t *)(p->d_base + o_order);
    p->d_res = (InstResult *)(p->d_base + o_res);
    p->d_masks = (int8_t *)(p->d_base + o_masks);
    p->d_queue = (uint32_t *)(p->d_base + o_queue);
    p->d_err = (int32_t *)(p->d_base + o_queue + 64);
    if (cudaMallocHost((void **)&p->h_res, sizeof(InstResult) * (size_t)std::max(C, 1)) != cudaSuccess ||
        cudaMallocHost((void **)&p->h_masks, p->mask_bytes) != cudaSuccess ||
        cudaMallocHost((void **)&p->h_err, 64) != cudaSuccess) {
      cudaGetLastError();
      mpld_free(p);
      return MPLD_E_OOM;
    }
    for (int c = 0; c < C; ++c) {
      InstDesc &d = p->h_desc[c];
      d.ro = p->d_arena + p->ro_off[c];
      d.scratch = p->d_scratch + scratch_off[c];
      d.mask = p->d_masks + mask_off[c];
      d.res = p->d_res + c;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = MPLD_OK;
    if (p->arena_bytes)
      rc |= cuda_ok(cudaMemcpyAsync(p->d_arena, p->h_arena.data(), p->arena_bytes,
                                    cudaMemcpyHostToDevice, st));
    if (C) {
      rc |= cuda_ok(cudaMemcpyAsync(p->d_desc, p->h_desc.data(), sizeof(InstDesc) * (size_t)C,
                                    cudaMemcpyHostToDevice, st));
      rc |= cuda_ok(cudaMemcpyAsync(p->d_order, p->h_order.data(), sizeof(int32_t) * (size_t)C,
                                    cudaMemcpyHostToDevice, st));
    }
    rc |= cuda_ok(cudaMemsetAsync(p->d_queue, 0, 256, st));
    rc |= cuda_ok(cudaStreamSynchronize(st));
    if (rc != MPLD_OK) {
      mpld_free(p);
      return MPLD_E_CUDA;
    }
  } catch (const std::bad_alloc &) {
    delete p;
    return MPLD_E_OOM;
  }
  *out = p;
  return MPLD_OK;
}

extern "C" void mpld_free(mpld_problem *p) {
  if (!p) return;
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->d_base) cudaFree(p->d_base);
  if (p->d_par) cudaFree(p->d_par);
  if (p->d_split) cudaFree(p->d_split);
  if (p->h_res) cudaFreeHost(p->h_res);
  if (p->h_masks) cudaFreeHost(p->h_masks);
  if (p->h_err) cudaFreeHost(p->h_err);
  delete p;
}

// ================================================================= launch

namespace {

int64_t time_limit_ns(const mpld_params *prm) {
  const int64_t ms = (prm && prm->time_limit_ms > 0) ? prm->time_limit_ms : DEFAULT_TIME_LIMIT_MS;
  return ms * 1000000ll;
}
int64_t budget_of(const mpld_params *prm) { return prm ? std::max<int64_t>(prm->node_budget, 0) : 0; }
int rule_of(const mpld_params *prm) { return (prm && (prm->flags & MPLD_COLUMN_BFS)) ? 1 : 0; }
// Parallel exact mode: instances of at least PAR_MIN_SEGMENTS segments are
// searched by a CTA whose warps split the subtrees.
constexpr int PAR_MIN_SEGMENTS = 16;
int par_of(const mpld_params *prm) { return (prm && (prm->flags & MPLD_PARALLEL_EXACT)) ? 1 : 0; }
int split_of(const mpld_params *prm) { return (prm && (prm->flags & MPLD_SPLIT_BUDGET)) ? 1 : 0; }
// The split exact search is exact only: with a node budget the nodes a
// subtree counts would depend on the order the warps finish.  The budgeted
// split search has its own per-search budgets and cannot be combined with it.
bool params_ok(const mpld_params *prm) {
  return !(par_of(prm) && budget_of(prm) != 0) && !(par_of(prm) && split_of(prm));
}
// The budgeted split search's subtree searches have no clique bound: a
// problem built with it is refused.
bool split_ok(const mpld_problem *p) {
  for (int32_t q : p->inst_nq)
    if (q > 0) return false;
  return true;
}
int cta_min_of(const mpld_params *prm) {
  if (par_of(prm)) return PAR_MIN_SEGMENTS;
  if (prm && prm->cta_segments < 0) return std::numeric_limits<int>::max();
  return (prm && prm->cta_segments > 0) ? prm->cta_segments : DEFAULT_CTA_SEGMENTS;
}
// Instances searched by a whole CTA: the leading entries of a largest-first
// order whose instance has at least `min_segments` segments.
template <typename SizeAt>
int count_large(int total, SizeAt size_at, int min_segments) {
  int nl = 0;
  while (nl < total && size_at(nl) >= min_segments) ++nl;
  return nl;
}

uint32_t max_footprint(mpld_problem *const *ps, int n) {
  uint32_t m = 0;
  for (int i = 0; i < n; ++i)
    for (uint32_t f : ps[i]->footprint) m = std::max(m, f);
  return m;
}

// Launch shape: explicit params, else the tuned cache entry, else a default
// that fits every instance of the batch in shared memory when possible.
Shape pick_shape(mpld_problem *const *ps, int n, const mpld_params *prm) {
  int nw = prm && prm->warps_per_cta > 0 ? prm->warps_per_cta : 0;
  int slot = prm && prm->slot_bytes > 0 ? prm->slot_bytes : 0;
  if (!nw || !slot) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(ps, n, prm));
    if (it != g_tune_cache.end()) {
      if (!nw) nw = it->second.warps_per_cta;
      if (!slot) slot = it->second.slot_bytes;
    }
  }
  if (!nw) nw = 4;
  nw = std::max(1, std::min(nw, 16));   // the kernel's launch bound: 512 threads
  const int maxslot = mpld_internal_max_slot_bytes(nw);
  if (!slot) slot = (int)mpld::align16(std::max<uint32_t>(max_footprint(ps, n), 16));
  slot = std::max(16, std::min(slot, maxslot)) & ~15;
  int per_sm = mpld_internal_ctas_per_sm(nw, slot);
  if (per_sm < 1) per_sm = 1;
  const int sms = std::max(1, mpld_internal_num_sms());
  return Shape{nw, slot, per_sm * sms};
}

// A shape with enough warps per CTA for the whole-CTA teams, when the launch
// has large instances.
Shape with_team(Shape sh, int n_large) {
  if (n_large <= 0 || sh.nw >= CTA_TEAM_WARPS) return sh;
  sh.nw = CTA_TEAM_WARPS;
  sh.slot = std::max(16, std::min(sh.slot, mpld_internal_max_slot_bytes(sh.nw))) & ~15;
  const int per_sm = std::max(1, mpld_internal_ctas_per_sm(sh.nw, sh.slot));
  sh.ctas = per_sm * std::max(1, mpld_internal_num_sms());
  return sh;
}

// Grid-wide split search of one instance: every warp of a full grid of
// 8-warp CTAs takes subtrees of it.  Used when a launch holds that instance
// alone (the plain path, a one-instance problem) and it fits the register
// form.
struct GridSplit {
  bool on = false;
  int slot = 0, ctas = 0;
  size_t bytes = 0;
};
GridSplit grid_split_of(const mpld_problem *p, int c, const mpld_params *prm) {
  GridSplit g;
  const InstDesc &d = p->h_desc[c];
  if (!par_of(prm) || d.n < PAR_MIN_SEGMENTS || !mpld::reg_fits(d.n, d.k)) return g;
  g.slot = (int)mpld::align16(mpld::reg_layout(d.n, d.k, 0).bytes);
  if (g.slot > mpld_internal_max_slot_bytes(CTA_TEAM_WARPS)) return g;
  const int per_sm = std::max(1, mpld_internal_ctas_per_sm(CTA_TEAM_WARPS, g.slot));
  g.ctas = per_sm * std::max(1, mpld_internal_num_sms());
  g.bytes = mpld::par_layout(g.ctas * CTA_TEAM_WARPS, d.n).bytes;
  g.on = true;
  return g;
}
// Grow the problem's split-context buffer (outside any stream capture).
int ensure_par_buf(mpld_problem *p, size_t bytes) {
  if (bytes <= p->par_bytes) return MPLD_OK;
  p->queue_ready = false;
  if (p->gexec) {   // a captured graph may hold the old buffer's address
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  if (p->d_par) {
    cudaFree(p->d_par);
    p->d_par = nullptr;
    p->par_bytes = 0;
  }
  if (cudaMalloc((void **)&p->d_par, bytes) != cudaSuccess) {
    cudaGetLastError();
    p->d_par = nullptr;
    return MPLD_E_OOM;
  }
  p->par_bytes = bytes;
  return MPLD_OK;
}
// Reset the context (no incumbent, every warp key ~0, totals 0) and launch.
int launch_grid_split(mpld_problem *p, int c, const GridSplit &g, const mpld_params *prm,
                      cudaStream_t st) {
  const int G = g.ctas * CTA_TEAM_WARPS;
  const mpld::ParLayout PL = mpld::par_layout(G, p->h_desc[c].n);
  int rc = cuda_ok(cudaMemsetAsync(p->d_par, 0xFF, PL.ctx + 8, st));
  rc |= cuda_ok(cudaMemsetAsync(p->d_par + PL.ctx + 8, 0, PL.bestx - PL.ctx - 8, st));
  if (rc) return MPLD_E_CUDA;
  mpld::LaunchArgs a;
  a.desc = p->d_desc + c;
  a.order = nullptr;
  a.n_inst = 1;
  a.slot_bytes = g.slot;
  a.queue = nullptr;
  a.err = p->d_err;
  a.budget = 0;
  a.time_limit_ns = time_limit_ns(prm);
  a.rule = rule_of(prm);
  a.n_large = 0;
  a.par = 2;
  a.split = 0;
  a.par_buf = p->d_par;
  return mpld_internal_launch(&a, g.ctas, CTA_TEAM_WARPS, st);
}

// Split-search queue of a batched problem: the PAR_QUEUE_MAX largest
// instances of at least PAR_MIN_SEGMENTS segments that fit the register form
// are split by every warp of the grid, one after another, in a launch before
// the batched one; the batched launch takes the rest (its own order, with the
// other split instances on CTAs).  Device block: 64-byte contexts, the
// queue's instance indices, the rest of the largest-first order.
constexpr int PAR_QUEUE_MAX = 16;
struct QueuePlan {
  int nq = 0, slot = 0, ctas = 0;
  std::vector<int32_t> idx, rest;
  size_t o_idx = 0, o_rest = 0, bytes = 0;
};
QueuePlan queue_plan_of(const mpld_problem *p, const mpld_params *prm) {
  QueuePlan q;
  if (!par_of(prm) || p->n_comp < 2) return q;
  const int maxslot = mpld_internal_max_slot_bytes(CTA_TEAM_WARPS);
  for (int i = 0; i < p->n_comp; ++i) {
    const int c = p->h_order[i];
    const InstDesc &d = p->h_desc[c];
    bool queued = false;
    if ((int)q.idx.size() < PAR_QUEUE_MAX && d.n >= PAR_MIN_SEGMENTS && mpld::reg_fits(d.n, d.k)) {
      const int sl = (int)mpld::align16(mpld::reg_layout(d.n, d.k, 0).bytes);
      if (sl <= maxslot) {
        q.idx.push_back(c);
        q.slot = std::max(q.slot, sl);
        queued = true;
      }
    }
    if (!queued) q.rest.push_back(c);
  }
  q.nq = (int)q.idx.size();
  if (!q.nq) return QueuePlan{};
  const int per_sm = std::max(1, mpld_internal_ctas_per_sm(CTA_TEAM_WARPS, q.slot));
  q.ctas = per_sm * std::max(1, mpld_internal_num_sms());
  q.o_idx = (64u * (size_t)q.nq + 255) & ~(size_t)255;
  q.o_rest = (q.o_idx + 4u * (size_t)q.nq + 255) & ~(size_t)255;
  q.bytes = q.o_rest + 4u * std::max<size_t>(q.rest.size(), 1);
  return q;
}
// Make the queue's device block ready (outside any stream capture).
int ensure_queue(mpld_problem *p, const QueuePlan &q) {
  if (ensure_par_buf(p, q.bytes) != MPLD_OK) return MPLD_E_OOM;
  if (p->queue_ready) return MPLD_OK;
  int rc = cuda_ok(cudaMemcpy(p->d_par + q.o_idx, q.idx.data(), 4u * q.idx.size(),
                              cudaMemcpyHostToDevice));
  if (!q.rest.empty())
    rc |= cuda_ok(cudaMemcpy(p->d_par + q.o_rest, q.rest.data(), 4u * q.rest.size(),
                             cudaMemcpyHostToDevice));
  if (rc) return MPLD_E_CUDA;
  p->queue_ready = true;
  return MPLD_OK;
}
// Reset the queue's contexts (no incumbent, totals 0) and launch it.
int launch_queue(mpld_problem *p, const QueuePlan &q, const mpld_params *prm, cudaStream_t st) {
  int rc = cuda_ok(cudaMemsetAsync(p->d_par, 0, 64u * (size_t)q.nq, st));
  rc |= cuda_ok(cudaMemset2DAsync(p->d_par, 64, 0xFF, 8, (size_t)q.nq, st));   // keys
  if (rc) return MPLD_E_CUDA;
  mpld::LaunchArgs a;
  a.desc = p->d_desc;
  a.order = (const int32_t *)(p->d_par + q.o_idx);
  a.n_inst = q.nq;
  a.slot_bytes = q.slot;
  a.queue = nullptr;
  a.err = p->d_err;
  a.budget = 0;
  a.time_limit_ns = time_limit_ns(prm);
  a.rule = rule_of(prm);
  a.n_large = 0;
  a.par = 3;
  a.split = 0;
  a.par_buf = p->d_par;
  return mpld_internal_launch(&a, q.ctas, CTA_TEAM_WARPS, st);
}

}  // namespace

// Budgeted split search (MPLD_SPLIT_BUDGET): the first phase is the batched
// (or plain) launch with split = 1, which searches every instance with its
// per-search budget and puts the ones that stop on it on a hard list; the
// second launch (par = 4) searches their subtrees, a lane or a warp per
// subtree.  Device block: the three hard lists (counts, then descriptor
// indices), one 64-byte context per descriptor, then the general-state
// region of each of the first gen_warps warps.
mpld::SplitPlan mpld::split_plan(const InstDesc *desc, int n_inst, const mpld_params *prm,
                                 size_t gen_cap_bytes) {
  SplitPlan q;
  if (!prm || !(prm->flags & MPLD_SPLIT_BUDGET) || n_inst < 1) return q;
  q.on = true;
  int reg_slot = 16;
  size_t gen = 0;
  // slot bytes that hold the largest general-form state with the read-only
  // block after it (the breadth-first tables only under column rule 1)
  uint32_t gen_slot = 0;
  const bool rule1 = (prm->flags & MPLD_COLUMN_BFS) != 0;
  bool any_reg = false;
  for (int i = 0; i < n_inst; ++i) {
    const InstDesc &d = desc[i];
    if (d.n > SPLIT_MAX_N) continue;   // never split
    int D;
    uint32_t S;
    split_cut(d.n, d.k, D, S);
    q.smax = std::max(q.smax, (int)S);
    const int list = split_list_of(d.n, d.k);
    if (list == 0) {
      reg_slot = std::max(reg_slot, (int)align16(reg_layout(d.n, d.k, 0).bytes));
      any_reg = true;
    }
    if (list == 2) {
      gen = std::max(gen, (size_t)d.state_bytes);
      const RoLayout R = ro_layout(d.n, d.ne2, d.ns2, 0);
      gen_slot = std::max(gen_slot, align16(state_layout(d.n, d.ne2, d.k, 0).bytes) +
                                        (rule1 ? R.bytes : R.rank));
    }
  }
  // with no register-form subtrees to share the SMs with, the slots are
  // sized for the general form's state and read-only block when they fit,
  // and every warp takes general-form subtrees with no global region;
  // otherwise the general form uses a warp's slot only when it fits there
  const bool gen_in_slot =
      !any_reg && gen_slot > 0 && (int)gen_slot <= mpld_internal_max_slot_bytes(1);
  if (gen_in_slot) reg_slot = std::max(reg_slot, (int)gen_slot);
  // as many warps per CTA as the slots allow (the launch bound is 16)
  q.nw = 1;
  for (int nw = 16; nw >= 1; --nw)
    if (mpld_internal_max_slot_bytes(nw) >= reg_slot) { q.nw = nw; break; }
  q.slot = reg_slot;
  const int per_sm = std::max(1, mpld_internal_ctas_per_sm(q.nw, q.slot));
  q.ctas = per_sm * std::max(1, mpld_internal_num_sms());
  q.state_bytes = (gen && !gen_in_slot) ? (int)((gen + 255) & ~(size_t)255) : 0;
  const int G = q.ctas * q.nw;
  q.gen_warps = gen_in_slot ? G
      : q.state_bytes
      ? (int)std::max<size_t>(1, std::min<size_t>((size_t)G, gen_cap_bytes / (size_t)q.state_bytes))
      : 0;
  q.cap = n_inst;
  // the lanes' list holds at most the instances the per-lane search takes
  int lane_cap = 0;
  for (int i = 0; i < n_inst; ++i)
    if (desc[i].n <= SPLIT_MAX_N && split_list_of(desc[i].n, desc[i].k) == 1) ++lane_cap;
  q.o_hard = 0;
  q.o_ctx = (4u * (size_t)(4 + 3 * n_inst) + 255) & ~(size_t)255;
  q.o_state = q.o_ctx + 64u * (size_t)n_inst;
  q.o_lmask = q.o_state + (size_t)q.gen_warps * (size_t)q.state_bytes;
  q.bytes = q.o_lmask + 16u * (size_t)lane_cap * (size_t)q.smax;
  return q;
}
// First-phase fields of a launch over `buf` (the plan's block).
void mpld::split_phase1_args(LaunchArgs &a, const SplitPlan &q, uint8_t *buf) {
  a.split = q.on ? 1 : 0;
  a.hard = q.on ? (int32_t *)(buf + q.o_hard) : nullptr;
  a.hard_cap = q.cap;
  a.par_buf = q.on ? buf + q.o_ctx : a.par_buf;
}
int mpld::split_warp_prefix(const InstDesc *h_desc, const int32_t *h_order, int n, int n_large) {
  auto lane = [&](int i) {
    const InstDesc &d = h_desc[h_order[i]];
    return d.n <= SPLIT_MAX_N && split_list_of(d.n, d.k) == 1;
  };
  int p = 0;
  while (p < n && !lane(p)) ++p;
  for (int i = p; i < n; ++i)
    if (!lane(i)) return n;
  return std::max(p, std::min(n_large, n));
}
int mpld::split_phase1_launch(const LaunchArgs &a, int ctas, int nw, int n_w, cudaStream_t st) {
  if (a.n_inst == 0) return MPLD_OK;
  int rc = MPLD_OK, c = 0;
  if (n_w > 0) {
    LaunchArgs w = a;
    w.n_inst = n_w;
    c = std::max(1, std::min(ctas, a.n_large + (n_w - a.n_large + nw - 1) / nw));
    rc = mpld_internal_launch(&w, c, nw, st);
  }
  if (rc || n_w >= a.n_inst) return rc;
  LaunchArgs l = a;
  l.order = a.order + n_w;
  l.n_inst = a.n_inst - n_w;
  l.n_large = 0;
  l.lane_phase1 = 1;
  if (n_w == 0) return mpld_internal_launch_lanes(&l, st);
  // a lane block takes a whole SM: one per SM the warps' CTAs leave free, so
  // that no block (and none of the instances it holds) waits for them
  const int sms = std::max(1, mpld_internal_num_sms());
  return mpld_internal_launch_lanes_overlapped(&l, c < sms ? sms - c : 0, st);
}
// Reset the hard lists before the first phase.
int mpld::split_reset(const SplitPlan &q, uint8_t *buf, cudaStream_t st) {
  return cudaMemsetAsync(buf + q.o_hard, 0, 16, st) == cudaSuccess ? MPLD_OK : MPLD_E_CUDA;
}
// The second launch, after the first on the same stream: its item counters
// (queue[0..2]) are reset, then every warp of the grid takes subtrees.
int mpld::split_phase2_launch(const LaunchArgs &a1, const InstDesc *desc, const SplitPlan &q,
                              uint8_t *buf, uint32_t *queue, cudaStream_t st) {
  if (cudaMemsetAsync(queue, 0, 16, st) != cudaSuccess) return MPLD_E_CUDA;
  LaunchArgs a = a1;
  a.desc = desc;   // the hard lists hold indices into the whole descriptor array
  a.order = nullptr;
  a.slot_bytes = q.slot;
  a.queue = queue;
  a.n_large = 0;
  a.par = 4;
  a.split = 0;
  a.hard = (int32_t *)(buf + q.o_hard);
  a.hard_cap = q.cap;
  a.par_buf = buf + q.o_ctx;
  a.split_scratch = q.state_bytes ? buf + q.o_state : nullptr;
  a.lane_masks = (unsigned long long *)(buf + q.o_lmask);
  a.split_gen_warps = q.gen_warps;
  a.smax = q.smax;
  a.split_state_bytes = q.state_bytes;
  // the lanes' subtrees in a kernel of their own, then the warps' (other
  // instances, other counters): that launch's blocks take SMs as the lanes'
  // blocks finish, and it completes only after the lanes' kernel
  const int rc = mpld_internal_launch_lanes(&a, st);
  if (rc) return rc;
  return mpld_internal_launch_overlapped(&a, q.ctas, q.nw, st);
}

namespace {

using mpld::SplitPlan;
// general-state regions of a batched call: at most this many bytes
constexpr size_t SPLIT_GEN_BYTES = (size_t)1 << 30;
SplitPlan split_plan_of(const InstDesc *desc, int n_inst, const mpld_params *prm) {
  return mpld::split_plan(desc, n_inst, prm, SPLIT_GEN_BYTES);
}
void split_phase1(mpld::LaunchArgs &a, const SplitPlan &q, uint8_t *buf) {
  mpld::split_phase1_args(a, q, buf);
}
int launch_split_phase2(const mpld::LaunchArgs &a1, const InstDesc *desc, const SplitPlan &q,
                        uint8_t *buf, uint32_t *queue, cudaStream_t st) {
  return mpld::split_phase2_launch(a1, desc, q, buf, queue, st);
}

// Grow the problem's split-search block (outside any stream capture).
int ensure_split_buf(mpld_problem *p, size_t bytes) {
  if (bytes <= p->split_bytes) return MPLD_OK;
  if (p->gexec) {   // a captured graph may hold the old block's address
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  if (p->d_split) {
    cudaFree(p->d_split);
    p->d_split = nullptr;
    p->split_bytes = 0;
  }
  if (cudaMalloc((void **)&p->d_split, bytes) != cudaSuccess) {
    cudaGetLastError();
    p->d_split = nullptr;
    return MPLD_E_OOM;
  }
  p->split_bytes = bytes;
  return MPLD_OK;
}
// n_w (budgeted split search): the first n_w entries of the order go to the
// warps, the rest to the lane kernel beside them (n_w < 0: all to the warps)
int launch_batch(const mpld::LaunchArgs &a, const Shape &sh, cudaStream_t st, uint32_t *queue,
                 int32_t *err, int n_w = -1) {
  int rc = cuda_ok(cudaMemsetAsync(queue, 0, 8, st));   // both work counters
  rc |= cuda_ok(cudaMemsetAsync(err, 0, 4, st));
  if (rc) return MPLD_E_CUDA;
  if (a.n_inst == 0) return MPLD_OK;
  if (a.split && n_w >= 0 && n_w < a.n_inst) return mpld::split_phase1_launch(a, sh.ctas, sh.nw, n_w, st);
  const int ctas = std::min(sh.ctas, a.n_large + (a.n_inst - a.n_large + sh.nw - 1) / sh.nw);
  return mpld_internal_launch(&a, std::max(ctas, 1), sh.nw, st);
}

bool capturable(void *stream) {
  return stream != nullptr && stream != (void *)cudaStreamLegacy &&
         stream != (void *)cudaStreamPerThread;
}

// Enqueue reset -> persistent search -> copy-back for one problem, as a
// captured CUDA graph when the stream allows capture.
int enqueue_single(mpld_problem *p, const mpld_params *prm, void *stream, bool copy_back) {
  if (!params_ok(prm)) return MPLD_E_INVALID;
  if (split_of(prm) && !split_ok(p)) return MPLD_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  mpld_problem *ps[1] = {p};
  const GridSplit gs = p->n_comp == 1 ? grid_split_of(p, 0, prm) : GridSplit{};
  if (gs.on && ensure_par_buf(p, gs.bytes) != MPLD_OK) return MPLD_E_OOM;
  const SplitPlan sp = split_plan_of(p->h_desc.data(), p->n_comp, prm);
  if (sp.on && ensure_split_buf(p, sp.bytes) != MPLD_OK) return MPLD_E_OOM;
  // the largest split instances go to the queue launch; the batched launch
  // then takes the rest in its own order
  const QueuePlan qp = gs.on ? QueuePlan{} : queue_plan_of(p, prm);
  if (qp.nq) {
    const int qrc = ensure_queue(p, qp);
    if (qrc) return qrc;
  }
  const int n_rest = qp.nq ? (int)qp.rest.size() : p->n_comp;
  const int n_large = qp.nq
      ? count_large(n_rest, [&](int i) { return p->h_desc[qp.rest[i]].n; }, cta_min_of(prm))
      : count_large(p->n_comp, [&](int i) { return p->h_desc[p->h_order[i]].n; }, cta_min_of(prm));
  const Shape sh = with_team(pick_shape(ps, 1, prm), n_large);
  mpld::LaunchArgs a;
  a.desc = p->d_desc;
  a.order = qp.nq ? (const int32_t *)(p->d_par + qp.o_rest) : p->d_order;
  a.n_inst = n_rest;
  a.slot_bytes = sh.slot;
  a.queue = p->d_queue;
  a.err = p->d_err;
  a.budget = budget_of(prm);
  a.time_limit_ns = time_limit_ns(prm);
  a.rule = rule_of(prm);
  a.n_large = n_large;
  a.par = par_of(prm);
  a.split = 0;
  a.par_buf = nullptr;
  split_phase1(a, sp, p->d_split);
  auto body = [&]() -> int {
    int rc = cuda_ok(cudaMemsetAsync(p->d_res, 0xFF, sizeof(InstResult) * (size_t)std::max(p->n_comp, 1), st));
    if (rc) return rc;
    if (sp.on) {
      // the first phase over every instance, then the subtrees of the hard ones
      rc = mpld::split_reset(sp, p->d_split, st);
      rc |= launch_batch(a, sh, st, p->d_queue, p->d_err,
                         mpld::split_warp_prefix(p->h_desc.data(), p->h_order.data(), p->n_comp,
                                                 n_large));
      if (rc == MPLD_OK) rc = launch_split_phase2(a, p->d_desc, sp, p->d_split, p->d_queue, st);
    } else if (gs.on) {
      rc = cuda_ok(cudaMemsetAsync(p->d_err, 0, 4, st));
      rc |= launch_grid_split(p, 0, gs, prm, st);
    } else if (qp.nq) {
      rc = cuda_ok(cudaMemsetAsync(p->d_err, 0, 4, st));
      rc |= cuda_ok(cudaMemsetAsync(p->d_queue, 0, 8, st));
      rc |= launch_queue(p, qp, prm, st);
      if (rc == MPLD_OK && n_rest > 0) {
        const int ctas = std::min(sh.ctas, n_large + (n_rest - n_large + sh.nw - 1) / sh.nw);
        rc = mpld_internal_launch(&a, std::max(ctas, 1), sh.nw, st);
      }
    } else {
      rc = launch_batch(a, sh, st, p->d_queue, p->d_err);
    }
    if (rc) return rc;
    if (copy_back) {
      if (p->n_comp)
        rc |= cuda_ok(cudaMemcpyAsync(p->h_res, p->d_res, sizeof(InstResult) * (size_t)p->n_comp,
                                      cudaMemcpyDeviceToHost, st));
      if (p->instance_segments)
        rc |= cuda_ok(cudaMemcpyAsync(p->h_masks, p->d_masks, (size_t)p->instance_segments,
                                      cudaMemcpyDeviceToHost, st));
      rc |= cuda_ok(cudaMemcpyAsync(p->h_err, p->d_err, 4, cudaMemcpyDeviceToHost, st));
    }
    return rc;
  };
  if (!capturable(stream)) return body();
  GraphKey key{sh.nw, sh.slot, sh.ctas, a.budget, a.time_limit_ns, a.rule, a.n_large * 4 + a.par};
  if (gs.on) {
    key.nw = CTA_TEAM_WARPS;
    key.slot = gs.slot;
    key.ctas = gs.ctas;
    key.n_large = 2;
  }
  key.queue_ctas = qp.ctas;
  key.queue_slot = qp.slot;
  key.split_nw = sp.on ? sp.nw : 0;
  key.split_ctas = sp.on ? sp.ctas : 0;
  const int kc = gs.on ? gs.ctas : sh.ctas;
  key.ctas = copy_back ? kc : -kc;  // copy-back variant is a different graph
  if (!p->gexec || !(p->gkey == key) || p->gstream != stream) {
    if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return body();
    }
    const int rc = body();
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc != MPLD_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return MPLD_E_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&p->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) { p->gexec = nullptr; cudaGetLastError(); return MPLD_E_CUDA; }
    p->gkey = key;
    p->gstream = stream;
  }
  return cuda_ok(cudaGraphLaunch(p->gexec, st));
}

}  // namespace

// Host side after the results are in host memory: scatter, recover, count.
int mpld_internal_finish(mpld_problem *p, const InstResult *hres, const int8_t *hmasks,
                         int32_t err, int8_t *mask_out, mpld_result *res) {
  const int C = p->n_comp;
  p->r_nodes.resize((size_t)C);
  p->r_cost.resize((size_t)C);
  p->r_status.resize((size_t)C);
  int status = MPLD_OK, nbud = 0;
  int64_t nodes = 0, csum = 0, work = 0;
  for (int c = 0; c < C; ++c) {
    const InstResult &r = hres[c];
    p->r_nodes[c] = r.nodes;
    p->r_cost[c] = r.cost;
    p->r_status[c] = r.status;
    if (r.status < 0 || r.status > MPLD_TIMEOUT) return MPLD_E_STATE;
    if (r.status != MPLD_OK) { status = MPLD_BUDGET; ++nbud; }
    nodes += r.nodes;
    csum += r.cost;
    work += r.work;
  }
  p->have_results = true;
  std::vector<int8_t> m((size_t)p->n_seg, (int8_t)-1);
  if (p->inst_attach.empty()) {
    // whole components: each segment in one instance
    parallel_for(C, 64, [&](int c) {
      for (int t = p->comp_ptr[c]; t < p->comp_ptr[c + 1]; ++t) m[p->comp_seg[t]] = hmasks[t];
    });
  }
  for (int c = 0; c < C && !p->inst_attach.empty(); ++c) {
    // a block attached at a segment already coloured takes the transposition
    // of masks that keeps that segment's mask (cost does not depend on the
    // names of the masks); instances come in an order where the attach
    // segment is always coloured first
    int from = -1, to = -1;
    const int att = p->inst_attach.empty() ? -1 : p->inst_attach[c];
    if (att >= 0) {
      from = hmasks[p->comp_ptr[c] + att];
      to = m[p->comp_seg[p->comp_ptr[c] + att]];
      if (to < 0) return MPLD_E_STATE;
    }
    for (int t = p->comp_ptr[c]; t < p->comp_ptr[c + 1]; ++t) {
      int x = hmasks[t];
      if (from >= 0) x = x == from ? to : x == to ? from : x;
      m[p->comp_seg[t]] = (int8_t)x;
    }
  }
  // density balance: renaming the masks of one component keeps its cost, so
  // each instance in instance order takes the permutation that pairs its
  // masks by decreasing segment count (lower mask first on ties) with the
  // layout's masks so far by increasing count (lower first); recovery then
  // gives a removed unit the least used of its free masks (lowest on ties)
  const bool balance = (p->flags & MPLD_DENSITY_BALANCE) != 0;
  int64_t tot_mask[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (balance) {
    const int k = p->k;
    for (int c = 0; c < C; ++c) {
      int64_t x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int t = p->comp_ptr[c]; t < p->comp_ptr[c + 1]; ++t) x[m[p->comp_seg[t]]]++;
      int src[8], dst[8], perm[8];
      for (int q = 0; q < k; ++q) src[q] = dst[q] = q;
      std::stable_sort(src, src + k, [&](int a, int b) { return x[a] > x[b]; });
      std::stable_sort(dst, dst + k, [&](int a, int b) { return tot_mask[a] < tot_mask[b]; });
      for (int q = 0; q < k; ++q) perm[src[q]] = dst[q];
      for (int t = p->comp_ptr[c]; t < p->comp_ptr[c + 1]; ++t)
        m[p->comp_seg[t]] = (int8_t)perm[m[p->comp_seg[t]]];
      for (int q = 0; q < k; ++q) tot_mask[perm[q]] += x[q];
    }
  }
  // recovery: reverse removal order, lowest mask unused by coloured neighbours
  // (the least used one under density balance).  Units a few places ahead in
  // that order have their ranges, segments, adjacency and neighbour masks
  // fetched early, as in the peel.
  {
    const int32_t *ro = p->removed_order.data(), *uptr = p->uptr.data(), *useg = p->useg.data(),
                  *cptr = p->cptr.data(), *cadj = p->cadj.data();
    for (int h = (int)p->removed_order.size() - 1; h >= 0; --h) {
      if (h >= 12) __builtin_prefetch(uptr + ro[h - 12]);
      if (h >= 8) __builtin_prefetch(useg + uptr[ro[h - 8]]);
      if (h >= 4) __builtin_prefetch(cadj + cptr[useg[uptr[ro[h - 4]]]]);
      if (h >= 2) {
        const int s2 = useg[uptr[ro[h - 2]]];
        for (int i = cptr[s2], e = std::min(cptr[s2 + 1], cptr[s2] + 8); i < e; ++i)
          __builtin_prefetch(m.data() + cadj[i]);
      }
      const int u = ro[h];
      unsigned used = 0;
      for (int t = uptr[u]; t < uptr[u + 1]; ++t) {
        const int s = useg[t];
        for (int i = cptr[s]; i < cptr[s + 1]; ++i) {
          const int x = m[cadj[i]];
          if (x >= 0) used |= 1u << x;
        }
      }
      int c = 0;
      if (balance) {
        c = -1;
        for (int q = 0; q < p->k; ++q)
          if (!((used >> q) & 1u) && (c < 0 || tot_mask[q] < tot_mask[c])) c = q;
        if (c < 0) c = p->k;
      } else {
        while (c < p->k && ((used >> c) & 1u)) ++c;
      }
      if (c == p->k) return MPLD_E_STATE;
      for (int t = uptr[u]; t < uptr[u + 1]; ++t) m[useg[t]] = (int8_t)c;
      if (balance) tot_mask[c] += uptr[u + 1] - uptr[u];
    }
  }
  // monochromatic conflict edges and cut stitch edges, counted in chunks
  std::atomic<int64_t> nconf_a{0}, nst_a{0};
  const int64_t ne = (int64_t)p->cu.size(), ns = (int64_t)p->su.size();
  constexpr int64_t CHUNK = 1 << 15;
  const int nchunks = (int)((ne + ns + CHUNK - 1) / CHUNK);
  parallel_for(nchunks, 1, [&](int q) {
    int64_t a = 0, b = 0;
    for (int64_t e = (int64_t)q * CHUNK, end = std::min<int64_t>(e + CHUNK, ne + ns); e < end; ++e)
      if (e < ne) a += m[p->cu[e]] == m[p->cv[e]];
      else b += m[p->su[e - ne]] != m[p->sv[e - ne]];
    nconf_a += a;
    nst_a += b;
  });
  const int64_t nconf = nconf_a.load(), nst = nst_a.load();
  const int64_t cost = p->Cc * nconf + p->Cs * nst;
  if (cost != csum) return MPLD_E_STATE;  // removed units must cost nothing
  if (mask_out && p->n_seg) std::memcpy(mask_out, m.data(), (size_t)p->n_seg);
  if (res) {
    res->status = status;
    res->n_components = C;
    res->n_conflicts = nconf;
    res->n_stitches = nst;
    res->cost = cost;
    res->nodes = nodes;
    res->n_removed_segments = p->n_removed_segments;
    res->max_component = p->max_component;
    res->n_budget_components = nbud;
    res->work = work;
  }
  if (err) return err;
  return status;
}

namespace {

int finish(mpld_problem *p, int8_t *mask_out, mpld_result *res) {
  return mpld_internal_finish(p, p->h_res, p->h_masks, *p->h_err, mask_out, res);
}

}  // namespace

extern "C" int mpld_search_plain_async(mpld_problem *p, const mpld_params *prm, void *stream) {
  if (!p || !params_ok(prm)) return MPLD_E_INVALID;
  if (!p->d_base) return MPLD_E_STATE;
  if (split_of(prm) && !split_ok(p)) return MPLD_E_INVALID;
  const SplitPlan sp = split_plan_of(p->h_desc.data(), p->n_comp, prm);
  if (sp.on && ensure_split_buf(p, sp.bytes) != MPLD_OK) return MPLD_E_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = cuda_ok(cudaMemsetAsync(p->d_err, 0, 4, st));
  rc |= cuda_ok(cudaMemsetAsync(p->d_res, 0xFF, sizeof(InstResult) * (size_t)std::max(p->n_comp, 1), st));
  const int maxslot = mpld_internal_max_slot_bytes(1);
  size_t par_need = 0;
  for (int c = 0; c < p->n_comp; ++c) {
    const GridSplit g = grid_split_of(p, c, prm);
    if (g.on) par_need = std::max(par_need, g.bytes);
  }
  if (rc == MPLD_OK && par_need) rc = ensure_par_buf(p, par_need);
  for (int c = 0; c < p->n_comp && rc == MPLD_OK; ++c) {
    const GridSplit g = grid_split_of(p, c, prm);
    if (g.on) {
      rc = launch_grid_split(p, c, g, prm, st);
      continue;
    }
    mpld::LaunchArgs a;
    a.desc = p->d_desc + c;
    a.order = nullptr;
    a.n_inst = 1;
    const int fp = (int)mpld::align16(p->footprint[c]);
    const bool large = p->h_desc[c].n >= cta_min_of(prm);   // searched by a whole CTA
    // a whole CTA keeps the state in global memory, unless its warps split
    // the instance (each then needs a slot)
    const int team_slot = mpld_internal_max_slot_bytes(CTA_TEAM_WARPS);
    // ... or, not split, its column classes in the CTA's slots, with as much
    // of its state beside them as fits (warp 0 then searches it alone;
    // without room for the classes every thread of the CTA scans)
    const int bk_slot = (int)mpld::align16((mpld::bucket_bytes(p->h_desc[c].n, p->h_desc[c].k) +
                                            CTA_TEAM_WARPS - 1) / CTA_TEAM_WARPS);
    a.slot_bytes = large ? (par_of(prm) ? (fp <= team_slot ? fp : 0) : (bk_slot <= team_slot ? team_slot : 0))
                         : (fp <= maxslot ? fp : 0);
    a.queue = nullptr;
    a.err = p->d_err;
    a.budget = budget_of(prm);
    a.time_limit_ns = time_limit_ns(prm);
    a.rule = rule_of(prm);
    a.n_large = large ? 1 : 0;
    a.par = par_of(prm);
    a.split = 0;
    a.par_buf = nullptr;
    if (sp.on) {
      // this instance's first search; if it stops on its budget, its
      // subtrees in a second launch
      split_phase1(a, sp, p->d_split);
      rc = mpld::split_reset(sp, p->d_split, st);
      if (rc == MPLD_OK) rc = mpld_internal_launch(&a, 1, large ? CTA_TEAM_WARPS : 1, st);
      if (rc == MPLD_OK) rc = launch_split_phase2(a, p->d_desc, sp, p->d_split, p->d_queue, st);
      continue;
    }
    rc = mpld_internal_launch(&a, 1, large ? CTA_TEAM_WARPS : 1, st);
  }
  p->searched = rc == MPLD_OK;
  p->results_copied = false;
  return rc;
}

extern "C" int mpld_search_batch_async(mpld_problem *const *ps, int32_t n, const mpld_params *prm,
                                       void *stream) {
  if (!ps || n < 1 || !params_ok(prm)) return MPLD_E_INVALID;
  for (int i = 0; i < n; ++i) {
    if (!ps[i]) return MPLD_E_INVALID;
    if (!ps[i]->d_base) return MPLD_E_STATE;
    if (split_of(prm) && !split_ok(ps[i])) return MPLD_E_INVALID;
  }
  if (n == 1) {
    const int rc = enqueue_single(ps[0], prm, stream, false);
    ps[0]->searched = rc == MPLD_OK;
    ps[0]->results_copied = false;
    return rc;
  }
  // several problems: one launch over the concatenated instance lists
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<InstDesc> desc;
  std::vector<int32_t> sizes;
  for (int i = 0; i < n; ++i) {
    desc.insert(desc.end(), ps[i]->h_desc.begin(), ps[i]->h_desc.end());
    for (int c = 0; c < ps[i]->n_comp; ++c) sizes.push_back(ps[i]->h_desc[c].n);
  }
  const int total = (int)desc.size();
  for (int i = 0; i < total; ++i) desc[i].idx = i;
  std::vector<int32_t> order((size_t)total);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sizes[x] > sizes[y]; });
  // under the split search the largest split instances of all the layouts
  // go to the queue launch first (as for one layout); the batched launch
  // takes the rest of the order
  std::vector<int32_t> qidx;
  int qslot = 0, qctas = 0;
  if (par_of(prm)) {
    const int maxslot = mpld_internal_max_slot_bytes(CTA_TEAM_WARPS);
    std::vector<int32_t> rest;
    for (int i = 0; i < total; ++i) {
      const InstDesc &d = desc[order[i]];
      bool queued = false;
      if ((int)qidx.size() < PAR_QUEUE_MAX && d.n >= PAR_MIN_SEGMENTS && mpld::reg_fits(d.n, d.k)) {
        const int sl = (int)mpld::align16(mpld::reg_layout(d.n, d.k, 0).bytes);
        if (sl <= maxslot) {
          qidx.push_back(order[i]);
          qslot = std::max(qslot, sl);
          queued = true;
        }
      }
      if (!queued) rest.push_back(order[i]);
    }
    if (!qidx.empty()) {
      order = std::move(rest);
      qctas = std::max(1, mpld_internal_ctas_per_sm(CTA_TEAM_WARPS, qslot)) *
              std::max(1, mpld_internal_num_sms());
    }
  }
  const int nq = (int)qidx.size(), n_rest = (int)order.size();
  const int n_large = count_large(n_rest, [&](int i) { return sizes[order[i]]; }, cta_min_of(prm));
  const Shape sh = with_team(pick_shape(ps, n, prm), n_large);
  void *buf = nullptr;
  const size_t dbytes = sizeof(InstDesc) * (size_t)std::max(total, 1);
  const size_t obytes = (sizeof(int32_t) * (size_t)std::max(total, 1) + 255) & ~(size_t)255;
  const size_t o_ctx = dbytes + obytes + 256;          // after desc, order, work counters
  const size_t o_qidx = o_ctx + 64u * (size_t)nq;
  const SplitPlan sp = split_plan_of(desc.data(), total, prm);
  const size_t o_split = (o_qidx + sizeof(int32_t) * (size_t)std::max(nq, 1) + 255) & ~(size_t)255;
  const size_t bytes = o_split + (sp.on ? sp.bytes : 0);
  if (cudaMallocAsync(&buf, bytes, st) != cudaSuccess) { cudaGetLastError(); return MPLD_E_OOM; }
  uint8_t *b = (uint8_t *)buf;
  int rc = MPLD_OK;
  if (total) {
    rc |= cuda_ok(cudaMemcpyAsync(b, desc.data(), sizeof(InstDesc) * (size_t)total,
                                  cudaMemcpyHostToDevice, st));
    if (n_rest)
      rc |= cuda_ok(cudaMemcpyAsync(b + dbytes, order.data(), sizeof(int32_t) * (size_t)n_rest,
                                    cudaMemcpyHostToDevice, st));
  }
  if (nq)
    rc |= cuda_ok(cudaMemcpyAsync(b + o_qidx, qidx.data(), sizeof(int32_t) * (size_t)nq,
                                  cudaMemcpyHostToDevice, st));
  // the sources are pageable vectors local to this call: wait for the copies
  // before they go out of scope (they may be read by the GPU directly)
  rc |= cuda_ok(cudaStreamSynchronize(st));
  uint32_t *queue = (uint32_t *)(b + dbytes + obytes);
  mpld::LaunchArgs a;
  a.desc = (const InstDesc *)b;
  a.order = (const int32_t *)(b + dbytes);
  a.n_inst = n_rest;
  a.slot_bytes = sh.slot;
  a.queue = queue;
  a.err = ps[0]->d_err;
  a.budget = budget_of(prm);
  a.time_limit_ns = time_limit_ns(prm);
  a.rule = rule_of(prm);
  a.n_large = n_large;
  a.par = par_of(prm);
  a.split = 0;
  a.par_buf = nullptr;
  for (int i = 0; i < n; ++i) {
    if (i) rc |= cuda_ok(cudaMemsetAsync(ps[i]->d_err, 0, 4, st));
    rc |= cuda_ok(cudaMemsetAsync(ps[i]->d_res, 0xFF,
                                  sizeof(InstResult) * (size_t)std::max(ps[i]->n_comp, 1), st));
  }
  if (!rc && nq) {
    // the queue launch: contexts reset (no incumbent, totals 0), then split
    rc |= cuda_ok(cudaMemsetAsync(ps[0]->d_err, 0, 4, st));
    rc |= cuda_ok(cudaMemsetAsync(b + o_ctx, 0, 64u * (size_t)nq, st));
    rc |= cuda_ok(cudaMemset2DAsync(b + o_ctx, 64, 0xFF, 8, (size_t)nq, st));
    mpld::LaunchArgs qa = a;
    qa.order = (const int32_t *)(b + o_qidx);
    qa.n_inst = nq;
    qa.slot_bytes = qslot;
    qa.queue = nullptr;
    qa.budget = 0;
    qa.n_large = 0;
    qa.par = 3;
    qa.par_buf = b + o_ctx;
    if (!rc) rc = mpld_internal_launch(&qa, qctas, CTA_TEAM_WARPS, st);
    if (!rc) rc = cuda_ok(cudaMemsetAsync(queue, 0, 8, st));
    if (!rc && n_rest) {
      const int ctas = std::min(sh.ctas, n_large + (n_rest - n_large + sh.nw - 1) / sh.nw);
      rc = mpld_internal_launch(&a, std::max(ctas, 1), sh.nw, st);
    }
  } else if (!rc && sp.on) {
    // the first phase over every instance, then the subtrees of the hard ones
    split_phase1(a, sp, b + o_split);
    rc = mpld::split_reset(sp, b + o_split, st);
    if (!rc)
      rc = launch_batch(a, sh, st, queue, ps[0]->d_err,
                        mpld::split_warp_prefix(desc.data(), order.data(), n_rest, n_large));
    if (!rc) rc = launch_split_phase2(a, a.desc, sp, b + o_split, queue, st);
  } else if (!rc) {
    rc = launch_batch(a, sh, st, queue, ps[0]->d_err);
  }
  rc |= cuda_ok(cudaFreeAsync(buf, st));
  for (int i = 0; i < n; ++i) {
    ps[i]->searched = rc == MPLD_OK;
    ps[i]->results_copied = false;
  }
  return rc ? MPLD_E_CUDA : MPLD_OK;
}

extern "C" int mpld_fetch(mpld_problem *p, int8_t *mask_out, mpld_result *res, void *stream) {
  if (!p) return MPLD_E_INVALID;
  if (!p->searched) return MPLD_E_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = MPLD_OK;
  if (!p->results_copied) {
    if (p->n_comp)
      rc |= cuda_ok(cudaMemcpyAsync(p->h_res, p->d_res, sizeof(InstResult) * (size_t)p->n_comp,
                                    cudaMemcpyDeviceToHost, st));
    if (p->instance_segments)
      rc |= cuda_ok(cudaMemcpyAsync(p->h_masks, p->d_masks, (size_t)p->instance_segments,
                                    cudaMemcpyDeviceToHost, st));
    rc |= cuda_ok(cudaMemcpyAsync(p->h_err, p->d_err, 4, cudaMemcpyDeviceToHost, st));
  }
  rc |= cuda_ok(cudaStreamSynchronize(st));
  if (rc) return MPLD_E_CUDA;
  p->searched = false;
  return finish(p, mask_out, res);
}

// ================================================================= shards

// One layout over several GPUs: its instances are independent (Sec. 1, task
// parallelism), so each rank searches a share of them and the ranks'
// per-instance results are gathered before the recovery.  Shares are longest
// processing time first: instances by decreasing estimated work (segments +
// adjacency entries; ties to the lower index), each to the rank with the
// least work so far (ties to the lower rank).
extern "C" int mpld_shard_instances(const mpld_problem *p, int32_t world, int32_t *owner_out) {
  if (!p || world < 1 || (!owner_out && p->n_comp > 0)) return MPLD_E_INVALID;
  const int C = p->n_comp;
  std::vector<int64_t> w((size_t)C);
  for (int c = 0; c < C; ++c) w[c] = (int64_t)p->h_desc[c].n + p->h_desc[c].ne2 + p->h_desc[c].ns2;
  std::vector<int32_t> ord((size_t)C);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return w[x] > w[y]; });
  std::vector<int64_t> load((size_t)world, 0);
  for (int c : ord) {
    int r = 0;
    for (int q = 1; q < world; ++q)
      if (load[q] < load[r]) r = q;
    owner_out[c] = r;
    load[r] += w[c];
  }
  return MPLD_OK;
}

extern "C" int mpld_instance_sizes(const mpld_problem *p, int32_t *sizes) {
  if (!p || (!sizes && p->n_comp > 0)) return MPLD_E_INVALID;
  for (int c = 0; c < p->n_comp; ++c) sizes[c] = p->comp_ptr[c + 1] - p->comp_ptr[c];
  return MPLD_OK;
}

// The batched search of the listed instances only, in one launch (two with
// the budgeted split search), largest first; the others are not searched.
extern "C" int mpld_search_subset_async(mpld_problem *p, const mpld_params *prm,
                                        const int32_t *inst, int32_t n, void *stream) {
  if (!p || n < 0 || (n > 0 && !inst) || !params_ok(prm) || par_of(prm)) return MPLD_E_INVALID;
  if (!p->d_base) return MPLD_E_STATE;
  if (split_of(prm) && !split_ok(p)) return MPLD_E_INVALID;
  std::vector<int32_t> order(inst, inst + n);
  std::vector<uint8_t> seen((size_t)p->n_comp, 0);
  for (int32_t c : order) {
    if (c < 0 || c >= p->n_comp || seen[c]) return MPLD_E_INVALID;
    seen[c] = 1;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return p->h_desc[x].n > p->h_desc[y].n || (p->h_desc[x].n == p->h_desc[y].n && x < y);
  });
  const SplitPlan sp = split_plan_of(p->h_desc.data(), p->n_comp, prm);
  if (sp.on && ensure_split_buf(p, sp.bytes) != MPLD_OK) return MPLD_E_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  mpld_problem *ps[1] = {p};
  const int n_large = count_large(n, [&](int i) { return p->h_desc[order[i]].n; }, cta_min_of(prm));
  const Shape sh = with_team(pick_shape(ps, 1, prm), n_large);
  void *buf = nullptr;
  if (cudaMallocAsync(&buf, 4u * (size_t)std::max(n, 1), st) != cudaSuccess) {
    cudaGetLastError();
    return MPLD_E_OOM;
  }
  int rc = cuda_ok(cudaMemsetAsync(p->d_res, 0xFF, sizeof(InstResult) * (size_t)std::max(p->n_comp, 1), st));
  if (n) rc |= cuda_ok(cudaMemcpyAsync(buf, order.data(), 4u * (size_t)n, cudaMemcpyHostToDevice, st));
  // the source is a vector local to this call
  rc |= cuda_ok(cudaStreamSynchronize(st));
  mpld::LaunchArgs a;
  a.desc = p->d_desc;
  a.order = (const int32_t *)buf;
  a.n_inst = n;
  a.slot_bytes = sh.slot;
  a.queue = p->d_queue;
  a.err = p->d_err;
  a.budget = budget_of(prm);
  a.time_limit_ns = time_limit_ns(prm);
  a.rule = rule_of(prm);
  a.n_large = n_large;
  a.par = 0;
  a.split = 0;
  a.par_buf = nullptr;
  if (!rc && sp.on) {
    split_phase1(a, sp, p->d_split);
    rc = mpld::split_reset(sp, p->d_split, st);
    if (!rc)
      rc = launch_batch(a, sh, st, p->d_queue, p->d_err,
                        mpld::split_warp_prefix(p->h_desc.data(), order.data(), n, n_large));
    if (!rc) rc = launch_split_phase2(a, p->d_desc, sp, p->d_split, p->d_queue, st);
  } else if (!rc) {
    rc = launch_batch(a, sh, st, p->d_queue, p->d_err);
  }
  rc |= cuda_ok(cudaFreeAsync(buf, st));
  p->searched = rc == MPLD_OK;
  p->results_copied = false;
  return rc ? MPLD_E_CUDA : MPLD_OK;
}

// Per-instance results of the last search, copied back: nodes, cost and
// status per instance (status -1: not searched), and the instances' masks,
// instance after instance, each in ascending segment id.
extern "C" int mpld_fetch_instances(mpld_problem *p, int64_t *nodes, int64_t *cost,
                                    int32_t *status, int8_t *inst_masks, void *stream) {
  if (!p) return MPLD_E_INVALID;
  if (!p->searched) return MPLD_E_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = MPLD_OK;
  if (!p->results_copied) {
    if (p->n_comp)
      rc |= cuda_ok(cudaMemcpyAsync(p->h_res, p->d_res, sizeof(InstResult) * (size_t)p->n_comp,
                                    cudaMemcpyDeviceToHost, st));
    if (p->instance_segments)
      rc |= cuda_ok(cudaMemcpyAsync(p->h_masks, p->d_masks, (size_t)p->instance_segments,
                                    cudaMemcpyDeviceToHost, st));
    rc |= cuda_ok(cudaMemcpyAsync(p->h_err, p->d_err, 4, cudaMemcpyDeviceToHost, st));
  }
  rc |= cuda_ok(cudaStreamSynchronize(st));
  if (rc) return MPLD_E_CUDA;
  if (*p->h_err) return *p->h_err < 0 ? *p->h_err : MPLD_E_STATE;
  p->results_copied = true;
  for (int c = 0; c < p->n_comp; ++c) {
    if (nodes) nodes[c] = p->h_res[c].nodes;
    if (cost) cost[c] = p->h_res[c].cost;
    if (status) status[c] = p->h_res[c].status;
  }
  if (inst_masks && p->instance_segments) std::memcpy(inst_masks, p->h_masks, (size_t)p->instance_segments);
  return MPLD_OK;
}

// Scatter per-instance results given by the caller (for instance gathered
// from the ranks that searched them), recover the removed segments and count
// (as mpld_fetch does after a search on this handle).  Works on host-only
// handles too.
extern "C" int mpld_finish_from(mpld_problem *p, const int64_t *nodes, const int64_t *cost,
                                const int32_t *status, const int8_t *inst_masks, int8_t *mask_out,
                                mpld_result *res) {
  if (!p || (p->n_comp > 0 && (!nodes || !cost || !status)) ||
      (p->instance_segments > 0 && !inst_masks))
    return MPLD_E_INVALID;
  std::vector<InstResult> r((size_t)std::max(p->n_comp, 1));
  for (int c = 0; c < p->n_comp; ++c) {
    r[c].cost = cost[c];
    r[c].nodes = nodes[c];
    r[c].status = status[c];
    r[c].sub = 0;
    r[c].work = 0;
  }
  return mpld_internal_finish(p, r.data(), inst_masks, 0, mask_out, res);
}

extern "C" int mpld_solve(mpld_problem *p, const mpld_params *prm, int8_t *mask_out,
                          mpld_result *res, void *stream) {
  const int rc = mpld_search_plain_async(p, prm, stream);
  if (rc < 0) return rc;
  return mpld_fetch(p, mask_out, res, stream);
}

extern "C" int mpld_solve_batch(mpld_problem *const *ps, int32_t n, const mpld_params *prm,
                                int8_t *const *masks_out, mpld_result *results, void *stream) {
  if (!ps || n < 1) return MPLD_E_INVALID;
  int rc;
  if (n == 1) {
    if (!ps[0]) return MPLD_E_INVALID;
    if (!ps[0]->d_base) return MPLD_E_STATE;
    rc = enqueue_single(ps[0], prm, stream, true);
    if (rc) return rc;
    ps[0]->searched = true;
    ps[0]->results_copied = true;
  } else {
    rc = mpld_search_batch_async(ps, n, prm, stream);
    if (rc) return rc;
  }
  int worst = MPLD_OK;
  for (int i = 0; i < n; ++i) {
    const int r = mpld_fetch(ps[i], masks_out ? masks_out[i] : nullptr,
                             results ? &results[i] : nullptr, stream);
    if (r < 0) return r;
    worst = std::max(worst, r);
  }
  return worst;
}

extern "C" const char *mpld_status_string(int code) {
  switch (code) {
    case MPLD_OK: return "ok";
    case MPLD_BUDGET: return "node budget or time limit reached; best assignment returned";
    case MPLD_TIMEOUT: return "time limit reached; best assignment returned";
    case MPLD_E_INVALID: return "invalid input";
    case MPLD_E_OOM: return "out of memory";
    case MPLD_E_CUDA: return "CUDA error";
    case MPLD_E_TIMEOUT: return "device-side wait timed out";
    case MPLD_E_TOO_LARGE: return "search instance too large";
    case MPLD_E_STATE: return "call out of order or inconsistent state";
    default: return "unknown status";
  }
}

extern "C" int mpld_problem_info(const mpld_problem *p, mpld_info *info) {
  if (!p || !info) return MPLD_E_INVALID;
  info->n_seg = p->n_seg;
  info->k = p->k;
  info->n_components = p->n_comp;
  info->max_component = p->max_component;
  info->n_removed_segments = p->n_removed_segments;
  info->arena_bytes = (int64_t)p->arena_bytes;
  info->state_bytes = (int64_t)p->scratch_bytes;
  info->instance_segments = p->instance_segments;
  return MPLD_OK;
}

extern "C" int mpld_component_results(const mpld_problem *p, int64_t *nodes, int64_t *cost,
                                      int32_t *status, int32_t *comp_of) {
  if (!p) return MPLD_E_INVALID;
  if (comp_of && p->n_seg) std::memcpy(comp_of, p->comp_of.data(), sizeof(int32_t) * (size_t)p->n_seg);
  if (!nodes && !cost && !status) return MPLD_OK;
  if (!p->have_results) return MPLD_E_STATE;
  const size_t C = (size_t)p->n_comp;
  if (nodes && C) std::memcpy(nodes, p->r_nodes.data(), sizeof(int64_t) * C);
  if (cost && C) std::memcpy(cost, p->r_cost.data(), sizeof(int64_t) * C);
  if (status && C) std::memcpy(status, p->r_status.data(), sizeof(int32_t) * C);
  return MPLD_OK;
}

extern "C" int mpld_export_matrix(const mpld_problem *p, int32_t comp, uint8_t *dense,
                                  int32_t *dims) {
  if (!p || comp < 0 || comp >= p->n_comp) return MPLD_E_INVALID;
  const InstDesc &d = p->h_desc[comp];
  const int n = d.n, k = p->k, ne = d.ne2 / 2;
  if (dims) { dims[0] = n; dims[1] = k; dims[2] = ne; }
  if (!dense) return MPLD_OK;
  // decode the packed read-only block as stored in the arena
  const mpld::RoLayout R = mpld::ro_layout(n, d.ne2, d.ns2);
  const uint8_t *blk = p->h_arena.data() + p->ro_off[comp];
  const int32_t *ptr = (const int32_t *)(blk + R.ptr);
  std::vector<int32_t> cptr((size_t)n + 1);
  for (int v = 0; v <= n; ++v) cptr[v] = ptr[2 * v];
  const uint16_t *cn = (const uint16_t *)(blk + R.cnbr);
  const size_t ncol = (size_t)(1 + n + k * ne);
  std::memset(dense, 0, (size_t)n * (size_t)k * ncol);
  // conflict edges numbered in ascending (min, max) local id
  std::vector<int32_t> eid((size_t)std::max(d.ne2, 1), -1);
  int e = 0;
  for (int v = 0; v < n; ++v)
    for (int i = cptr[v]; i < cptr[v + 1]; ++i)
      if (cn[i] > v) eid[i] = e++;
  for (int v = 0; v < n; ++v)
    for (int i = cptr[v]; i < cptr[v + 1]; ++i)
      if (cn[i] < v) {
        const int u = cn[i];
        for (int j = cptr[u]; j < cptr[u + 1]; ++j)
          if (cn[j] == v) { eid[i] = eid[j]; break; }
      }
  for (int v = 0; v < n; ++v)
    for (int c = 0; c < k; ++c) {
      uint8_t *row = dense + ((size_t)v * k + c) * ncol;
      row[1 + v] = 1;
      for (int i = cptr[v]; i < cptr[v + 1]; ++i) row[1 + n + (size_t)eid[i] * k + c] = 1;
    }
  return MPLD_OK;
}

extern "C" int mpld_autotune(mpld_problem *const *ps, int32_t n, const mpld_params *prm,
                             void *stream, mpld_tune *best_out) {
  if (!ps || n < 1 || !params_ok(prm)) return MPLD_E_INVALID;
  for (int i = 0; i < n; ++i) {
    if (!ps[i]) return MPLD_E_INVALID;
    if (!ps[i]->d_base) return MPLD_E_STATE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // candidate shapes: warps per CTA x slot size (fit-all, or the 90th
  // percentile footprint so that the largest instances spill)
  std::vector<uint32_t> fp;
  for (int i = 0; i < n; ++i) fp.insert(fp.end(), ps[i]->footprint.begin(), ps[i]->footprint.end());
  if (fp.empty()) return MPLD_OK;
  std::sort(fp.begin(), fp.end());
  const uint32_t fmax = fp.back(), f90 = fp[(fp.size() * 9) / 10];
  const int nws[] = {1, 2, 4, 8, 16};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MPLD_E_CUDA;
  mpld_tune best{};
  best.ms = 1e30f;
  int rc = MPLD_OK;
  for (int nw : nws) {
    const int maxslot = mpld_internal_max_slot_bytes(nw);
    std::vector<int> slots = {(int)mpld::align16(fmax), (int)mpld::align16(f90)};
    for (size_t si = 0; si < slots.size(); ++si) {
      int slot = std::min(std::max(slots[si], 16), maxslot) & ~15;
      if (si == 1 && slot == (std::min(std::max(slots[0], 16), maxslot) & ~15)) continue;
      mpld_params q = prm ? *prm : mpld_params{};
      q.warps_per_cta = nw;
      q.slot_bytes = slot;
      rc = mpld_search_batch_async(ps, n, &q, stream);  // warm-up (captures the graph)
      if (rc) break;
      cudaEventRecord(e0, st);
      rc = mpld_search_batch_async(ps, n, &q, stream);
      cudaEventRecord(e1, st);
      if (rc) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = MPLD_E_CUDA; break; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      int spilled = 0;
      for (uint32_t f : fp) spilled += (int)mpld::align16(f) > slot;
      if (ms < best.ms) {
        best.ms = ms;
        best.warps_per_cta = nw;
        best.slot_bytes = slot;
        best.ctas_per_sm = mpld_internal_ctas_per_sm(nw, slot);
        best.n_instances_spilled = spilled;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < n; ++i) ps[i]->searched = false;
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[tune_key(ps, n, prm)] = best;
  }
  if (best_out) *best_out = best;
  return MPLD_OK;
}
