// mpld_serve.cpp -- serving loop of libmpld: continuous batching of whole
// layouts on one GPU.
//
// Request life: submit (copy) -> a worker builds it host-side (simplify,
// split, pack, as mpld_build_matrix) -> poll admits built layouts in
// submission order (one still being built holds none back; one waiting for
// device memory holds back those after it) when their device bytes fit the
// arena and fewer than max_in_flight layouts are on the device -> on one of the server's streams: upload, one
// persistent launch of the batched search kernel over its instances, copy of
// the results into pinned memory, an event -> poll sees the event, returns
// the device bytes (admitting waiting layouts) -> a worker recovers the
// removed segments and counts (Sec. 2.2) -> mpld_server_result hands the
// masks out.  Launches of layouts admitted at different times run side by
// side on the device; each is the same kernel and search as
// mpld_solve_batch, so results do not depend on the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mpld.h"
#include "mpld_internal.h"
#include "mpld_problem.h"

using mpld::InstDesc;
using mpld::InstResult;

namespace {

constexpr uint64_t ALIGN = 256;

uint64_t round_up(uint64_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

// First-fit allocator over [0, size), 256-byte granules, with coalescing.
class FirstFit {
 public:
  void reset(uint64_t size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
    used_ = 0;
  }
  bool alloc(uint64_t bytes, uint64_t *off) {
    bytes = round_up(std::max<uint64_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const uint64_t start = it->first + bytes, rem = it->second - bytes;
      free_.erase(it);
      if (rem) free_[start] = rem;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = round_up(std::max<uint64_t>(bytes, 1));
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t size() const { return size_; }
  uint64_t used() const { return used_; }

 private:
  std::map<uint64_t, uint64_t> free_;
  uint64_t size_ = 0, used_ = 0;
};

enum class State { Building, Built, Admitted, Finishing, Done };

// Byte layout of one admitted layout in the device arena and in the pinned
// result pool (256-byte aligned sections).
struct Sections {
  uint64_t ro, state, desc, order, res, masks, ctrl, split, total;   // device
  uint64_t h_res, h_masks, h_err, h_total;                           // pinned
};

// general-state regions of the budgeted split search, per layout
constexpr size_t SPLIT_GEN_BYTES = (size_t)64 << 20;

Sections sections_of(const mpld_problem *p, const mpld::SplitPlan &sp) {
  const uint64_t C = (uint64_t)std::max(p->n_comp, 1);
  const uint64_t segs = (uint64_t)std::max<int64_t>(p->instance_segments, 1);
  Sections S;
  uint64_t o = 0;
  S.ro = o; o += round_up(std::max<uint64_t>(p->arena_bytes, 16));
  S.state = o; o += round_up(std::max<uint64_t>(p->scratch_bytes, 16));
  S.desc = o; o += round_up(sizeof(InstDesc) * C);
  S.order = o; o += round_up(sizeof(int32_t) * C);
  S.res = o; o += round_up(sizeof(InstResult) * C);
  S.masks = o; o += round_up(segs);
  S.ctrl = o; o += ALIGN;   // work counters at 0, status word at 16
  S.split = o; o += sp.on ? round_up(sp.bytes) : 0;   // budgeted split search block
  S.total = o;
  o = 0;
  S.h_res = o; o += round_up(sizeof(InstResult) * C);
  S.h_masks = o; o += round_up(segs);
  S.h_err = o; o += ALIGN;
  S.h_total = o;
  return S;
}

struct Req {
  int64_t ticket = 0;
  State state = State::Building;
  std::vector<int32_t> cu, cv, su, sv, poly;
  mpld_graph g{};
  uint32_t flags = 0;
  mpld_problem *p = nullptr;
  int n_seg = 0;
  // admission
  Sections sec{};
  mpld::SplitPlan split{};      // the budgeted split search's block and second launch
  uint64_t arena_off = 0, pool_off = 0;
  std::vector<InstDesc> desc;   // upload source, alive until the layout is finished
  cudaEvent_t done = nullptr;
  // outcome
  std::vector<int8_t> mask;
  mpld_result res{};
  int rc = MPLD_OK;
};

using ReqPtr = std::shared_ptr<Req>;

int cuda_ok(cudaError_t e) {
  if (e == cudaSuccess) return MPLD_OK;
  cudaGetLastError();
  return MPLD_E_CUDA;
}

}  // namespace

struct mpld_server {
  mpld_server_config cfg{};
  int64_t budget = 0, tl_ns = 0;
  int rule = 0;
  mpld_params search{};   // flags: the column rule and the budgeted split search
  int cta_min = 4096;   // instances this large get a whole CTA
  int nsm = 1, max_slot = 0;
  std::vector<cudaStream_t> streams;
  uint64_t next_stream = 0;
  uint8_t *d_arena = nullptr;
  uint8_t *h_pool = nullptr;   // pinned
  FirstFit arena, pool;
  // requests
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ReqPtr> build_q, finish_q;
  std::map<int64_t, ReqPtr> reqs;
  std::deque<int64_t> admit_order;
  std::vector<ReqPtr> inflight;
  std::deque<int64_t> done_tickets;
  std::vector<std::thread> workers;
  bool stopping = false;
  int64_t next_ticket = 1;
  mpld_server_stats st{};
};

namespace {

void worker_loop(mpld_server *s) {
  for (;;) {
    ReqPtr r;
    bool finish = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stopping || !s->build_q.empty() || !s->finish_q.empty(); });
      if (s->stopping) return;
      if (!s->finish_q.empty()) {
        r = s->finish_q.front();
        s->finish_q.pop_front();
        finish = true;
      } else {
        r = s->build_q.front();
        s->build_q.pop_front();
      }
    }
    if (!finish) {
      mpld_params prm{};
      prm.flags = r->flags | MPLD_HOST_ONLY;
      mpld_problem *p = nullptr;
      const int rc = mpld_build_matrix(&r->g, &prm, nullptr, &p);
      std::lock_guard<std::mutex> lk(s->mu);
      r->cu = {};
      r->cv = {};
      r->su = {};
      r->sv = {};
      r->poly = {};
      if (rc != MPLD_OK) {
        r->rc = rc;
        r->state = State::Done;
        s->done_tickets.push_back(r->ticket);
        s->st.failed++;
      } else {
        r->p = p;
        r->state = State::Built;
        s->st.built++;
      }
    } else {
      r->mask.assign((size_t)std::max(r->n_seg, 1), (int8_t)-1);
      const uint8_t *hp = s->h_pool + r->pool_off;
      const int32_t err = *reinterpret_cast<const int32_t *>(hp + r->sec.h_err);
      const int rc = mpld_internal_finish(r->p, reinterpret_cast<const InstResult *>(hp + r->sec.h_res),
                                          reinterpret_cast<const int8_t *>(hp + r->sec.h_masks), err,
                                          r->mask.data(), &r->res);
      std::lock_guard<std::mutex> lk(s->mu);
      s->pool.release(r->pool_off, r->sec.h_total);
      mpld_free(r->p);
      r->p = nullptr;
      r->desc = {};
      r->rc = rc;
      r->state = State::Done;
      s->done_tickets.push_back(r->ticket);
      s->st.completed++;
    }
  }
}

// Upload one admitted layout and enqueue its search on the next stream:
// upload, reset, one persistent launch of the batched kernel, copy back,
// event.  Every host source stays alive until the layout is finished.
int launch_request(mpld_server *s, Req &r) {
  mpld_problem *p = r.p;
  const int C = p->n_comp;
  const Sections &S = r.sec;
  uint8_t *base = s->d_arena + r.arena_off;
  uint8_t *hp = s->h_pool + r.pool_off;
  cudaStream_t st = s->streams[s->next_stream++ % s->streams.size()];
  InstDesc *d_desc = reinterpret_cast<InstDesc *>(base + S.desc);
  InstResult *d_res = reinterpret_cast<InstResult *>(base + S.res);
  int8_t *d_masks = reinterpret_cast<int8_t *>(base + S.masks);
  uint32_t *d_queue = reinterpret_cast<uint32_t *>(base + S.ctrl);
  int32_t *d_err = reinterpret_cast<int32_t *>(base + S.ctrl + 16);
  std::vector<uint64_t> state_off((size_t)C);
  uint64_t so = 0;
  uint32_t fmax = 16;
  for (int c = 0; c < C; ++c) {
    state_off[c] = so;
    so += (uint64_t)p->h_desc[c].state_bytes;
    fmax = std::max(fmax, p->footprint[c]);
  }
  r.desc.resize((size_t)C);
  for (int c = 0; c < C; ++c) {
    InstDesc d = p->h_desc[c];
    d.ro = base + S.ro + p->ro_off[c];
    d.scratch = base + S.state + state_off[c];
    d.mask = d_masks + p->comp_ptr[c];
    d.res = d_res + c;
    r.desc[c] = d;
  }
  int rc = MPLD_OK;
  if (p->arena_bytes)
    rc |= cuda_ok(cudaMemcpyAsync(base + S.ro, p->h_arena.data(), p->arena_bytes,
                                  cudaMemcpyHostToDevice, st));
  rc |= cuda_ok(cudaMemcpyAsync(d_desc, r.desc.data(), sizeof(InstDesc) * (size_t)C,
                                cudaMemcpyHostToDevice, st));
  rc |= cuda_ok(cudaMemcpyAsync(base + S.order, p->h_order.data(), sizeof(int32_t) * (size_t)C,
                                cudaMemcpyHostToDevice, st));
  rc |= cuda_ok(cudaMemsetAsync(base + S.ctrl, 0, ALIGN, st));
  rc |= cuda_ok(cudaMemsetAsync(d_res, 0xFF, sizeof(InstResult) * (size_t)C, st));
  if (rc) return MPLD_E_CUDA;
  // instances of at least cta_min segments (the first of the largest-first
  // order) are searched by whole CTAs of at least 8 warps
  int n_large = 0;
  while (n_large < C && p->h_desc[p->h_order[n_large]].n >= s->cta_min) ++n_large;
  const int nw = n_large > 0 ? std::max(s->cfg.warps_per_cta, 8) : s->cfg.warps_per_cta;
  const int max_slot = n_large > 0 ? mpld_internal_max_slot_bytes(nw) : s->max_slot;
  const int slot = (int)std::min<uint32_t>(mpld::align16(fmax), (uint32_t)max_slot) & ~15;
  const int per_sm = std::max(1, mpld_internal_ctas_per_sm(nw, slot));
  const int ctas = std::max(1, std::min(s->nsm * per_sm, n_large + (C - n_large + nw - 1) / nw));
  mpld::LaunchArgs a;
  a.desc = d_desc;
  a.order = reinterpret_cast<const int32_t *>(base + S.order);
  a.n_inst = C;
  a.slot_bytes = slot;
  a.queue = d_queue;
  a.err = d_err;
  a.budget = s->budget;
  a.time_limit_ns = s->tl_ns;
  a.rule = s->rule;
  a.n_large = n_large;
  a.par = 0;
  a.split = 0;
  a.par_buf = nullptr;
  if (r.split.on) {
    // budgeted split search: every instance with its share of the budget,
    // then the subtrees of the ones that stop on it
    uint8_t *sb = base + S.split;
    mpld::split_phase1_args(a, r.split, sb);
    rc = mpld::split_reset(r.split, sb, st);
    if (!rc)
      rc = mpld::split_phase1_launch(
          a, ctas, nw, mpld::split_warp_prefix(p->h_desc.data(), p->h_order.data(), C, n_large), st);
    if (!rc) rc = mpld::split_phase2_launch(a, d_desc, r.split, sb, d_queue, st);
    s->st.kernel_launches++;
  } else {
    rc = mpld_internal_launch(&a, ctas, nw, st);
  }
  if (rc) return rc;
  rc |= cuda_ok(cudaMemcpyAsync(hp + S.h_res, d_res, sizeof(InstResult) * (size_t)C,
                                cudaMemcpyDeviceToHost, st));
  if (p->instance_segments)
    rc |= cuda_ok(cudaMemcpyAsync(hp + S.h_masks, d_masks, (size_t)p->instance_segments,
                                  cudaMemcpyDeviceToHost, st));
  rc |= cuda_ok(cudaMemcpyAsync(hp + S.h_err, d_err, 4, cudaMemcpyDeviceToHost, st));
  if (cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return MPLD_E_CUDA;
  }
  rc |= cuda_ok(cudaEventRecord(r.done, st));
  s->st.kernel_launches++;
  s->st.instances_launched += C;
  return rc ? MPLD_E_CUDA : MPLD_OK;
}

}  // namespace

extern "C" int mpld_server_create(const mpld_server_config *cfg_in, const mpld_params *search,
                                  mpld_server **out) {
  if (!out) return MPLD_E_INVALID;
  *out = nullptr;
  mpld_server_config cfg = cfg_in ? *cfg_in : mpld_server_config{};
  if (cfg.arena_bytes < 0 || cfg.result_pool_bytes < 0 || cfg.max_in_flight < 0 ||
      cfg.streams < 0 || cfg.warps_per_cta < 0 || cfg.warps_per_cta > 16 ||
      cfg.worker_threads < 0)
    return MPLD_E_INVALID;
  if (!cfg.arena_bytes) cfg.arena_bytes = (int64_t)1 << 30;
  if (!cfg.result_pool_bytes) cfg.result_pool_bytes = (int64_t)256 << 20;
  if (!cfg.max_in_flight) cfg.max_in_flight = 64;
  if (!cfg.streams) cfg.streams = 8;
  if (!cfg.warps_per_cta) cfg.warps_per_cta = 4;
  // three quarters of the hardware threads: under load every worker builds
  // one layout on its own thread, and the host pool's loops take the rest
  if (!cfg.worker_threads)
    cfg.worker_threads = (int32_t)std::max(1u, 3u * std::thread::hardware_concurrency() / 4);

  mpld_server *s = new (std::nothrow) mpld_server();
  if (!s) return MPLD_E_OOM;
  s->cfg = cfg;
  s->budget = search ? std::max<int64_t>(search->node_budget, 0) : 0;
  s->tl_ns = ((search && search->time_limit_ms > 0) ? search->time_limit_ms : 60000) * 1000000ll;
  s->rule = (search && (search->flags & MPLD_COLUMN_BFS)) ? 1 : 0;
  if (search) {
    s->search = *search;
    s->search.flags &= MPLD_COLUMN_BFS | MPLD_SPLIT_BUDGET;
  }
  if (search && search->cta_segments != 0)
    s->cta_min = search->cta_segments > 0 ? search->cta_segments : INT32_MAX;
  s->nsm = std::max(1, mpld_internal_num_sms());
  s->max_slot = mpld_internal_max_slot_bytes(cfg.warps_per_cta);
  if (s->max_slot <= 0) {
    delete s;
    return MPLD_E_CUDA;
  }
  for (int i = 0; i < cfg.streams; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      mpld_server_destroy(s);
      return MPLD_E_CUDA;
    }
    s->streams.push_back(st);
  }
  if (cudaMalloc((void **)&s->d_arena, (size_t)cfg.arena_bytes) != cudaSuccess ||
      cudaMallocHost((void **)&s->h_pool, (size_t)cfg.result_pool_bytes) != cudaSuccess) {
    cudaGetLastError();
    mpld_server_destroy(s);
    return MPLD_E_OOM;
  }
  s->arena.reset((uint64_t)cfg.arena_bytes);
  s->pool.reset((uint64_t)cfg.result_pool_bytes);
  for (int i = 0; i < cfg.worker_threads; ++i) s->workers.emplace_back(worker_loop, s);
  *out = s;
  return MPLD_OK;
}

extern "C" int mpld_server_submit(mpld_server *s, const mpld_graph *g, uint32_t flags,
                                  int64_t *ticket) {
  if (!s || !g || !ticket) return MPLD_E_INVALID;
  // the budgeted split search has no clique bound
  if ((s->search.flags & MPLD_SPLIT_BUDGET) && (flags & MPLD_CLIQUE_BOUND)) return MPLD_E_INVALID;
  auto r = std::make_shared<Req>();
  const int n = std::max(g->n_seg, 0);
  try {
    if (g->n_conf > 0 && g->conf_u && g->conf_v) {
      r->cu.assign(g->conf_u, g->conf_u + g->n_conf);
      r->cv.assign(g->conf_v, g->conf_v + g->n_conf);
    }
    if (g->n_stitch > 0 && g->st_u && g->st_v) {
      r->su.assign(g->st_u, g->st_u + g->n_stitch);
      r->sv.assign(g->st_v, g->st_v + g->n_stitch);
    }
    if (g->polygon_of) r->poly.assign(g->polygon_of, g->polygon_of + n);
  } catch (const std::bad_alloc &) {
    return MPLD_E_OOM;
  }
  r->g = *g;
  r->g.conf_u = r->cu.empty() ? nullptr : r->cu.data();
  r->g.conf_v = r->cv.empty() ? nullptr : r->cv.data();
  r->g.st_u = r->su.empty() ? nullptr : r->su.data();
  r->g.st_v = r->sv.empty() ? nullptr : r->sv.data();
  r->g.polygon_of = r->poly.empty() ? nullptr : r->poly.data();
  r->flags = flags & (MPLD_NO_SIMPLIFY | MPLD_SINGLE_INSTANCE | MPLD_BICONNECTED | MPLD_CLIQUE_BOUND |
                      MPLD_DENSITY_BALANCE);
  r->n_seg = n;
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  *ticket = r->ticket;
  s->reqs[r->ticket] = r;
  s->admit_order.push_back(r->ticket);
  s->build_q.push_back(r);
  s->st.submitted++;
  s->cv.notify_one();
  return MPLD_OK;
}

extern "C" int mpld_server_poll(mpld_server *s, int64_t *done, int32_t max_done,
                                int32_t *n_done) {
  if (!s || (max_done > 0 && !done)) return MPLD_E_INVALID;
  // finished layouts: their stream passed the copy-back
  for (size_t i = 0; i < s->inflight.size();) {
    ReqPtr r = s->inflight[i];
    const cudaError_t q = cudaEventQuery(r->done);
    if (q == cudaErrorNotReady) {
      cudaGetLastError();
      ++i;
      continue;
    }
    if (q != cudaSuccess) return cuda_ok(q);
    cudaEventDestroy(r->done);
    r->done = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    s->arena.release(r->arena_off, r->sec.total);
    r->state = State::Finishing;
    s->finish_q.push_back(r);
    s->cv.notify_one();
    s->inflight[i] = s->inflight.back();
    s->inflight.pop_back();
  }
  // admission of built layouts in submission order: one still being built
  // does not hold back the built ones behind it, while one that waits for
  // device memory does (so that a large layout is never passed over)
  for (;;) {
    ReqPtr r;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      size_t pos = 0;
      while (pos < s->admit_order.size()) {
        auto it = s->reqs.find(s->admit_order[pos]);
        if (it == s->reqs.end() || it->second->state == State::Done) {
          s->admit_order.erase(s->admit_order.begin() + (ptrdiff_t)pos);  // failed while building
          continue;
        }
        if (it->second->state == State::Built) {
          r = it->second;
          break;
        }
        ++pos;   // still being built
      }
      if (!r) break;
      if ((int)s->inflight.size() >= s->cfg.max_in_flight) break;
      mpld_problem *p = r->p;
      r->split = mpld::split_plan(p->h_desc.data(), p->n_comp, &s->search, SPLIT_GEN_BYTES);
      r->sec = sections_of(p, r->split);
      if (r->sec.total > s->arena.size() || r->sec.h_total > s->pool.size()) {
        // can never fit: fail the ticket
        mpld_free(p);
        r->p = nullptr;
        r->rc = MPLD_E_TOO_LARGE;
        r->state = State::Done;
        s->done_tickets.push_back(r->ticket);
        s->st.failed++;
        s->admit_order.erase(s->admit_order.begin() + (ptrdiff_t)pos);
        continue;
      }
      if (!s->arena.alloc(r->sec.total, &r->arena_off)) break;
      if (!s->pool.alloc(r->sec.h_total, &r->pool_off)) {
        s->arena.release(r->arena_off, r->sec.total);
        break;
      }
      s->admit_order.erase(s->admit_order.begin() + (ptrdiff_t)pos);
      s->st.arena_used_bytes = (int64_t)s->arena.used();
      s->st.arena_peak_bytes = std::max(s->st.arena_peak_bytes, s->st.arena_used_bytes);
      s->st.admitted++;
    }
    if (r->p->n_comp == 0) {
      // nothing to search: recover straight away
      std::memset(s->h_pool + r->pool_off, 0, r->sec.h_total);
      std::lock_guard<std::mutex> lk(s->mu);
      s->arena.release(r->arena_off, r->sec.total);
      r->state = State::Finishing;
      s->finish_q.push_back(r);
      s->cv.notify_one();
      continue;
    }
    const int rc = launch_request(s, *r);
    if (rc) return rc;
    r->state = State::Admitted;
    s->inflight.push_back(r);
    s->st.max_concurrent = std::max(s->st.max_concurrent, (int64_t)s->inflight.size());
  }
  int32_t nd = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    while (nd < max_done && !s->done_tickets.empty()) {
      done[nd++] = s->done_tickets.front();
      s->done_tickets.pop_front();
    }
  }
  if (n_done) *n_done = nd;
  return MPLD_OK;
}

extern "C" int mpld_server_result(mpld_server *s, int64_t ticket, int8_t *mask_out,
                                  mpld_result *result) {
  if (!s) return MPLD_E_INVALID;
  ReqPtr r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second->state != State::Done) return MPLD_E_STATE;
    r = it->second;
    s->reqs.erase(it);
  }
  if (r->rc < 0) return r->rc;
  if (mask_out && r->n_seg) std::memcpy(mask_out, r->mask.data(), (size_t)r->n_seg);
  if (result) *result = r->res;
  return r->rc;
}

extern "C" int mpld_server_stats_get(const mpld_server *s, mpld_server_stats *out) {
  if (!s || !out) return MPLD_E_INVALID;
  mpld_server *m = const_cast<mpld_server *>(s);
  std::lock_guard<std::mutex> lk(m->mu);
  *out = s->st;
  int64_t waiting = 0;
  for (const auto &kv : s->reqs)
    if (kv.second->state == State::Built) ++waiting;
  out->waiting = waiting;
  out->in_flight = (int64_t)s->inflight.size();
  out->arena_used_bytes = (int64_t)s->arena.used();
  return MPLD_OK;
}

extern "C" void mpld_server_destroy(mpld_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (auto &t : s->workers) t.join();
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  for (auto &r : s->inflight)
    if (r->done) cudaEventDestroy(r->done);
  // a request still waiting to be finished is also in the map: each
  // problem is freed once
  for (auto &kv : s->reqs)
    if (kv.second->p) {
      mpld_free(kv.second->p);
      kv.second->p = nullptr;
    }
  for (auto &r : s->finish_q)
    if (r->p) {
      mpld_free(r->p);
      r->p = nullptr;
    }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  if (s->d_arena) cudaFree(s->d_arena);
  if (s->h_pool) cudaFreeHost(s->h_pool);
  delete s;
}
