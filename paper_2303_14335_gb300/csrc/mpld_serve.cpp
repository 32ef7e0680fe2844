// mpld_serve.cpp -- serving loop of libmpld: continuous batching of whole
// layouts onto one resident search kernel.
//
// Request life: submit (copy) -> worker builds it host-side (simplify, split,
// pack, as mpld_build_matrix) -> poll admits it in submission order when its
// device bytes fit the arena and its instances fit the ring -> upload of the
// packed matrices, descriptors appended to the device ring, tail published ->
// the resident kernel searches its instances next to those of every other
// admitted request, writing results into pinned host memory and counting
// finished instances -> poll sees the count complete, frees the device bytes
// (which lets waiting requests in) -> a worker recovers removed segments and
// counts (Sec. 2.2) -> mpld_server_result hands the masks out.
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
constexpr uint32_t TAIL_VALUES = 4096;  // pinned sources of in-flight tail copies

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

struct Req {
  int64_t ticket = 0;
  State state = State::Building;
  std::vector<int32_t> cu, cv, su, sv, poly;
  mpld_graph g{};
  uint32_t flags = 0;
  mpld_problem *p = nullptr;
  int n_seg = 0;
  // admission
  uint64_t arena_off = 0, arena_bytes = 0, pool_off = 0, pool_bytes = 0;
  uint32_t *counter = nullptr;
  InstResult *hres = nullptr;
  int8_t *hmasks = nullptr;
  int C = 0;
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
  int64_t budget = 0, tl_ns = 0, idle_ns = 0;
  cudaStream_t kstream = nullptr, cstream = nullptr;
  cudaEvent_t kdone = nullptr;
  bool launched = false;
  int ctas = 1;
  // device
  uint8_t *d_arena = nullptr;
  InstDesc *d_ring = nullptr;
  uint32_t *d_ctrl = nullptr;  // [0] head, [32] tail, [64] status word
  // pinned host
  InstDesc *h_ring = nullptr;       // staging copy of the ring
  uint32_t *h_tail = nullptr;       // TAIL_VALUES tail values
  uint32_t *h_stop = nullptr;       // mapped stop flag, then the kernel's status word
  uint8_t *h_pool = nullptr;        // mapped results, masks, counters
  uint8_t *d_pool = nullptr;        // device address of h_pool
  uint32_t *d_stop = nullptr;
  FirstFit arena, pool;
  uint64_t published = 0, done_instances = 0, tail_copies = 0;
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
      r->cu.clear(); r->cu.shrink_to_fit();
      r->cv.clear(); r->cv.shrink_to_fit();
      r->su.clear(); r->su.shrink_to_fit();
      r->sv.clear(); r->sv.shrink_to_fit();
      r->poly.clear(); r->poly.shrink_to_fit();
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
      const int rc = mpld_internal_finish(r->p, r->hres, r->hmasks, 0, r->mask.data(), &r->res);
      std::lock_guard<std::mutex> lk(s->mu);
      s->pool.release(r->pool_off, r->pool_bytes);
      mpld_free(r->p);
      r->p = nullptr;
      r->rc = rc;
      r->state = State::Done;
      s->done_tickets.push_back(r->ticket);
      s->st.completed++;
    }
  }
}

// Device bytes of a built request: read-only blocks, then state regions.
uint64_t device_bytes(const mpld_problem *p) {
  return round_up(p->arena_bytes) + round_up(p->scratch_bytes);
}
uint64_t pool_bytes_of(const mpld_problem *p) {
  return 64 + sizeof(InstResult) * (uint64_t)std::max(p->n_comp, 1) +
         (uint64_t)std::max<int64_t>(p->instance_segments, 1);
}

// Upload one request and append its instances to the ring (largest first).
int admit(mpld_server *s, Req &r) {
  mpld_problem *p = r.p;
  const int C = p->n_comp;
  uint8_t *base = s->d_arena + r.arena_off;
  uint8_t *state_base = base + round_up(p->arena_bytes);
  int rc = MPLD_OK;
  if (p->arena_bytes)
    rc |= cuda_ok(cudaMemcpyAsync(base, p->h_arena.data(), p->arena_bytes, cudaMemcpyHostToDevice,
                                  s->cstream));
  uint8_t *hp = s->h_pool + r.pool_off;
  uint8_t *dp = s->d_pool + r.pool_off;
  r.counter = reinterpret_cast<uint32_t *>(hp);
  __atomic_store_n(r.counter, 0u, __ATOMIC_RELEASE);
  r.hres = reinterpret_cast<InstResult *>(hp + 64);
  r.hmasks = reinterpret_cast<int8_t *>(hp + 64 + sizeof(InstResult) * (size_t)std::max(C, 1));
  uint32_t *d_counter = reinterpret_cast<uint32_t *>(dp);
  InstResult *d_res = reinterpret_cast<InstResult *>(dp + 64);
  int8_t *d_masks = reinterpret_cast<int8_t *>(dp + 64 + sizeof(InstResult) * (size_t)std::max(C, 1));
  std::vector<uint64_t> state_off((size_t)C);
  uint64_t so = 0;
  for (int c = 0; c < C; ++c) {
    state_off[c] = so;
    so += (uint64_t)p->h_desc[c].state_bytes;
  }
  const uint32_t cap = (uint32_t)s->cfg.ring_capacity;
  const uint64_t first = s->published;
  const uint8_t *region_end = base + r.arena_bytes;
  const uint8_t *pool_end = dp + r.pool_bytes;
  for (int j = 0; j < C; ++j) {
    const int c = p->h_order[j];
    InstDesc d = p->h_desc[c];
    d.ro = base + p->ro_off[c];
    d.scratch = state_base + state_off[c];
    d.mask = d_masks + p->comp_ptr[c];
    d.res = d_res + c;
    d.done = d_counter;
    // every pointer the kernel will follow stays inside this request's regions
    if (d.ro + d.ro_bytes > state_base || d.scratch + d.state_bytes > region_end ||
        (const uint8_t *)(d.mask + d.n) > pool_end || (const uint8_t *)(d.res + 1) > pool_end ||
        ((uintptr_t)d.ro & 15) || ((uintptr_t)d.scratch & 15))
      return MPLD_E_STATE;
    s->h_ring[(first + j) % cap] = d;
  }
  // copy the new ring slots (one or two pieces), then publish the tail
  const uint32_t s0 = (uint32_t)(first % cap);
  const uint32_t n0 = std::min<uint32_t>((uint32_t)C, cap - s0);
  if (n0)
    rc |= cuda_ok(cudaMemcpyAsync(s->d_ring + s0, s->h_ring + s0, sizeof(InstDesc) * n0,
                                  cudaMemcpyHostToDevice, s->cstream));
  if ((uint32_t)C > n0)
    rc |= cuda_ok(cudaMemcpyAsync(s->d_ring, s->h_ring, sizeof(InstDesc) * ((uint32_t)C - n0),
                                  cudaMemcpyHostToDevice, s->cstream));
  s->published += (uint64_t)C;
  uint32_t *tv = s->h_tail + (s->tail_copies % TAIL_VALUES);
  *tv = (uint32_t)s->published;
  rc |= cuda_ok(cudaMemcpyAsync(s->d_ctrl + 32, tv, 4, cudaMemcpyHostToDevice, s->cstream));
  if (++s->tail_copies % (TAIL_VALUES / 2) == 0) rc |= cuda_ok(cudaStreamSynchronize(s->cstream));
  // p->h_arena stays alive until the request is finished: an asynchronous
  // copy from pageable memory may read it after this call returns (on
  // systems where the GPU reads host memory directly, nothing stages it)
  r.C = C;
  return rc ? MPLD_E_CUDA : MPLD_OK;
}

int relaunch_if_needed(mpld_server *s) {
  if (s->published == s->done_instances) return MPLD_OK;
  if (s->launched) {
    const cudaError_t q = cudaEventQuery(s->kdone);
    if (q == cudaErrorNotReady) return MPLD_OK;  // still running
    if (q != cudaSuccess) return cuda_ok(q);
  }
  mpld::ServeArgs a;
  a.ring = s->d_ring;
  a.cap = (uint32_t)s->cfg.ring_capacity;
  a.slot_bytes = s->cfg.slot_bytes;
  a.head = s->d_ctrl;
  a.tail = s->d_ctrl + 32;
  a.stop = s->d_stop;
  a.err = reinterpret_cast<int32_t *>(s->d_stop + 8);   // host-mapped (byte 32), read by every poll
  a.arena_lo = s->d_arena;
  a.arena_hi = s->d_arena + s->cfg.arena_bytes;
  a.pool_lo = s->d_pool;
  a.pool_hi = s->d_pool + s->cfg.result_pool_bytes;
  a.budget = s->budget;
  a.time_limit_ns = s->tl_ns;
  a.idle_ns = s->idle_ns;
  int rc = mpld_internal_serve_launch(&a, s->ctas, s->cfg.warps_per_cta, s->kstream);
  if (rc) return rc;
  rc = cuda_ok(cudaEventRecord(s->kdone, s->kstream));
  s->launched = true;
  s->st.kernel_launches++;
  return rc;
}

}  // namespace

extern "C" int mpld_server_create(const mpld_server_config *cfg_in, const mpld_params *search,
                                  mpld_server **out) {
  if (!out) return MPLD_E_INVALID;
  *out = nullptr;
  mpld_server_config cfg = cfg_in ? *cfg_in : mpld_server_config{};
  if (cfg.arena_bytes < 0 || cfg.result_pool_bytes < 0 || cfg.ring_capacity < 0 ||
      cfg.warps_per_cta < 0 || cfg.warps_per_cta > 16 || cfg.slot_bytes < 0 ||
      cfg.worker_threads < 0 || cfg.idle_exit_ms < 0)
    return MPLD_E_INVALID;
  if (!cfg.arena_bytes) cfg.arena_bytes = (int64_t)1 << 30;
  if (!cfg.result_pool_bytes) cfg.result_pool_bytes = (int64_t)256 << 20;
  if (!cfg.ring_capacity) cfg.ring_capacity = 1 << 18;
  if (!cfg.warps_per_cta) cfg.warps_per_cta = 4;
  if (!cfg.slot_bytes) cfg.slot_bytes = 12288;
  cfg.slot_bytes = (cfg.slot_bytes + 15) & ~15;
  if (cfg.slot_bytes > mpld_internal_max_slot_bytes(cfg.warps_per_cta))
    cfg.slot_bytes = mpld_internal_max_slot_bytes(cfg.warps_per_cta);
  if (!cfg.worker_threads)
    cfg.worker_threads = std::max(1u, std::thread::hardware_concurrency() / 2);
  if (!cfg.idle_exit_ms) cfg.idle_exit_ms = 200;

  mpld_server *s = new (std::nothrow) mpld_server();
  if (!s) return MPLD_E_OOM;
  s->cfg = cfg;
  s->budget = search ? std::max<int64_t>(search->node_budget, 0) : 0;
  s->tl_ns = ((search && search->time_limit_ms > 0) ? search->time_limit_ms : 60000) * 1000000ll;
  s->idle_ns = cfg.idle_exit_ms * 1000000ll;
  int rc = MPLD_OK;
  auto fail = [&](int code) {
    mpld_server_destroy(s);
    return code;
  };
  if (cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(MPLD_E_CUDA);
  }
  const size_t ring_bytes = sizeof(InstDesc) * (size_t)cfg.ring_capacity;
  if (cudaMalloc((void **)&s->d_arena, (size_t)cfg.arena_bytes) != cudaSuccess ||
      cudaMalloc((void **)&s->d_ring, ring_bytes) != cudaSuccess ||
      cudaMalloc((void **)&s->d_ctrl, 512) != cudaSuccess) {
    cudaGetLastError();
    return fail(MPLD_E_OOM);
  }
  if (cudaMallocHost((void **)&s->h_ring, ring_bytes) != cudaSuccess ||
      cudaMallocHost((void **)&s->h_tail, sizeof(uint32_t) * TAIL_VALUES) != cudaSuccess ||
      cudaHostAlloc((void **)&s->h_stop, 128, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc((void **)&s->h_pool, (size_t)cfg.result_pool_bytes, cudaHostAllocMapped) !=
          cudaSuccess) {
    cudaGetLastError();
    return fail(MPLD_E_OOM);
  }
  if (cudaHostGetDevicePointer((void **)&s->d_pool, s->h_pool, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void **)&s->d_stop, s->h_stop, 0) != cudaSuccess) {
    cudaGetLastError();
    return fail(MPLD_E_CUDA);
  }
  std::memset(s->h_stop, 0, 128);
  rc |= cuda_ok(cudaMemsetAsync(s->d_ctrl, 0, 512, s->cstream));
  rc |= cuda_ok(cudaStreamSynchronize(s->cstream));
  if (rc) return fail(MPLD_E_CUDA);
  s->arena.reset((uint64_t)cfg.arena_bytes);
  s->pool.reset((uint64_t)cfg.result_pool_bytes);
  // one resident CTA per SM and occupancy slot of the chosen shape
  int per_sm = 0;
  {
    const size_t smem = mpld::align16(8u * (uint32_t)cfg.warps_per_cta) +
                        (size_t)cfg.warps_per_cta * (size_t)cfg.slot_bytes;
    per_sm = std::max(1, std::min(mpld_internal_ctas_per_sm(cfg.warps_per_cta, cfg.slot_bytes),
                                  (int)((227 * 1024) / std::max<size_t>(smem, 1))));
  }
  s->ctas = std::max(1, mpld_internal_num_sms()) * per_sm;
  for (int i = 0; i < cfg.worker_threads; ++i) s->workers.emplace_back(worker_loop, s);
  *out = s;
  return MPLD_OK;
}

extern "C" int mpld_server_submit(mpld_server *s, const mpld_graph *g, uint32_t flags,
                                  int64_t *ticket) {
  if (!s || !g || !ticket) return MPLD_E_INVALID;
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
  r->flags = flags & (MPLD_NO_SIMPLIFY | MPLD_SINGLE_INSTANCE);
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
  int rc = MPLD_OK;
  // status word of the resident kernel: a descriptor it refused, or a
  // bulk copy that did not land
  if (__atomic_load_n(reinterpret_cast<int32_t *>(s->h_stop + 8), __ATOMIC_ACQUIRE) != 0)
    return MPLD_E_STATE;
  // finished requests: every instance counted by the kernel
  for (size_t i = 0; i < s->inflight.size();) {
    ReqPtr r = s->inflight[i];
    const uint32_t c = __atomic_load_n(r->counter, __ATOMIC_ACQUIRE);
    if ((int)c == r->C) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->arena.release(r->arena_off, r->arena_bytes);
      s->done_instances += (uint64_t)r->C;
      s->st.instances_done += r->C;
      r->state = State::Finishing;
      s->finish_q.push_back(r);
      s->cv.notify_one();
      s->inflight[i] = s->inflight.back();
      s->inflight.pop_back();
    } else {
      ++i;
    }
  }
  // admission in submission order
  for (;;) {
    ReqPtr r;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      while (!s->admit_order.empty()) {
        auto it = s->reqs.find(s->admit_order.front());
        if (it == s->reqs.end() || it->second->state == State::Done) {
          s->admit_order.pop_front();  // failed while building
          continue;
        }
        break;
      }
      if (s->admit_order.empty()) break;
      r = s->reqs[s->admit_order.front()];
      if (r->state != State::Built) break;
      mpld_problem *p = r->p;
      const uint64_t dbytes = device_bytes(p), pbytes = pool_bytes_of(p);
      if (dbytes > s->arena.size() || pbytes > s->pool.size() ||
          (int64_t)p->n_comp > (int64_t)s->cfg.ring_capacity) {
        // can never fit: fail the ticket
        mpld_free(p);
        r->p = nullptr;
        r->rc = MPLD_E_TOO_LARGE;
        r->state = State::Done;
        s->done_tickets.push_back(r->ticket);
        s->st.failed++;
        s->admit_order.pop_front();
        continue;
      }
      if (s->published - s->done_instances + (uint64_t)p->n_comp > (uint64_t)s->cfg.ring_capacity)
        break;
      if (!s->arena.alloc(dbytes, &r->arena_off)) break;
      if (!s->pool.alloc(pbytes, &r->pool_off)) {
        s->arena.release(r->arena_off, dbytes);
        break;
      }
      r->arena_bytes = dbytes;
      r->pool_bytes = pbytes;
      s->admit_order.pop_front();
      s->st.arena_used_bytes = (int64_t)s->arena.used();
      s->st.arena_peak_bytes = std::max(s->st.arena_peak_bytes, s->st.arena_used_bytes);
    }
    if (r->p->n_comp == 0) {
      // nothing to search: recover straight away
      r->C = 0;
      r->counter = reinterpret_cast<uint32_t *>(s->h_pool + r->pool_off);
      r->hres = reinterpret_cast<InstResult *>(s->h_pool + r->pool_off + 64);
      r->hmasks = reinterpret_cast<int8_t *>(s->h_pool + r->pool_off + 64 + sizeof(InstResult));
      std::lock_guard<std::mutex> lk(s->mu);
      s->arena.release(r->arena_off, r->arena_bytes);
      r->state = State::Finishing;
      s->st.admitted++;
      s->finish_q.push_back(r);
      s->cv.notify_one();
      continue;
    }
    rc = admit(s, *r);
    if (rc) return rc;
    r->state = State::Admitted;
    s->inflight.push_back(r);
    s->st.admitted++;
    s->st.instances_published += r->C;
  }
  rc = relaunch_if_needed(s);
  if (rc) return rc;
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
  std::lock_guard<std::mutex> lk(const_cast<mpld_server *>(s)->mu);
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
  if (s->h_stop) __atomic_store_n(s->h_stop, 1u, __ATOMIC_RELEASE);
  if (s->kstream) cudaStreamSynchronize(s->kstream);
  if (s->cstream) cudaStreamSynchronize(s->cstream);
  for (auto &kv : s->reqs)
    if (kv.second->p) mpld_free(kv.second->p);
  for (auto &r : s->finish_q)
    if (r->p) mpld_free(r->p);
  if (s->kdone) cudaEventDestroy(s->kdone);
  if (s->kstream) cudaStreamDestroy(s->kstream);
  if (s->cstream) cudaStreamDestroy(s->cstream);
  if (s->d_arena) cudaFree(s->d_arena);
  if (s->d_ring) cudaFree(s->d_ring);
  if (s->d_ctrl) cudaFree(s->d_ctrl);
  if (s->h_ring) cudaFreeHost(s->h_ring);
  if (s->h_tail) cudaFreeHost(s->h_tail);
  if (s->h_stop) cudaFreeHost(s->h_stop);
  if (s->h_pool) cudaFreeHost(s->h_pool);
  delete s;
}
