// mpld_search.cu -- the matrix-cover search (Sec. 2.3, Algorithm 1) for
// sm_103a.
//
// One warp runs one search instance (a sub-graph of the layout).  The EC
// matrix's active rows are a bitset in shared memory; the three operations
// of Algorithm 1 become word operations:
//   * column choice (Algorithm 1, "select an uncovered column"): for every
//     uncovered primary column P_v, popc(activeRows & colRows[P_v]); the
//     KP-bit fields of a word are counted at once with a SWAR popcount, and
//     the warp takes the minimum of (count, v) with __reduce_min_sync, so
//     ties go to the lowest segment index;
//   * cover of row (v, c) (Eq. 2 "Cover", Algorithm 1 "cover rw and its
//     affected rows"): activeRows &= ~colRows[j] for every column j of the
//     row, i.e. v's field and the (u, c) bit of every conflict neighbour u;
//     the cleared bits are recorded per adjacency entry;
//   * uncover (Eq. 2 "Uncover"): OR the recorded bits back, newest level
//     first, through an explicit per-level stack instead of recursion.
// Rows of the chosen column are visited in ascending (added cost, mask),
// including rows that are no longer active: those are the "conflict
// candidates" of Algorithm 1 and pay the conflict cost of Eq. 1.  A node is
// pruned when its cost plus cost_conflict times the number of uncovered
// columns with no active row reaches the incumbent.
//
// Batched form: a persistent grid whose warps pull instance indices from a
// device work counter over a largest-first order (Sec. 2.3 / Sec. 3 run one
// block per sub-graph; here the sub-graphs are the work queue).  The plain
// form launches the same kernel once per instance.
//
// Memory spaces: an instance whose state and read-only block fit the warp's
// slot runs entirely in shared memory (the SM = true instantiation, whose
// pointers all derive from the shared array, so every access is a shared
// access); a larger one keeps its state in its own global scratch region
// (SM = false).
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpld_internal.h"
#include "../../include/mpld.h"

namespace mpld {
namespace {

extern __shared__ __align__(16) uint8_t g_smem[];

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int64_t INF = INT64_MAX;
constexpr uint32_t TMA_MIN_BYTES = 1024;     // smaller blocks use vector loads
constexpr uint32_t WAIT_LIMIT = 1u << 22;    // bounded mbarrier wait

template <int KP> struct Fields;
template <> struct Fields<4> {
  static constexpr uint64_t LO = 0x1111111111111111ull;
  static constexpr uint64_t HI = 0x8888888888888888ull;
  static constexpr uint64_t FILL = 0x7777777777777777ull;  // > any count for k <= 4
  static constexpr uint64_t FM = 0xFull;
  static constexpr int PER_WORD = 16;
};
template <> struct Fields<8> {
  static constexpr uint64_t LO = 0x0101010101010101ull;
  static constexpr uint64_t HI = 0x8080808080808080ull;
  static constexpr uint64_t FILL = 0x0F0F0F0F0F0F0F0Full;  // 15 > any count for k <= 8
  static constexpr uint64_t FM = 0xFFull;
  static constexpr int PER_WORD = 8;
};

// Number of set bits in every KP-bit field of a (SWAR popcount).
template <int KP>
__device__ __forceinline__ uint64_t field_counts(uint64_t a) {
  a = a - ((a >> 1) & 0x5555555555555555ull);
  a = (a & 0x3333333333333333ull) + ((a >> 2) & 0x3333333333333333ull);
  if (KP == 8) a = (a + (a >> 4)) & 0x0F0F0F0F0F0F0F0Full;
  return a;
}

// Fields whose value is <= t (top bit of each selected field set).  Field
// values are < 2^(KP-1), so OR-ing the top bit and subtracting t+1 never
// borrows across fields.
template <int KP>
__device__ __forceinline__ uint64_t fields_le(uint64_t key, uint32_t t) {
  using F = Fields<KP>;
  return ~((key | F::HI) - (uint64_t)(t + 1) * F::LO) & F::HI;
}

__device__ __forceinline__ void cas_u32(uint32_t &a, uint32_t &b) {
  const uint32_t lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// Sort keys ((inc << 3) | mask) ascending with a fixed network.
template <int KP> __device__ __forceinline__ void sort_keys(uint32_t (&k)[KP]);
template <> __device__ __forceinline__ void sort_keys<4>(uint32_t (&k)[4]) {
  cas_u32(k[0], k[1]); cas_u32(k[2], k[3]); cas_u32(k[0], k[2]); cas_u32(k[1], k[3]);
  cas_u32(k[1], k[2]);
}
template <> __device__ __forceinline__ void sort_keys<8>(uint32_t (&k)[8]) {
  cas_u32(k[0], k[2]); cas_u32(k[1], k[3]); cas_u32(k[4], k[6]); cas_u32(k[5], k[7]);
  cas_u32(k[0], k[4]); cas_u32(k[1], k[5]); cas_u32(k[2], k[6]); cas_u32(k[3], k[7]);
  cas_u32(k[0], k[1]); cas_u32(k[2], k[3]); cas_u32(k[4], k[5]); cas_u32(k[6], k[7]);
  cas_u32(k[2], k[4]); cas_u32(k[3], k[5]); cas_u32(k[1], k[4]); cas_u32(k[3], k[6]);
  cas_u32(k[1], k[2]); cas_u32(k[3], k[4]); cas_u32(k[5], k[6]);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- shared-memory bulk copy (TMA, non-tensor) ---------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// ---- the search ----------------------------------------------------------

struct State {
  uint64_t *active, *unas;
  int64_t *lv_g;
  int32_t *lv_inc;
  uint32_t *lv_ord;
  int32_t *lv_v;
  uint8_t *lv_next;
  int8_t *x;
  uint8_t *oldnib;
  uint8_t *clrb;
  const int32_t *cptr, *sptr;
  const uint16_t *cnbr, *snbr;
};

// 32-bit half of activeRows holding bit position p of word w.
__device__ __forceinline__ uint32_t *half_of(uint64_t *active, int w, int p) {
  return reinterpret_cast<uint32_t *>(active + w) + (p >> 5);
}

template <int KP>
__device__ __forceinline__ void cover_row(const State &s, int v, int c, int lane) {
  using F = Fields<KP>;
  if (lane == 0) {
    const int p = v * KP;
    const uint32_t fm = (uint32_t)F::FM << (p & 31);
    const uint32_t old = atomicAnd(half_of(s.active, p >> 6, p & 63), ~fm);
    s.oldnib[v] = (uint8_t)((old & fm) >> (p & 31));
    uint32_t *uh = half_of(s.unas, p >> 6, p & 63);
    *uh &= ~fm;
    s.x[v] = (int8_t)c;
  }
  const int ce = s.cptr[v + 1];
  for (int i = s.cptr[v] + lane; i < ce; i += 32) {
    const int p = (int)s.cnbr[i] * KP + c;
    const uint32_t bit = 1u << (p & 31);
    const uint32_t old = atomicAnd(half_of(s.active, p >> 6, p & 63), ~bit);
    s.clrb[i] = (old & bit) ? 1 : 0;
  }
  __syncwarp();
}

template <int KP>
__device__ __forceinline__ void uncover_row(const State &s, int v, int c, int lane) {
  using F = Fields<KP>;
  const int ce = s.cptr[v + 1];
  for (int i = s.cptr[v] + lane; i < ce; i += 32) {
    if (s.clrb[i]) {
      const int p = (int)s.cnbr[i] * KP + c;
      atomicOr(half_of(s.active, p >> 6, p & 63), 1u << (p & 31));
    }
  }
  if (lane == 0) {
    const int p = v * KP;
    atomicOr(half_of(s.active, p >> 6, p & 63), (uint32_t)s.oldnib[v] << (p & 31));
    uint32_t *uh = half_of(s.unas, p >> 6, p & 63);
    *uh |= (uint32_t)F::FM << (p & 31);
    s.x[v] = -1;
  }
  __syncwarp();
}

// Per-mask counts of neighbours holding each mask, summed over the warp
// (8-bit packed lanes contributions, one reduction per 4 masks).
template <int KP>
__device__ __forceinline__ void count_masks(const uint16_t *nbr, int b, int e, const int8_t *x,
                                            int lane, int (&cnt)[KP]) {
  for (int base = b; base < e; base += 32) {
    const int i = base + lane;
    uint32_t lo = 0, hi = 0;
    if (i < e) {
      const int xu = x[nbr[i]];
      if (xu >= 0) {
        if (KP == 4 || xu < 4) lo = 1u << (8 * xu);
        else hi = 1u << (8 * (xu - 4));
      }
    }
    lo = __reduce_add_sync(FULL, lo);
    if (KP == 8) hi = __reduce_add_sync(FULL, hi);
#pragma unroll
    for (int c = 0; c < KP; ++c)
      cnt[c] += (int)(((c < 4) ? (lo >> (8 * c)) : (hi >> (8 * (c - 4)))) & 0xFFu);
  }
}

// Depth-first search of one instance; the state is initialised already.
template <int KP>
__device__ __forceinline__ int search(const State &s, const InstDesc &d, int lane, int64_t budget,
                                      int64_t time_limit_ns, int64_t &best_out,
                                      int64_t &nodes_out, int64_t &work_out) {
  using F = Fields<KP>;
  const int n = d.n, W = d.W, k = d.k;
  const int Cc = d.cost_conflict, Cs = d.cost_stitch;
  int64_t best = INF, nodes = 0, g = 0, work = 0;
  int level = 0;
  int status = MPLD_OK;
  const uint64_t t0 = globaltimer();
  bool enter = true;

  for (;;) {
    if (enter) {
      // ---- a node: one call of the recursive search ----
      if (budget > 0 && best < INF && nodes >= budget) { status = MPLD_BUDGET; break; }
      ++nodes;
      work += 2 * (int64_t)(n - level);
      if ((nodes & 1023) == 0) {
        uint64_t now = lane == 0 ? globaltimer() : 0;
        now = __shfl_sync(FULL, now, 0);
        if ((int64_t)(now - t0) > time_limit_ns) { status = MPLD_TIMEOUT; break; }
      }
      // column choice: min over uncovered P_v of popc(activeRows & colRows[P_v])
      uint32_t key = 0xFFFFFFFFu, z = 0;
      for (int w = lane; w < W; w += 32) {
        const uint64_t a = s.active[w], um = s.unas[w];
        const uint64_t key4 = field_counts<KP>(a) | (~um & F::FILL);
        uint64_t le = fields_le<KP>(key4, 0);
        z += __popcll(le);
        uint32_t t = 0;
        while (!le && t < (uint32_t)k) le = fields_le<KP>(key4, ++t);
        if (le) {
          const uint32_t seg =
              (uint32_t)(w * F::PER_WORD) + (uint32_t)((__ffsll((long long)le) - 1) / KP);
          key = min(key, (t << 24) | seg);
        }
      }
      key = __reduce_min_sync(FULL, key);
      z = __reduce_add_sync(FULL, z);
      if (key == 0xFFFFFFFFu) {
        // leaf: every primary column covered
        if (g < best) {
          best = g;
          for (int i = lane; i < n; i += 32) d.mask[i] = s.x[i];
          if (best == 0) break;
        }
        enter = false;
        continue;
      }
      if (best < INF && g + (int64_t)Cc * z >= best) { enter = false; continue; }
      const int v = (int)(key & 0xFFFFFFu);
      // added cost of each row (v, c) against the current assignment (Eq. 1)
      int cc[KP], sc[KP];
#pragma unroll
      for (int c = 0; c < KP; ++c) { cc[c] = 0; sc[c] = 0; }
      const int cb = s.cptr[v], ce = s.cptr[v + 1];
      const int sb = s.sptr[v], se = s.sptr[v + 1];
      count_masks<KP>(s.cnbr, cb, ce, s.x, lane, cc);
      count_masks<KP>(s.snbr, sb, se, s.x, lane, sc);
      int stot = 0;
#pragma unroll
      for (int c = 0; c < KP; ++c) stot += sc[c];
      work += (int64_t)k * (ce - cb + se - sb) + 5 * (1 + ce - cb);
      uint32_t keys[KP];
#pragma unroll
      for (int c = 0; c < KP; ++c) {
        const uint32_t inc = (uint32_t)(Cc * cc[c] + Cs * (stot - sc[c]));
        keys[c] = c < k ? ((inc << 3) | (uint32_t)c) : 0xFFFFFFFFu;
      }
      sort_keys<KP>(keys);
      uint32_t ord = 0;
#pragma unroll
      for (int i = 0; i < KP; ++i) ord |= (keys[i] & 7u) << (4 * i);
      if (lane == 0) {
        s.lv_g[level] = g;
        s.lv_v[level] = v;
        s.lv_ord[level] = ord;
        s.lv_next[level] = 1;
#pragma unroll
        for (int i = 1; i < KP; ++i)
          if (i < k) s.lv_inc[level * KP + i] = (int32_t)(keys[i] >> 3);
      }
      cover_row<KP>(s, v, (int)(ord & 0xFu), lane);
      g += (int64_t)(keys[0] >> 3);
      ++level;
      continue;
    }
    // ---- backtrack: uncover the row of the level above, try its next row ----
    if (level == 0) break;
    --level;
    const int v = s.lv_v[level];
    const int nxt = s.lv_next[level];
    const uint32_t ord = s.lv_ord[level];
    uncover_row<KP>(s, v, (int)((ord >> (4 * (nxt - 1))) & 0xFu), lane);
    if (nxt >= k) continue;  // every row of this column tried
    const int c = (int)((ord >> (4 * nxt)) & 0xFu);
    g = s.lv_g[level] + s.lv_inc[level * KP + nxt];
    work += 5 * (1 + s.cptr[v + 1] - s.cptr[v]);
    if (lane == 0) s.lv_next[level] = (uint8_t)(nxt + 1);
    cover_row<KP>(s, v, c, lane);
    ++level;
    enter = true;
  }
  best_out = best;
  nodes_out = nodes;
  work_out = work;
  return status;
}

// Initialise the state at `base` and search; SM selects the memory space of
// `base` and `ro` at compile time.
template <int KP, bool SM>
__device__ __forceinline__ void run_in(const InstDesc &d, uint8_t *base, const uint8_t *ro,
                                       const LaunchArgs &a, int lane) {
  using F = Fields<KP>;
  const int n = d.n, W = d.W;
  const StateLayout L = state_layout(n, W, d.ne2, KP);
  const RoLayout R = ro_layout(n, d.ne2, d.ns2);
  State s;
  s.active = (uint64_t *)(base + L.active);
  s.unas = (uint64_t *)(base + L.unas);
  s.lv_g = (int64_t *)(base + L.lv_g);
  s.lv_inc = (int32_t *)(base + L.lv_inc);
  s.lv_ord = (uint32_t *)(base + L.lv_ord);
  s.lv_v = (int32_t *)(base + L.lv_v);
  s.lv_next = base + L.lv_next;
  s.x = (int8_t *)(base + L.x);
  s.oldnib = base + L.oldnib;
  s.clrb = base + L.clrb;
  s.cptr = (const int32_t *)(ro + R.cptr);
  s.sptr = (const int32_t *)(ro + R.sptr);
  s.cnbr = (const uint16_t *)(ro + R.cnbr);
  s.snbr = (const uint16_t *)(ro + R.snbr);

  // initial state: every row active, every primary column uncovered
  const uint64_t kmask = (1ull << d.k) - 1ull;
  uint64_t rowpat = 0, fieldpat = 0;
#pragma unroll
  for (int j = 0; j < F::PER_WORD; ++j) {
    rowpat |= kmask << (j * KP);
    fieldpat |= F::FM << (j * KP);
  }
  for (int w = lane; w < W; w += 32) {
    const int segs = n - w * F::PER_WORD;
    const uint64_t keep = segs >= F::PER_WORD ? ~0ull : ((1ull << (segs * KP)) - 1ull);
    s.active[w] = rowpat & keep;
    s.unas[w] = fieldpat & keep;
  }
  for (int i = lane; i < n; i += 32) s.x[i] = -1;
  __syncwarp();

  int64_t best = INF, nodes = 0, work = 0;
  const int st = search<KP>(s, d, lane, a.budget, a.time_limit_ns, best, nodes, work);
  if (lane == 0) {
    d.res->cost = best;
    d.res->nodes = nodes;
    d.res->status = st;
    d.res->work = work;
  }
  __syncwarp();
}

// Stage and run one instance.  Returns false when the warp's slot must not
// be used again (a bulk copy into it did not complete within the wait limit;
// the instance then runs from global memory).
template <int KP>
__device__ __forceinline__ bool run_instance(const InstDesc &d, uint32_t slot_off, int slot_bytes,
                                             uint64_t *bar, uint32_t &phase, const LaunchArgs &a,
                                             int lane) {
  const StateLayout L = state_layout(d.n, d.W, d.ne2, KP);
  const RoLayout R = ro_layout(d.n, d.ne2, d.ns2);
  if (slot_bytes <= 0 || (int)(L.bytes + R.bytes) > slot_bytes) {
    run_in<KP, false>(d, d.scratch, d.ro, a, lane);
    return true;
  }
  uint8_t *slot = g_smem + slot_off;
  uint8_t *dst = slot + L.bytes;
  if (R.bytes >= TMA_MIN_BYTES) {
    // one bulk copy of the whole read-only block into shared memory
    __syncwarp();
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar, R.bytes);
      bulk_copy_g2s(dst, d.ro, R.bytes, bar);
    }
    bool ok = false;
    for (uint32_t it = 0; it < WAIT_LIMIT && !ok; ++it) ok = mbar_try_wait(bar, phase);
    phase ^= 1u;
    if (!ok) {
      if (lane == 0) atomicExch(a.err, MPLD_E_TIMEOUT);
      for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, phase ^ 1u)) break;
      run_in<KP, false>(d, d.scratch, d.ro, a, lane);
      return false;
    }
  } else {
    const uint4 *src = (const uint4 *)d.ro;
    uint4 *d4 = (uint4 *)dst;
    for (uint32_t i = lane; i < R.bytes / 16; i += 32) d4[i] = __ldg(src + i);
  }
  run_in<KP, true>(d, slot, dst, a, lane);
  return true;
}

__global__ void __launch_bounds__(512, 1) mpld_search_kernel(const LaunchArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  uint64_t *bars = (uint64_t *)g_smem;
  const uint32_t bar_bytes = align16(8u * (uint32_t)nw);
  const uint32_t slot_off = bar_bytes + (uint32_t)warp * (uint32_t)(a.slot_bytes > 0 ? a.slot_bytes : 0);
  int slot_bytes = a.slot_bytes;
  uint64_t *bar = bars + warp;
  if (lane == 0) mbar_init(bar);
  __syncwarp();
  if (lane == 0) fence_proxy_async();
  __syncwarp();
  uint32_t phase = 0;

  int idx = a.queue ? 0 : blockIdx.x * nw + warp;
  for (;;) {
    if (a.queue) {
      uint32_t t = 0;
      if (lane == 0) t = atomicAdd(a.queue, 1u);
      idx = (int)__shfl_sync(FULL, t, 0);
    }
    if (idx >= a.n_inst) break;
    const InstDesc d = a.desc[a.order ? a.order[idx] : idx];
    const bool ok = d.k <= 4 ? run_instance<4>(d, slot_off, slot_bytes, bar, phase, a, lane)
                             : run_instance<8>(d, slot_off, slot_bytes, bar, phase, a, lane);
    if (!ok) slot_bytes = 0;
    if (!a.queue) break;
  }
}

// Largest dynamic shared memory size already granted to the kernel; the
// attribute is only raised, and only outside stream capture (the shape is
// chosen, and the attribute set, before any capture begins).
int g_smem_granted = 48 * 1024;

int ensure_smem(size_t smem) {
  if ((int)smem <= g_smem_granted) return MPLD_OK;
  if (cudaFuncSetAttribute(mpld_search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return MPLD_E_CUDA;
  }
  g_smem_granted = (int)smem;
  return MPLD_OK;
}

}  // namespace
}  // namespace mpld

using mpld::LaunchArgs;

extern "C" int mpld_internal_launch(const LaunchArgs *a, int ctas, int warps_per_cta,
                                    void *stream) {
  const size_t smem = mpld::align16(8u * (uint32_t)warps_per_cta) +
                      (size_t)warps_per_cta * (size_t)(a->slot_bytes > 0 ? a->slot_bytes : 0);
  if (mpld::ensure_smem(smem) != MPLD_OK) return MPLD_E_CUDA;
  mpld::mpld_search_kernel<<<ctas, warps_per_cta * 32, smem, (cudaStream_t)stream>>>(*a);
  return cudaGetLastError() == cudaSuccess ? MPLD_OK : MPLD_E_CUDA;
}

extern "C" int mpld_internal_num_sms(void) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// Largest per-warp slot for a CTA of `warps_per_cta` warps (opt-in maximum).
extern "C" int mpld_internal_max_slot_bytes(int warps_per_cta) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  const int avail = optin - (int)mpld::align16(8u * (uint32_t)warps_per_cta);
  return (avail / warps_per_cta) & ~15;
}

extern "C" int mpld_internal_ctas_per_sm(int warps_per_cta, int slot_bytes) {
  const size_t smem =
      mpld::align16(8u * (uint32_t)warps_per_cta) + (size_t)warps_per_cta * (size_t)slot_bytes;
  if (mpld::ensure_smem(smem) != MPLD_OK) return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, mpld::mpld_search_kernel,
                                                    warps_per_cta * 32, smem) != cudaSuccess)
    return 0;
  return blocks;
}
