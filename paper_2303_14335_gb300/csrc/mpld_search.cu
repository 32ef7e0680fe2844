// mpld_search.cu -- the matrix-cover search (Sec. 2.3, Algorithm 1) for
// sm_103a.
//
// One warp runs one search instance (a sub-graph of the layout).  The EC
// matrix's active rows are a bitset in shared memory with one field per
// segment (its k row bits plus a top "column uncovered" bit), and the three
// operations of Algorithm 1 become bit operations on it:
//   * column choice (Algorithm 1, "select an uncovered column"): lane l
//     takes the uncovered primary columns P_v, v = l, l+32, ..., computes
//     popc(activeRows & colRows[P_v]) on v's field, and the warp takes the
//     minimum of (count, v) with __reduce_min_sync, so ties go to the lowest
//     segment index;
//   * cover of row (v, c) (Eq. 2 "Cover", Algorithm 1 "cover rw and its
//     affected rows"): activeRows &= ~colRows[j] for every column j of the
//     row -- v's field, and bit c of every conflict neighbour u (column
//     S_{(v,u),c}); lane i handles neighbour i with a 32-bit shared atomic
//     AND and records whether it cleared the bit;
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
constexpr int32_t INF32 = 0x7FFFFFFF;
constexpr uint32_t TMA_MIN_BYTES = 1024;     // smaller blocks use vector loads
constexpr uint32_t WAIT_LIMIT = 1u << 22;    // bounded mbarrier wait

__device__ __forceinline__ void cas_u32(uint32_t &a, uint32_t &b) {
  const uint32_t lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// Sort keys ((inc << 3) | mask) ascending with a fixed network.
template <int MK> __device__ __forceinline__ void sort_keys(uint32_t (&k)[MK]);
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

// FT: field type of the activeRows bitset (uint8_t for k <= 7, uint16_t for
// k = 8); MK: width of the row sort (4 for k <= 4, else 8).
template <typename FT, int MK>
struct Search {
  static constexpr uint32_t FB = 8 * sizeof(FT);   // bits per field
  static constexpr uint32_t FLAG = 1u << (FB - 1);  // column P_v uncovered
  static constexpr uint32_t FMASK = (FB == 8) ? 0xFFu : 0xFFFFu;

  FT *rows;        // activeRows fields
  FT *oldf;        // field of v before its row was covered
  int8_t *x;
  uint8_t *clrb;
  uint4 *lv;       // {g, v | tried << 16, order, inc of row 1}
  int32_t *lvx;    // inc of rows 2.. per level (MK entries per level)
  const int2 *ptr; // {conflict offset, stitch offset} per segment
  const uint16_t *cnbr, *snbr;
  int n, k;
  int Cc, Cs;
  uint32_t kmask;

  __device__ __forceinline__ uint32_t *word_of(int v) const {
    return reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(rows) +
                                        (((uint32_t)v * sizeof(FT)) & ~3u));
  }
  __device__ __forceinline__ uint32_t shift_of(int v) const {
    return (((uint32_t)v * sizeof(FT)) & 3u) * 8u;
  }

  // Cover row (v, c): clear v's field and bit c of every conflict neighbour;
  // `u` is lane's neighbour (valid for lane < ce - cb, first 32 only).
  __device__ __forceinline__ void cover(int v, int c, int cb, int ce, int u, int lane) const {
    if (lane == 0) {
      const uint32_t sh = shift_of(v);
      const uint32_t old = atomicAnd(word_of(v), ~(FMASK << sh));
      oldf[v] = (FT)((old >> sh) & FMASK);
      x[v] = (int8_t)c;
    }
    for (int i = cb + lane; i < ce; i += 32) {
      if (i >= cb + 32) u = cnbr[i];
      const uint32_t bit = 1u << (shift_of(u) + (uint32_t)c);
      const uint32_t old = atomicAnd(word_of(u), ~bit);
      clrb[i] = (old & bit) ? 1 : 0;
    }
    __syncwarp();
  }

  // Uncover row (v, c); leaves lane's first neighbour in `u`.
  __device__ __forceinline__ void uncover(int v, int c, int cb, int ce, int &u, int lane) const {
    for (int i = cb + lane; i < ce; i += 32) {
      const int w = cnbr[i];
      if (i < cb + 32) u = w;
      if (clrb[i]) atomicOr(word_of(w), 1u << (shift_of(w) + (uint32_t)c));
    }
    if (lane == 0) {
      atomicOr(word_of(v), (uint32_t)oldf[v] << shift_of(v));
      x[v] = -1;
    }
    __syncwarp();
  }

  // Per-mask counts of a neighbour list, packed 8 bits per mask, warp-summed.
  __device__ __forceinline__ void count(const uint16_t *nbr, int b, int e, int lane, int &first,
                                        uint32_t &lo, uint32_t &hi) const {
    lo = 0;
    hi = 0;
    for (int base = b; base < e; base += 32) {
      const int i = base + lane;
      uint32_t l = 0, h = 0;
      if (i < e) {
        const int w = nbr[i];
        if (base == b) first = w;
        const int xu = x[w];
        if (xu >= 0) {
          if (MK == 4 || xu < 4) l = 1u << (8 * xu);
          else h = 1u << (8 * (xu - 4));
        }
      }
      lo += __reduce_add_sync(FULL, l);
      if (MK == 8) hi += __reduce_add_sync(FULL, h);
    }
  }

  __device__ __forceinline__ int run(int lane, int64_t budget, int64_t time_limit_ns,
                                     int8_t *best_mask, int32_t &best_out, int64_t &nodes_out,
                                     int64_t &work_out) const {
    int32_t best = INF32, g = 0;
    int64_t nodes = 0, work = 0;
    int level = 0;
    int status = MPLD_OK;
    const uint64_t t0 = globaltimer();
    bool enter = true;
    for (;;) {
      if (enter) {
        // ---- a node: one call of the recursive search ----
        if (budget > 0 && best < INF32 && nodes >= budget) { status = MPLD_BUDGET; break; }
        ++nodes;
        work += 2 * (int64_t)(n - level);
        if ((nodes & 1023) == 0) {
          uint64_t now = lane == 0 ? globaltimer() : 0;
          now = __shfl_sync(FULL, now, 0);
          if ((int64_t)(now - t0) > time_limit_ns) { status = MPLD_TIMEOUT; break; }
        }
        // column choice: min over uncovered P_v of popc(activeRows & colRows[P_v])
        uint32_t key = 0xFFFFFFFFu, z = 0;
        for (int v = lane; v < n; v += 32) {
          const uint32_t f = rows[v];
          const uint32_t cnt = __popc(f & kmask);
          const uint32_t kv = (f & FLAG) ? ((cnt << 16) | (uint32_t)v) : 0xFFFFFFFFu;
          key = min(key, kv);
          z += kv <= 0xFFFFu;  // uncovered with no active row
        }
        key = __reduce_min_sync(FULL, key);
        if (key == 0xFFFFFFFFu) {
          // leaf: every primary column covered
          if (g < best) {
            best = g;
            for (int i = lane; i < n; i += 32) best_mask[i] = x[i];
            if (best == 0) break;
          }
          enter = false;
          continue;
        }
        if (best < INF32) {
          z = __reduce_add_sync(FULL, z);
          if ((int64_t)g + (int64_t)Cc * z >= best) { enter = false; continue; }
        }
        const int v = (int)(key & 0xFFFFu);
        // added cost of each row (v, c) against the current assignment (Eq. 1)
        const int2 p0 = ptr[v], p1 = ptr[v + 1];
        int u = 0, us = 0;
        uint32_t clo, chi, slo, shi;
        count(cnbr, p0.x, p1.x, lane, u, clo, chi);
        count(snbr, p0.y, p1.y, lane, us, slo, shi);
        work += (int64_t)k * (p1.x - p0.x + p1.y - p0.y) + 5 * (1 + p1.x - p0.x);
        int stot = 0;
#pragma unroll
        for (int c = 0; c < MK; ++c)
          stot += (int)((((c < 4) ? (slo >> (8 * c)) : (shi >> (8 * (c - 4))))) & 0xFFu);
        uint32_t keys[MK];
#pragma unroll
        for (int c = 0; c < MK; ++c) {
          const int cc = (int)((((c < 4) ? (clo >> (8 * c)) : (chi >> (8 * (c - 4))))) & 0xFFu);
          const int sc = (int)((((c < 4) ? (slo >> (8 * c)) : (shi >> (8 * (c - 4))))) & 0xFFu);
          const uint32_t inc = (uint32_t)(Cc * cc + Cs * (stot - sc));
          keys[c] = c < k ? ((inc << 3) | (uint32_t)c) : 0xFFFFFFFFu;
        }
        sort_keys<MK>(keys);
        uint32_t ord = 0;
#pragma unroll
        for (int i = 0; i < MK; ++i) ord |= (keys[i] & 7u) << (4 * i);
        if (lane == 0) {
          lv[level] = make_uint4((uint32_t)g, (uint32_t)v | (1u << 16), ord, keys[1] >> 3);
#pragma unroll
          for (int i = 2; i < MK; ++i)
            if (i < k) lvx[level * MK + i] = (int32_t)(keys[i] >> 3);
        }
        cover(v, (int)(ord & 7u), p0.x, p1.x, u, lane);
        g += (int32_t)(keys[0] >> 3);
        ++level;
        continue;
      }
      // ---- backtrack: uncover the row of the level above, try its next row ----
      if (level == 0) break;
      --level;
      const uint4 rec = lv[level];
      const int v = (int)(rec.y & 0xFFFFu);
      const int nxt = (int)(rec.y >> 16);
      const int2 p0 = ptr[v], p1 = ptr[v + 1];
      int u = 0;
      uncover(v, (int)((rec.z >> (4 * (nxt - 1))) & 7u), p0.x, p1.x, u, lane);
      if (nxt >= k) continue;  // every row of this column tried
      const int c = (int)((rec.z >> (4 * nxt)) & 7u);
      g = (int32_t)rec.x + (nxt == 1 ? (int32_t)rec.w : lvx[level * MK + nxt]);
      work += 5 * (1 + p1.x - p0.x);
      if (lane == 0) lv[level].y = (uint32_t)v | ((uint32_t)(nxt + 1) << 16);
      cover(v, c, p0.x, p1.x, u, lane);
      ++level;
      enter = true;
    }
    best_out = best;
    nodes_out = nodes;
    work_out = work;
    return status;
  }
};

// Initialise the state at `base` and search.  SM says at compile time
// whether `base` and `ro` point into shared memory.
template <typename FT, int MK, bool SM>
__device__ __forceinline__ void run_in(const InstDesc &d, uint8_t *base, const uint8_t *ro,
                                       const LaunchArgs &a, int lane) {
  const int n = d.n;
  const StateLayout L = state_layout(n, d.ne2, d.k);
  const RoLayout R = ro_layout(n, d.ne2, d.ns2);
  Search<FT, MK> s;
  s.rows = (FT *)(base + L.rows);
  s.oldf = (FT *)(base + L.oldf);
  s.x = (int8_t *)(base + L.x);
  s.clrb = base + L.clrb;
  s.lv = (uint4 *)(base + L.lv);
  s.lvx = (int32_t *)(base + L.lvx);
  s.ptr = (const int2 *)(ro + R.ptr);
  s.cnbr = (const uint16_t *)(ro + R.cnbr);
  s.snbr = (const uint16_t *)(ro + R.snbr);
  s.n = n;
  s.k = d.k;
  s.Cc = d.cost_conflict;
  s.Cs = d.cost_stitch;
  s.kmask = (1u << d.k) - 1u;
  // initial state: every row active, every primary column uncovered
  const FT init = (FT)(s.kmask | Search<FT, MK>::FLAG);
  for (int i = lane; i < n; i += 32) {
    s.rows[i] = init;
    s.x[i] = -1;
  }
  __syncwarp();
  int32_t best = INF32;
  int64_t nodes = 0, work = 0;
  const int st = s.run(lane, a.budget, a.time_limit_ns, d.mask, best, nodes, work);
  if (lane == 0) {
    d.res->cost = best == INF32 ? INT64_MAX : (int64_t)best;
    d.res->nodes = nodes;
    d.res->status = st;
    d.res->work = work;
  }
  __syncwarp();
}

template <typename FT, int MK>
__device__ __forceinline__ bool run_instance(const InstDesc &d, uint32_t slot_off, int slot_bytes,
                                             uint64_t *bar, uint32_t &phase, const LaunchArgs &a,
                                             int lane) {
  const StateLayout L = state_layout(d.n, d.ne2, d.k);
  const RoLayout R = ro_layout(d.n, d.ne2, d.ns2);
  if (slot_bytes <= 0 || (int)(L.bytes + R.bytes) > slot_bytes) {
    run_in<FT, MK, false>(d, d.scratch, d.ro, a, lane);
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
      // the copy did not land: record it, wait (bounded) for the copy still
      // in flight, run from global memory and give up the slot
      if (lane == 0) atomicExch(a.err, MPLD_E_TIMEOUT);
      for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, phase ^ 1u)) break;
      run_in<FT, MK, false>(d, d.scratch, d.ro, a, lane);
      return false;
    }
  } else {
    const uint4 *src = (const uint4 *)d.ro;
    uint4 *d4 = (uint4 *)dst;
    for (uint32_t i = lane; i < R.bytes / 16; i += 32) d4[i] = __ldg(src + i);
  }
  run_in<FT, MK, true>(d, slot, dst, a, lane);
  return true;
}

__global__ void __launch_bounds__(512, 1) mpld_search_kernel(const LaunchArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  uint64_t *bars = (uint64_t *)g_smem;
  const uint32_t bar_bytes = align16(8u * (uint32_t)nw);
  const uint32_t slot_off =
      bar_bytes + (uint32_t)warp * (uint32_t)(a.slot_bytes > 0 ? a.slot_bytes : 0);
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
    bool ok;
    if (d.k <= 4) ok = run_instance<uint8_t, 4>(d, slot_off, slot_bytes, bar, phase, a, lane);
    else if (d.k <= 7) ok = run_instance<uint8_t, 8>(d, slot_off, slot_bytes, bar, phase, a, lane);
    else ok = run_instance<uint16_t, 8>(d, slot_off, slot_bytes, bar, phase, a, lane);
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
