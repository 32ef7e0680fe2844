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
//     S_{(v,u),c}); lane i handles neighbour i and saves u's field first;
//   * uncover (Eq. 2 "Uncover"): the saved fields are written back, newest
//     level first, through an explicit per-level stack instead of
//     recursion.
// Rows of the chosen column are visited in ascending (added cost, mask),
// including rows that are no longer active: those are the "conflict
// candidates" of Algorithm 1 and pay the conflict cost of Eq. 1.  A node is
// pruned when its cost plus cost_conflict times the number of uncovered
// columns with no active row reaches the incumbent; children whose path
// cost alone reaches it are counted without being entered.
//
// Instances of at most 32 words of fields (n <= 128 segments for k <= 7)
// run a register-resident form of the same search (reg_search): each lane
// keeps its four fields, masks and per-mask neighbour counts in registers
// and the adjacency becomes a bit matrix; larger instances run Search.
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

#include <algorithm>
#include <mutex>

#include "mpld_internal.h"
#include "../../include/mpld.h"

namespace mpld {
namespace {

extern __shared__ __align__(16) uint8_t g_smem[];

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int32_t INF32 = 0x7FFFFFFF;
constexpr uint32_t TMA_MIN_BYTES = 1024;     // smaller blocks use vector loads
constexpr uint32_t WAIT_LIMIT = 1u << 22;    // bounded mbarrier wait
constexpr uint32_t TEAM_BYTES = 320;          // a CTA team's reduction words and
                                              // the split exact search's context
constexpr uint32_t PAR_CTX_OFF = 128;         // ParCtx (48 bytes)
constexpr uint32_t PAR_WKEY_OFF = 176;        // each warp's best key (16 warps)
static_assert(PAR_CTX_OFF + sizeof(ParCtx) <= PAR_WKEY_OFF && PAR_WKEY_OFF + 16 * 8 <= TEAM_BYTES,
              "split-search context must fit the shared-memory head");

// Dynamic shared memory of the batched kernel: the CTA team's reduction
// words, one mbarrier per warp, then one slot per warp.
__host__ __device__ __forceinline__ uint32_t kernel_head_bytes(int warps_per_cta) {
  return TEAM_BYTES + ((8u * (uint32_t)warps_per_cta + 15u) & ~15u);
}

__device__ __forceinline__ void cas_u32(uint32_t &a, uint32_t &b) {
  const uint32_t lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}

// Sort keys ((inc << 3) | mask) ascending with a fixed network.
template <int MK> __device__ __forceinline__ void sort_keys(uint32_t (&k)[MK]);
template <> __device__ __forceinline__ void sort_keys<2>(uint32_t (&k)[2]) { cas_u32(k[0], k[1]); }
template <> __device__ __forceinline__ void sort_keys<3>(uint32_t (&k)[3]) {
  cas_u32(k[0], k[1]); cas_u32(k[1], k[2]); cas_u32(k[0], k[1]);
}
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

// Programmatic dependent launch: let the grid launched after this one (with
// programmatic stream serialization) start its blocks as SMs free up, and,
// in that grid, wait until the grids before it have completed and their
// memory is visible.  Both return at once when no such launch is involved.
__device__ __forceinline__ void launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;");
}
__device__ __forceinline__ void wait_prerequisites() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
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

// Read-only data (adjacency) of an instance whose block stays in global
// memory is read from L2: device memory of finished work may be rewritten
// while a grid runs, and an SM's L1 may still hold lines of it.
template <bool SM, typename T>
__device__ __forceinline__ T ro_ld(const T *p) {
  if constexpr (SM) return *p;
  else return __ldcg(p);
}

// The threads that search one instance together.  WarpTeam: one warp, with
// warp-synchronous primitives.  CtaTeam: every thread of a CTA (instances
// too large for one warp's pace), with reductions through a few words of
// shared memory; every member calls every primitive (the search's control
// flow depends only on reduced values).
struct WarpTeam {
  int rank;
  __device__ __forceinline__ int size() const { return 32; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ uint32_t min(uint32_t v) const { return __reduce_min_sync(FULL, v); }
  __device__ __forceinline__ uint32_t sum(uint32_t v) const { return __reduce_add_sync(FULL, v); }
  __device__ __forceinline__ uint64_t bcast0(uint64_t v) const { return __shfl_sync(FULL, v, 0); }
};
struct CtaTeam {
  int rank, nthreads;
  uint32_t *red;   // shared: one word per warp, then two for a broadcast
  __device__ __forceinline__ int size() const { return nthreads; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ uint32_t min(uint32_t v) const {
    v = __reduce_min_sync(FULL, v);
    if ((rank & 31) == 0) red[rank >> 5] = v;
    __syncthreads();
    uint32_t r = red[0];
    for (int w = 1; w < (nthreads >> 5); ++w) r = ::min(r, red[w]);
    __syncthreads();
    return r;
  }
  __device__ __forceinline__ uint32_t sum(uint32_t v) const {
    v = __reduce_add_sync(FULL, v);
    if ((rank & 31) == 0) red[rank >> 5] = v;
    __syncthreads();
    uint32_t r = 0;
    for (int w = 0; w < (nthreads >> 5); ++w) r += red[w];
    __syncthreads();
    return r;
  }
  __device__ __forceinline__ uint64_t bcast0(uint64_t v) const {
    const int w = nthreads >> 5;
    if (rank == 0) {
      red[w] = (uint32_t)v;
      red[w + 1] = (uint32_t)(v >> 32);
    }
    __syncthreads();
    const uint64_t r = (uint64_t)red[w] | ((uint64_t)red[w + 1] << 32);
    __syncthreads();
    return r;
  }
};

// Column classes of a giant instance, for a column choice that does not scan
// every segment: per count class m (0..k), a bit per segment that is
// uncovered with exactly m active rows, a summary bit per 32-bit word of it
// that may be non-zero (set when a segment joins the word; a bit whose word
// has emptied is cleared when the column choice meets it), and the class
// size; under column rule 1 also a bit per breadth-first rank that is
// uncovered, with an exact summary.  The fewest-rows column is then the
// lowest set bit of the first non-empty class (lowest index on ties, as the
// scan gives), found through the summary; covers and undos move only the
// segment and its neighbours between classes, with atomics whose results
// nothing waits for.  One warp keeps them in shared memory.
struct Buckets {
  uint32_t *cls;   // [k+1][w32]
  uint32_t *sum;   // [k+1][s32]
  int32_t *cnt;    // [k+1]
  uint32_t *ur;    // [w32] rank space (rule 1)
  uint32_t *urs;   // [s32]
  int w32, s32, k;   // layout: bucket_bytes(n, k) bytes
  __device__ void carve(uint8_t *base, int n, int kk) {
    k = kk;
    w32 = (n + 31) / 32;
    s32 = (w32 + 31) / 32;
    uint32_t *p = (uint32_t *)base;
    cls = p; p += (k + 1) * w32;
    sum = p; p += (k + 1) * s32;
    cnt = (int32_t *)p; p += k + 1;
    ur = p; p += w32;
    urs = p;
  }
  // every segment uncovered with k active rows (one warp)
  __device__ void init(int n, int lane) const {
    // classes below k and every summary start empty; class k and the rank
    // map hold every segment
    for (int i = lane; i < k * w32; i += 32) cls[i] = 0u;
    for (int i = lane; i < (k + 1) * s32; i += 32) sum[i] = 0u;
    for (int i = lane; i < s32; i += 32) urs[i] = 0u;
    for (int w = lane; w < w32; w += 32) {
      const int lo = 32 * w;
      const uint32_t bits = n - lo >= 32 ? 0xFFFFFFFFu : ((1u << (n - lo)) - 1u);
      cls[k * w32 + w] = bits;
      ur[w] = bits;
    }
    for (int i = lane; i <= k; i += 32) cnt[i] = i == k ? n : 0;
    __syncwarp();
    for (int w = lane; w < w32; w += 32) {
      atomicOr(&sum[k * s32 + (w >> 5)], 1u << (w & 31));
      atomicOr(&urs[w >> 5], 1u << (w & 31));
    }
    __syncwarp();
  }
  // segment v leaves class a (a < 0: none) and joins class b (b < 0: none)
  __device__ __forceinline__ void move(int v, int a, int b) const {
    if (a == b) return;
    const uint32_t bit = 1u << (v & 31);
    const int w = v >> 5;
    if (a >= 0) {
      atomicAnd(&cls[a * w32 + w], ~bit);
      atomicSub(&cnt[a], 1);
    }
    if (b >= 0) {
      atomicOr(&cls[b * w32 + w], bit);
      atomicAdd(&cnt[b], 1);
      atomicOr(&sum[b * s32 + (w >> 5)], 1u << (w & 31));
    }
  }
  // lowest segment of class m, which is not empty (every lane gets it);
  // summary bits met on the way whose word has emptied are cleared
  __device__ __forceinline__ int lowest_in(int m, int lane) const {
    uint32_t *sm = sum + m * s32;
    const uint32_t *bm = cls + m * w32;
    for (int base = 0; base < s32;) {
      const uint32_t sv = base + lane < s32 ? sm[base + lane] : 0u;
      const uint32_t nz = __ballot_sync(FULL, sv != 0u);
      if (!nz) {
        base += 32;
        continue;
      }
      const int l = __ffs(nz) - 1;
      uint32_t s0 = __shfl_sync(FULL, sv, l);
      bool stale = false;
      while (s0) {
        const int j = __ffs(s0) - 1;
        const int w = (base + l) * 32 + j;
        const uint32_t wv = bm[w];
        if (wv) {
          // a cleared bit is ordered before the moves of the next cover
          if (stale) __syncwarp();
          return w * 32 + __ffs(wv) - 1;
        }
        if (lane == 0) atomicAnd(&sm[base + l], ~(1u << j));
        stale = true;
        s0 &= s0 - 1u;
      }
      __syncwarp();   // every bit of this summary word was stale: read it again
    }
    return -1;
  }
  __device__ __forceinline__ void rank_set(int r, bool on) const {
    const uint32_t bit = 1u << (r & 31);
    const int w = r >> 5;
    if (on) {
      atomicOr(&ur[w], bit);
      atomicOr(&urs[w >> 5], 1u << (w & 31));
    } else {
      const uint32_t old = atomicAnd(&ur[w], ~bit);
      if ((old & ~bit) == 0u) atomicAnd(&urs[w >> 5], ~(1u << (w & 31)));
    }
  }
  // lowest set bit of a bit map with summary `sm` (s32 words), -1 if none;
  // every lane gets the answer
  __device__ __forceinline__ int lowest(const uint32_t *bm, const uint32_t *sm, int lane) const {
    for (int base = 0; base < s32; base += 32) {
      const uint32_t sv = base + lane < s32 ? sm[base + lane] : 0u;
      const uint32_t nz = __ballot_sync(FULL, sv != 0u);
      if (nz) {
        const int l = __ffs(nz) - 1;
        const uint32_t s0 = __shfl_sync(FULL, sv, l);
        const int w = (base + l) * 32 + __ffs(s0) - 1;
        return w * 32 + __ffs(bm[w]) - 1;
      }
    }
    return -1;
  }
};

// What a search does with the levels above the cut of the budgeted split
// search.  Default: nothing (the canonical search of the whole tree).
//   track:  first phase -- the subtree (row places of the first `cut`
//           levels) of each leaf taken is kept in `sub_out`;
//   forced: one subtree -- at level i < cut only the row at place digit i of
//           `prefix` (base k, most significant first) is taken, the search
//           never backtracks above the cut, and the incumbent starts at
//           `init_best` (a leaf must cost less); `replay` stops at the first
//           leaf taken.
struct SplitSpec {
  int cut = 0;
  bool track = false, forced = false, replay = false;
  uint32_t prefix = 0;
  int32_t init_best = 0x7FFFFFFF;
  uint32_t sub_out = 0;   // track: subtree of the incumbent's leaf
  bool found = false;     // forced: a leaf was taken
};

// FT: field type of the activeRows bitset (uint8_t for k <= 7, uint16_t for
// k = 8); MK: width of the row sort (k for k <= 4, else 8); SM: state and
// read-only block in shared memory.  Each segment's field is written by one
// lane at a time, so covers are plain loads and stores: the cover of row
// (v, c) saves every neighbour's field before clearing bit c, and the undo
// writes the saved fields back.  Next to the bitset, every segment keeps
// 16-bit counts of its conflict and stitch neighbours per mask, updated by
// the same lanes, so the added cost of a segment's rows (Eq. 1) is read in
// one load instead of gathered from its neighbours.
// Instances of at most 32 words of fields go to reg_search below instead.
template <typename FT, int MK, bool SM, typename Team, bool BK = false>
struct Search {
  static constexpr uint32_t FB = 8 * sizeof(FT);    // bits per field
  static constexpr uint32_t FLAG = 1u << (FB - 1);   // column P_v uncovered
  static constexpr uint32_t FMASK = (FB == 8) ? 0xFFu : 0xFFFFu;
  static constexpr int PER_WORD = 4 / (int)sizeof(FT);
  static constexpr int CW = MK <= 4 ? 1 : 2;          // 64-bit count words per segment

  uint4 *lv;          // two uint4 per level
  int32_t *lvx;       // cost of rows 3.. per level (MK entries per level)
  uint64_t *ccnt, *scnt;
  FT *rows;           // activeRows fields
  FT *oldf;           // field of v before its first row was covered
  FT *savf;           // neighbour fields saved by the cover of v's row
  int8_t *x;
  const int2 *ptr;    // {conflict offset, stitch offset} per segment
  const uint16_t *cnbr, *snbr;
  const uint16_t *rank, *order;   // breadth-first rank / segment of each rank
  const int32_t *qptr;            // second bound mode: each segment's cliques
  const uint16_t *qlist;
  uint8_t *qcnt;                  // members of each clique assigned
  int32_t *qlev;                  // per level: cliques its assignment touched
  int nq;
  int n, k;
  int Cc, Cs;
  uint32_t kmask;
  int rule;           // 0: fewest rows, lowest index; 1: single row, else BFS order

  __device__ __forceinline__ static uint64_t one(int c) { return 1ull << (16 * (c & 3)); }
  __device__ __forceinline__ static int lane16(uint64_t w, int c) {
    return (int)((w >> (16 * (c & 3))) & 0xFFFFull);
  }
  Team team;          // the threads searching this instance together
  Buckets bk;         // BK: the column classes (one warp, shared memory)
  // BK, when the room allows (k <= 4 and every degree below 256): the
  // per-mask neighbour counts as 8-bit lanes of one word per segment, and
  // the adjacency offsets as 16-bit offsets from the first segment of each
  // block of 64 (`cob`, `sob`: the blocks' own offsets), in shared memory;
  // a node then reads only its neighbour lists from global memory
  uint32_t *bcc = nullptr, *bsc = nullptr;
  uint16_t *co16 = nullptr, *so16 = nullptr;
  int32_t *cob = nullptr, *sob = nullptr;
  // 8-bit lanes 0..3 of w as the 16-bit lanes of the global count words
  __device__ __forceinline__ static uint64_t widen8(uint32_t w) {
    return (uint64_t)__byte_perm(w, 0u, 0x4140u) | ((uint64_t)__byte_perm(w, 0u, 0x4342u) << 32);
  }
  __device__ __forceinline__ int cls_of(uint32_t f) const {
    return (f & FLAG) ? __popc(f & kmask) : -1;
  }
  // f(i) for i = rank, rank + team size, ... < d
  template <typename F>
  __device__ __forceinline__ void each(int d, int rank, F &&f) const {
    for (int i = rank; i < d; i += team.size()) f(i);
  }

  // count word holding mask c of segment u
  __device__ __forceinline__ uint64_t *cw_of(uint64_t *cnt, int u, int c) const {
    return cnt + (size_t)u * CW + (c >> 2);
  }
  // counts of segment u: mask c_new gains one neighbour, c_old (if >= 0) loses one
  __device__ __forceinline__ void move_count(uint64_t *cnt, int u, int c_new, int c_old) const {
    if (c_old < 0) {
      *cw_of(cnt, u, c_new) += one(c_new);
    } else if (CW == 1 || (c_new >> 2) == (c_old >> 2)) {
      *cw_of(cnt, u, c_new) += one(c_new) - one(c_old);
    } else {
      *cw_of(cnt, u, c_new) += one(c_new);
      *cw_of(cnt, u, c_old) -= one(c_old);
    }
  }

  // First row (v, c) of v's column: save and clear v's field (column P_v
  // and all its rows), clear bit c of every conflict neighbour (column
  // S_{(v,u),c}) saving its field, and count mask c at every neighbour.
  // upre / spre: this lane's first conflict / stitch neighbour when the
  // caller has loaded it already (BK), else -1.
  __device__ __forceinline__ void cover_first(int v, int c, int cb, int dc, int sb, int ds,
                                              int lane, int upre = -1, int spre = -1) const {
    if (lane == 0) {
      const FT fv = rows[v];
      oldf[v] = fv;
      rows[v] = 0;
      x[v] = (int8_t)c;
      if constexpr (BK) {
        bk.move(v, cls_of(fv), -1);
        if (rule) bk.rank_set(ro_ld<SM>(rank + v), false);
      }
    }
    const uint32_t clr = ~(1u << c);
    if constexpr (BK) {
      each(dc, lane, [&](int i) {
        const int u = (i == lane && upre >= 0) ? upre : (int)ro_ld<SM>(cnbr + cb + i);
        const FT f = rows[u];
        savf[cb + i] = f;
        rows[u] = (FT)(f & clr);
        if (bcc) bcc[u] += 1u << (8 * c);
        else move_count(ccnt, u, c, -1);
        bk.move(u, cls_of(f), cls_of(f & clr));
      });
      each(ds, lane, [&](int i) {
        const int u = (i == lane && spre >= 0) ? spre : (int)ro_ld<SM>(snbr + sb + i);
        if (bsc) bsc[u] += 1u << (8 * c);
        else move_count(scnt, u, c, -1);
      });
      team.sync();
    } else {
      each(dc, lane, [&](int i) {
        const int u = ro_ld<SM>(cnbr + cb + i);
        const FT f = rows[u];
        savf[cb + i] = f;
        rows[u] = (FT)(f & clr);
        move_count(ccnt, u, c, -1);
      });
      each(ds, lane, [&](int i) { move_count(scnt, ro_ld<SM>(snbr + sb + i), c, -1); });
      team.sync();
    }
  }

  // Next row (v, c) of the same column, replacing row (v, c_old): every
  // neighbour gets its saved field with bit c cleared.
  __device__ __forceinline__ void switch_row(int v, int c_old, int c, int cb, int dc, int sb,
                                             int ds, int lane) const {
    if (lane == 0) x[v] = (int8_t)c;
    const uint32_t clr = ~(1u << c), clr_old = ~(1u << c_old);
    each(dc, lane, [&](int i) {
      const int u = ro_ld<SM>(cnbr + cb + i);
      const FT f = savf[cb + i];
      rows[u] = (FT)(f & clr);
      if (BK && bcc) bcc[u] += (1u << (8 * c)) - (1u << (8 * c_old));
      else move_count(ccnt, u, c, c_old);
      if constexpr (BK) bk.move(u, cls_of(f & clr_old), cls_of(f & clr));
    });
    each(ds, lane, [&](int i) {
      const int u = ro_ld<SM>(snbr + sb + i);
      if (BK && bsc) bsc[u] += (1u << (8 * c)) - (1u << (8 * c_old));
      else move_count(scnt, u, c, c_old);
    });
    team.sync();
  }

  // Every row of v's column tried (the last was c_last): put v's field and
  // its neighbours back.
  __device__ __forceinline__ void restore(int v, int c_last, int cb, int dc, int sb, int ds,
                                          int lane) const {
    if (lane == 0) {
      const FT fv = oldf[v];
      rows[v] = fv;
      x[v] = -1;
      if constexpr (BK) {
        bk.move(v, -1, cls_of(fv));
        if (rule) bk.rank_set(ro_ld<SM>(rank + v), true);
      }
    }
    const uint32_t clr_last = ~(1u << c_last);
    each(dc, lane, [&](int i) {
      const int u = ro_ld<SM>(cnbr + cb + i);
      const FT f = savf[cb + i];
      rows[u] = f;
      if (BK && bcc) bcc[u] -= 1u << (8 * c_last);
      else *cw_of(ccnt, u, c_last) -= one(c_last);
      if constexpr (BK) bk.move(u, cls_of(f & clr_last), cls_of(f));
    });
    each(ds, lane, [&](int i) {
      const int u = ro_ld<SM>(snbr + sb + i);
      if (BK && bsc) bsc[u] -= 1u << (8 * c_last);
      else *cw_of(scnt, u, c_last) -= one(c_last);
    });
    team.sync();
  }

  __device__ __forceinline__ int run(int lane, int64_t budget, int64_t time_limit_ns,
                                     int8_t *best_mask, int32_t &best_out, int64_t &nodes_out,
                                     int64_t &work_out, SplitSpec &sp,
                                     uint64_t t0 = 0) const {
    int32_t best = sp.forced ? sp.init_best : INF32, g = 0;
    int64_t nodes = 0, work = 0;
    uint32_t work32 = 0;
    int level = 0;
    int status = MPLD_OK;
    // a forced subtree search never backtracks above the cut
    const int floor_level = sp.forced ? sp.cut : 0;
    if (t0 == 0) t0 = globaltimer();
    const uint32_t *rows32 = reinterpret_cast<const uint32_t *>(rows);
    const int nwords = (n + PER_WORD - 1) / PER_WORD;
    int64_t next_check = 1024;
    // m child nodes pruned on entry by their path cost alone, counted as
    // the recursive search would (see reg_search); they add no work
    auto count_pruned = [&](int m) -> bool {
      const int64_t room = budget > 0 ? budget - nodes : (int64_t)m;
      nodes += room < m ? (room > 0 ? room : 0) : (int64_t)m;
      return room < m;
    };
    int untouched = nq;   // cliques of the second bound mode with no member assigned
    // member counts of v's cliques move (the caller keeps `untouched`)
    auto clique_move = [&](int v, int dir) {
      const int q0 = ro_ld<SM>(qptr + v), q1 = ro_ld<SM>(qptr + v + 1);
      for (int i = q0 + lane; i < q1; i += team.size()) {
        const int q = ro_ld<SM>(qlist + i);
        qcnt[q] = (uint8_t)(qcnt[q] + dir);
      }
      team.sync();
    };
    auto untouched_after = [&](int v) -> int {
      const int q0 = ro_ld<SM>(qptr + v), q1 = ro_ld<SM>(qptr + v + 1);
      int left = untouched;
      for (int i = q0 + lane; i - lane < q1; i += team.size())
        left -= (int)team.sum(i < q1 && qcnt[ro_ld<SM>(qlist + i)] == 0);
      return left;
    };
    bool enter = true;
    for (;;) {
      if (enter) {
        // ---- a node: one call of the recursive search ----
        if (budget > 0 && best < INF32 && nodes >= budget) { status = MPLD_BUDGET; break; }
        ++nodes;
        work32 += 2u * (uint32_t)(n - level);
        if (nodes >= next_check) {
          next_check = nodes + 1024;
          work += work32;
          work32 = 0;
          const uint64_t now = team.bcast0(lane == 0 ? globaltimer() : 0);
          if ((int64_t)(now - t0) > time_limit_ns) { status = MPLD_TIMEOUT; break; }
        }
        // column choice: min over uncovered P_v of popc(activeRows & colRows[P_v]),
        // PER_WORD fields per 32-bit load.  Rule 0 keys (count, v); rule 1
        // (the paper's) keys single-row columns by v ahead of all others,
        // which go by breadth-first rank.
        uint32_t key = 0xFFFFFFFFu, z = 0;
        if (BK) {
          // the column classes: the first non-empty one's lowest segment
          // (rule 0), or a single-row column, else the lowest uncovered
          // breadth-first rank (rule 1); z = the dead columns
          int m0 = -1;
          for (int m = k; m >= 0; --m)
            if (*(volatile int32_t *)&bk.cnt[m] > 0) m0 = m;
          if (m0 >= 0) {
            if (rule == 0) {
              key = ((uint32_t)m0 << 16) | (uint32_t)bk.lowest_in(m0, lane);
            } else if (*(volatile int32_t *)&bk.cnt[1] > 0) {
              key = (uint32_t)bk.lowest_in(1, lane);
            } else {
              key = 0x10000u | (uint32_t)bk.lowest(bk.ur, bk.urs, lane);
            }
          }
          z = (uint32_t)*(volatile int32_t *)&bk.cnt[0];
        } else if (rule == 0) {
          // four words per thread in flight: an instance whose state is in
          // global memory waits on one load latency per four words
          const int ts = team.size();
          for (int wb = lane; wb < nwords; wb += 4 * ts) {
            uint32_t wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) wv[u] = wb + ts * u < nwords ? rows32[wb + ts * u] : 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int j = 0; j < PER_WORD; ++j) {
                const uint32_t f = (wv[u] >> (FB * j)) & FMASK;
                const uint32_t kv = (f & FLAG)
                                        ? ((uint32_t)__popc(f & kmask) << 16) |
                                              (uint32_t)((wb + ts * u) * PER_WORD + j)
                                        : 0xFFFFFFFFu;
                key = min(key, kv);
                z += kv <= 0xFFFFu;  // uncovered column with no active row
              }
          }
        } else {
          const int ts = team.size();
          for (int wb = lane; wb < nwords; wb += 4 * ts) {
            uint32_t wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) wv[u] = wb + ts * u < nwords ? rows32[wb + ts * u] : 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int j = 0; j < PER_WORD; ++j) {
                const uint32_t f = (wv[u] >> (FB * j)) & FMASK;
                const uint32_t seg = (uint32_t)((wb + ts * u) * PER_WORD + j);
                const uint32_t cnt = (uint32_t)__popc(f & kmask);
                uint32_t kv = 0xFFFFFFFFu;
                if (f & FLAG) kv = cnt == 1 ? seg : 0x10000u | (uint32_t)ro_ld<SM>(rank + seg);
                key = min(key, kv);
                z += (f & FLAG) && cnt == 0;
              }
          }
        }
        if (!BK) key = team.min(key);
        if (key == 0xFFFFFFFFu) {
          // leaf: every primary column covered
          if (g < best) {
            best = g;
            sp.found = true;
            if (best_mask)
              for (int i = lane; i < n; i += team.size()) best_mask[i] = x[i];
            if (sp.track) {
              // the row place taken at each level above the cut (rows tried - 1)
              uint32_t sub = 0;
              for (int i = 0; i < sp.cut; ++i) sub = sub * (uint32_t)k + ((lv[2 * i].y >> 16) - 1u);
              sp.sub_out = sub;
            }
            if (best == 0 || sp.replay) break;
          }
          enter = false;
          continue;
        }
        if (best < INF32) {
          // the bound needs the number of uncovered columns with no active
          // row; under rule 0 there is one only when the minimum count is 0
          if (!BK) z = (rule != 0 || (key >> 16) == 0) ? team.sum(z) : 0u;
          if ((int64_t)g + (int64_t)Cc * (z + (uint32_t)untouched) >= best) { enter = false; continue; }
        }
        const int v = (rule == 0 || key < 0x10000u) ? (int)(key & 0xFFFFu)
                                                     : (int)ro_ld<SM>(order + (key & 0xFFFFu));
        // added cost of each row (v, c) against the current assignment (Eq. 1)
        int cb, dc, sb, ds;
        int upre = -1, spre = -1;
        uint64_t cc0, sc0, cc1 = 0ull, sc1 = 0ull;
        if (BK && bcc) {
          const int v1 = v + 1;
          cb = cob[v >> 6] + (int)co16[v];
          dc = cob[v1 >> 6] + (int)co16[v1] - cb;
          sb = sob[v >> 6] + (int)so16[v];
          ds = sob[v1 >> 6] + (int)so16[v1] - sb;
          cc0 = widen8(bcc[v]);
          sc0 = widen8(bsc[v]);
          // the cover below needs v's neighbour lists whichever row it takes:
          // their loads overlap the row costs
          if (lane < dc) upre = (int)ro_ld<SM>(cnbr + cb + lane);
          if (lane < ds) spre = (int)ro_ld<SM>(snbr + sb + lane);
        } else {
          const int2 p0 = ro_ld<SM>(ptr + v), p1 = ro_ld<SM>(ptr + v + 1);
          cc0 = ccnt[(size_t)v * CW];
          sc0 = scnt[(size_t)v * CW];
          if (CW == 2) {
            cc1 = ccnt[(size_t)v * CW + 1];
            sc1 = scnt[(size_t)v * CW + 1];
          }
          cb = p0.x, dc = p1.x - p0.x, sb = p0.y, ds = p1.y - p0.y;
        }
        work32 += (uint32_t)(k * (dc + ds) + 5 * (1 + dc));
        int stot = 0;
#pragma unroll
        for (int c = 0; c < MK; ++c) stot += lane16(c < 4 ? sc0 : sc1, c);
        uint32_t keys[MK];
#pragma unroll
        for (int c = 0; c < MK; ++c) {
          const int inc = Cc * lane16(c < 4 ? cc0 : cc1, c) + Cs * (stot - lane16(c < 4 ? sc0 : sc1, c));
          keys[c] = (MK == 8 && c >= k) ? 0xFFFFFFFFu : (((uint32_t)inc << 3) | (uint32_t)c);
        }
        sort_keys<MK>(keys);
        // each child's bound is at least its path cost plus cost_conflict
        // times the cliques untouched once v is assigned
        const int left = nq > 0 ? untouched_after(v) : 0;
        const int32_t floor_c = Cc * left;
        if (level < floor_level) {
          // above the cut of a forced subtree: only the row at the prefix's
          // place is taken; if its child is pruned on entry the subtree ends
          uint32_t pw = 1;
          for (int i = level + 1; i < sp.cut; ++i) pw *= (uint32_t)k;
          const int place = (int)((sp.prefix / pw) % (uint32_t)k);
          uint32_t kp = keys[0];
#pragma unroll
          for (int i = 1; i < MK; ++i) kp = i == place ? keys[i] : kp;
          if (best < INF32 && g + (int32_t)(kp >> 3) + floor_c >= best) {
            if (count_pruned(1)) status = MPLD_BUDGET;
            break;
          }
          uint32_t ord = 0;
#pragma unroll
          for (int i = 0; i < MK; ++i) ord |= (keys[i] & 7u) << (4 * i);
          if (lane == 0) {
            lv[2 * level] = make_uint4((uint32_t)g, (uint32_t)v | ((uint32_t)(place + 1) << 16), ord,
                                       (uint32_t)cb);
            lv[2 * level + 1] = make_uint4((uint32_t)dc | ((uint32_t)ds << 16), (uint32_t)sb, 0u, 0u);
          }
          cover_first(v, (int)(kp & 7u), cb, dc, sb, ds, lane);
          g += (int32_t)(kp >> 3);
          ++level;
          continue;
        }
        if (best < INF32 && g + (int32_t)(keys[0] >> 3) + floor_c >= best) {
          // rows are in ascending cost: every child is pruned on entry
          if (count_pruned(k)) { status = MPLD_BUDGET; break; }
          enter = false;
          continue;
        }
        uint32_t ord = 0;
#pragma unroll
        for (int i = 0; i < MK; ++i) ord |= (keys[i] & 7u) << (4 * i);
        if (lane == 0) {
          lv[2 * level] = make_uint4((uint32_t)g, (uint32_t)v | (1u << 16), ord, (uint32_t)cb);
          lv[2 * level + 1] = make_uint4((uint32_t)dc | ((uint32_t)ds << 16), (uint32_t)sb,
                                         MK > 1 ? keys[1] >> 3 : 0u, MK > 2 ? keys[MK > 2 ? 2 : 0] >> 3 : 0u);
#pragma unroll
          for (int i = 3; i < MK; ++i)
            if (i < k) lvx[level * MK + i] = (int32_t)(keys[i] >> 3);
        }
        cover_first(v, (int)(ord & 7u), cb, dc, sb, ds, lane, upre, spre);
        if (nq > 0) {
          if (lane == 0) qlev[level] = untouched - left;
          clique_move(v, 1);
          untouched = left;
        }
        g += (int32_t)(keys[0] >> 3);
        ++level;
        continue;
      }
      // ---- backtrack: next row of the level above, or undo its column ----
      if (level <= floor_level) break;
      --level;
      const uint4 r0 = lv[2 * level], r1 = lv[2 * level + 1];
      team.sync();   // read by every thread before the first rewrites it below
      const int v = (int)(r0.y & 0xFFFFu);
      const int nxt = (int)(r0.y >> 16);
      const int cb = (int)r0.w, dc = (int)(r1.x & 0xFFFFu), sb = (int)r1.y, ds = (int)(r1.x >> 16);
      const int c_last = (int)((r0.z >> (4 * (nxt - 1))) & 7u);
      if (nxt >= k) {  // every row of this column tried
        restore(v, c_last, cb, dc, sb, ds, lane);
        if (nq > 0) {
          clique_move(v, -1);
          untouched += qlev[level];
        }
        continue;
      }
      const int c = (int)((r0.z >> (4 * nxt)) & 7u);
      g = (int32_t)r0.x + (nxt == 1 ? (int32_t)r1.z : nxt == 2 ? (int32_t)r1.w : lvx[level * MK + nxt]);
      if (best < INF32 && g + Cc * untouched >= best) {
        // this row and the ones after it: children pruned on entry
        if (count_pruned(k - nxt)) { status = MPLD_BUDGET; break; }
        restore(v, c_last, cb, dc, sb, ds, lane);
        if (nq > 0) {
          clique_move(v, -1);
          untouched += qlev[level];
        }
        continue;
      }
      work32 += 5u * (uint32_t)(1 + dc);
      if (lane == 0) lv[2 * level].y = (uint32_t)v | ((uint32_t)(nxt + 1) << 16);
      switch_row(v, c_last, c, cb, dc, sb, ds, lane);
      ++level;
      enter = true;
    }
    best_out = best;
    nodes_out = nodes;
    work_out = work + work32;
    return status;
  }
};

// Budgeted split search, first phase: an instance that stopped on its
// per-search budget goes on a hard list (the lanes' for instances the
// per-lane search takes, else the warps'), with a fresh context whose key is
// its incumbent (cost << 32 | subtree of the incumbent's leaf).  Lane 0 only.
__device__ __forceinline__ void split_enlist(const LaunchArgs &a, const InstDesc &d, int32_t best,
                                             uint32_t sub) {
  const int kind = split_list_of(d.n, d.k);
  const int j = atomicAdd(a.hard + kind, 1);
  a.hard[4 + kind * a.hard_cap + j] = d.idx;
  ParCtx *c = (ParCtx *)(a.par_buf + (size_t)d.idx * 64);
  c->key = ((unsigned long long)(uint32_t)best << 32) | sub;
  c->nodes = 0;
  c->work = 0;
  c->next = 0;
  c->timed_out = 0;
  c->done = 0;
  c->pad = 0;
  c->t0 = 0;
}

// ---- register-resident search (n <= 32 words of fields) -------------------
//
// The same search as Search above, for instances whose fields fit one
// 32-bit word per lane: lane l holds the fields of segments l*P .. l*P+P-1
// (P = 4 byte fields, or 2 for k = 8) in a register `w`, their masks in `xw`
// (one byte per segment, 0xFF = none), and, per mask c, the number of their
// conflict and stitch neighbours holding c (`cc[c]`, `sc[c]`, one byte per
// segment).  The adjacency is a bit matrix: adj[v*32 + l] says which of lane
// l's segments neighbour v.  Per node:
//   * column choice: popc of the lane's P fields, one __reduce_min_sync;
//   * row costs (Eq. 1): the lane that holds v packs v's counts (byte
//     permutes) and one shuffle per kind hands them to the warp;
//   * cover of row (v, c): w &= ~(neighbour bits << c), the counts of mask c
//     gain v's neighbours, and the owner lane clears v's field.  The undo
//     record per lane is 16 bits: which neighbour fields had row c active,
//     and the lane's conflict and stitch neighbour bits of v.
// No field, count or neighbour list is read from memory on the way down.

// bit j of a nibble -> bit 0 of field j (8-bit fields: bytes; 16-bit: halves)
template <int FB> __device__ __forceinline__ uint32_t spread_bits(uint32_t b) {
  if constexpr (FB == 8) return (b * 0x00204081u) & 0x01010101u;
  else return (b & 1u) | ((b & 2u) << 15);
}
// inverse of spread_bits for words holding only bit 0 of each field
template <int FB> __device__ __forceinline__ uint32_t gather_bits(uint32_t t) {
  if constexpr (FB == 8) return (t * 0x10204080u) >> 28;
  else return (t | (t >> 15)) & 3u;
}

// byte j (uniform) of four count words, packed as bytes 0..3
__device__ __forceinline__ uint32_t pick_bytes(uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                               uint32_t sel) {
  return __byte_perm(__byte_perm(a, b, sel), __byte_perm(c, d, sel), 0x5410u);
}

template <typename FT, int MK, int RULE, bool CQ>
__device__ __forceinline__ void reg_search(const InstDesc &d, uint8_t *base, const LaunchArgs &a,
                                           int lane) {
  constexpr uint32_t FB = 8 * sizeof(FT);
  constexpr uint32_t FLAG = 1u << (FB - 1);
  constexpr uint32_t FMASK = (FB == 8) ? 0xFFu : 0xFFFFu;
  constexpr int P = 4 / (int)sizeof(FT);
  constexpr int RS = MK <= 4 ? 8 : 12;   // words per level record
  constexpr int NC = MK;                 // count registers per kind (one per mask)
  const int n = d.n, k = d.k;
  const int Cc = d.cost_conflict, Cs = d.cost_stitch;
  const uint32_t kmask = (1u << k) - 1u;
  const int nq = CQ ? d.nq : 0;   // CQ: instances built with the clique bound
  const RegLayout R = reg_layout(n, k, nq);
  uint8_t *adj = base + R.adj;
  uint32_t *deg = (uint32_t *)(base + R.deg);
  uint32_t *rec = (uint32_t *)(base + R.rec);
  uint16_t *sav = (uint16_t *)(base + R.sav);
  uint16_t *qptr = (uint16_t *)(base + R.qptr);
  uint16_t *qlist = (uint16_t *)(base + R.qlist);
  uint8_t *qcnt = base + R.qcnt;

  // adjacency bit matrix and degrees, from the read-only block (via L2)
  {
    const RoLayout Q = ro_layout(n, d.ne2, d.ns2);
    const int2 *ptr = (const int2 *)(d.ro + Q.ptr);
    const uint16_t *cnbr = (const uint16_t *)(d.ro + Q.cnbr);
    const uint16_t *snbr = (const uint16_t *)(d.ro + Q.snbr);
    uint32_t *adj32 = (uint32_t *)adj;
    for (int i = lane; i < 8 * n; i += 32) adj32[i] = 0u;
    __syncwarp();
    for (int v = lane; v < n; v += 32) {
      const int2 p0 = __ldcg(ptr + v), p1 = __ldcg(ptr + v + 1);
      uint8_t *row = adj + v * 32;
      for (int i = p0.x; i < p1.x; ++i) {
        const int u = __ldcg(cnbr + i);
        row[u / P] |= (uint8_t)(1u << (u % P));
      }
      for (int i = p0.y; i < p1.y; ++i) {
        const int u = __ldcg(snbr + i);
        row[u / P] |= (uint8_t)(1u << (4 + u % P));
      }
      deg[v] = (uint32_t)(p1.x - p0.x) | ((uint32_t)(p1.y - p0.y) << 16);
    }
  }
  if (nq > 0) {
    // the second bound mode's cliques: each segment's list, and per clique
    // the number of members assigned
    const RoLayout Q = ro_layout(n, d.ne2, d.ns2, nq * (k + 1));
    const int32_t *gq = (const int32_t *)(d.ro + Q.qptr);
    const uint16_t *gl = (const uint16_t *)(d.ro + Q.qlist);
    for (int i = lane; i <= n; i += 32) qptr[i] = (uint16_t)__ldcg(gq + i);
    for (int i = lane; i < nq * (k + 1); i += 32) qlist[i] = __ldcg(gl + i);
    for (int i = lane; i < nq; i += 32) qcnt[i] = 0;
  }
  // every row active, every primary column uncovered, no mask assigned
  uint32_t w = 0u, xw = 0xFFFFFFFFu, rk = 0u;
  uint32_t cc[NC], sc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) cc[c] = sc[c] = 0u;
  {
    const RoLayout Q = ro_layout(n, d.ne2, d.ns2);
    const uint16_t *rank = (const uint16_t *)(d.ro + Q.rank);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const int s = lane * P + j;
      if (s < n) {
        w |= (kmask | FLAG) << (FB * j);
        if (RULE) rk |= (uint32_t)__ldcg(rank + s) << (8 * j);
      }
    }
  }
  __syncwarp();

  int32_t best = INF32, g = 0;
  int64_t nodes = 0, work = 0;
  uint32_t work32 = 0;
  int level = 0;
  int status = MPLD_OK;
  int64_t budget = a.budget;
  const int64_t time_limit_ns = a.time_limit_ns;
  // budgeted split search, first phase: this search's share of the budget,
  // and the subtree (row places of the first cut_d levels) of each leaf taken
  int cut_d = 0;
  uint32_t cut_s = 1, best_sub = 0;
  if (a.split) {
    split_cut(n, k, cut_d, cut_s);
    budget = split_search_budget(a.budget, cut_s);
  }
  const uint64_t t0 = globaltimer();
  int64_t next_check = 1024;
  int untouched = nq;   // cliques with no member assigned
  // v assigned (dir = +1) or released (-1): the member counts of its
  // cliques move (the caller keeps `untouched`)
  auto clique_move = [&](int v, int dir) {
    const int q0 = qptr[v], q1 = qptr[v + 1];
    for (int i = q0 + lane; i < q1; i += 32) qcnt[qlist[i]] = (uint8_t)(qcnt[qlist[i]] + dir);
    __syncwarp();
  };
  // m child nodes that are pruned on entry (their path cost alone reaches
  // the incumbent, so neither a cover nor a column scan is needed to know
  // it): counted as the recursive search would, stopping where the node
  // budget does.  They add no work: nothing is computed for them.
  auto count_pruned = [&](int m) -> bool {
    const int64_t room = budget > 0 ? budget - nodes : (int64_t)m;
    nodes += room < m ? (room > 0 ? room : 0) : (int64_t)m;
    return room < m;
  };
  // the counts of mask c gain (add) or lose the neighbours spread in cb8 /
  // sb8 (bytes never go below zero, so a wrapped add is a bytewise one)
  auto move_counts = [&](int c, uint32_t cb8, uint32_t sb8, bool add) {
    const uint32_t dcw = add ? cb8 : 0u - cb8, dsw = add ? sb8 : 0u - sb8;
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const bool hit = m == c;
      cc[m] += hit ? dcw : 0u;
      sc[m] += hit ? dsw : 0u;
    }
  };
  // untouched cliques once v is assigned (v's untouched cliques drop out)
  auto untouched_after = [&](int v) -> int {
    const int q0 = qptr[v], q1 = qptr[v + 1];
    int left = untouched;
    for (int i = q0 + lane; i - lane < q1; i += 32)
      left -= __popc(__ballot_sync(FULL, i < q1 && qcnt[qlist[i]] == 0));
    return left;
  };
  bool enter = true;
  for (;;) {
    if (enter) {
      // ---- a node: one call of the recursive search ----
      if (budget > 0 && best < INF32 && nodes >= budget) { status = MPLD_BUDGET; break; }
      ++nodes;
      work32 += 2u * (uint32_t)(n - level);
      if (nodes >= next_check) {
        next_check = nodes + 1024;
        work += work32;
        work32 = 0;
        uint64_t now = lane == 0 ? globaltimer() : 0;
        now = __shfl_sync(FULL, now, 0);
        if ((int64_t)(now - t0) > time_limit_ns) { status = MPLD_TIMEOUT; break; }
      }
      // column choice.  Rule 0 keys (count, v); rule 1 keys single-row
      // columns by v ahead of all others, which go by breadth-first rank.
      uint32_t key = 0xFFFFFFFFu;
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const uint32_t f = (w >> (FB * j)) & FMASK;
        const uint32_t cnt = (uint32_t)__popc(f & kmask);
        const uint32_t sg = (uint32_t)(lane * P + j);
        uint32_t kv;
        if constexpr (RULE == 0) kv = (cnt << 8) | sg;
        else kv = cnt == 1 ? sg : (0x10000u | (((rk >> (8 * j)) & 0xFFu) << 8) | sg);
        kv = (f & FLAG) ? kv : 0xFFFFFFFFu;
        key = min(key, kv);
      }
      key = __reduce_min_sync(FULL, key);
      if (key == 0xFFFFFFFFu) {
        // leaf: every primary column covered
        if (g < best) {
          best = g;
#pragma unroll
          for (int j = 0; j < P; ++j)
            if (lane * P + j < n) d.mask[lane * P + j] = (int8_t)((xw >> (8 * j)) & 0xFFu);
          if (cut_d > 0) {
            // the row place taken at each level above the cut (next row - 1)
            uint32_t sub = 0;
            for (int i = 0; i < cut_d; ++i) sub = sub * (uint32_t)k + (((rec[i * RS] >> 8) & 0xFu) - 1u);
            best_sub = sub;
          }
          if (best == 0) break;
        }
        enter = false;
        continue;
      }
      if (best < INF32) {
        // uncovered columns with no active row; under rule 0 there is one
        // only when the minimum count is 0, so only then are they counted
        uint32_t z = 0;
        if (RULE != 0 || key < 0x100u) {
#pragma unroll
          for (int j = 0; j < P; ++j) {
            const uint32_t f = (w >> (FB * j)) & FMASK;
            z += (f & FLAG) && (f & kmask) == 0;
          }
          z = __reduce_add_sync(FULL, z);
        }
        if ((int64_t)g + (int64_t)Cc * (z + (uint32_t)untouched) >= best) { enter = false; continue; }
      }
      const int v = (int)(key & 0xFFu);
      const int jv = v % P, src = v / P;
      // the lane's neighbour bits of v (for the cover), loaded while the
      // owner's counts travel
      const uint32_t ab = adj[v * 32 + lane];
      const uint32_t dd = deg[v];
      // v's neighbours per mask (Eq. 1 row costs): one byte per mask
      const uint32_t sel = (uint32_t)jv | ((uint32_t)(jv + 4) << 4);
      // masks past NC have no register and count as zero
      auto ccr = [&](int m) -> uint32_t { return m < NC ? cc[m < NC ? m : 0] : 0u; };
      auto scr = [&](int m) -> uint32_t { return m < NC ? sc[m < NC ? m : 0] : 0u; };
      uint32_t cw0 = pick_bytes(ccr(0), ccr(1), ccr(2), ccr(3), sel);
      uint32_t sw0 = pick_bytes(scr(0), scr(1), scr(2), scr(3), sel);
      uint32_t cw1 = 0u, sw1 = 0u;
      if constexpr (NC == 8) {
        cw1 = pick_bytes(ccr(4), ccr(5), ccr(6), ccr(7), sel);
        sw1 = pick_bytes(scr(4), scr(5), scr(6), scr(7), sel);
      }
      cw0 = __shfl_sync(FULL, cw0, src);
      sw0 = __shfl_sync(FULL, sw0, src);
      if constexpr (NC == 8) {
        cw1 = __shfl_sync(FULL, cw1, src);
        sw1 = __shfl_sync(FULL, sw1, src);
      }
      const int stot = (int)(((sw0 * 0x01010101u) >> 24) + ((sw1 * 0x01010101u) >> 24));
      uint32_t keys[MK];
      uint32_t oldf = FLAG;   // v's field: row c active iff no conflict neighbour holds c
#pragma unroll
      for (int c = 0; c < MK; ++c) {
        const uint32_t cwd = c < 4 ? cw0 : cw1, swd = c < 4 ? sw0 : sw1;
        const int sh = 8 * (c & 3);
        const int ncf = (int)((cwd >> sh) & 0xFFu);
        const int inc = Cc * ncf + Cs * (stot - (int)((swd >> sh) & 0xFFu));
        keys[c] = (MK == 8 && c >= k) ? 0xFFFFFFFFu : (((uint32_t)inc << 3) | (uint32_t)c);
        if (c < k && ncf == 0) oldf |= 1u << c;
      }
      sort_keys<MK>(keys);
      // every child's bound is at least its path cost plus cost_conflict
      // times the cliques still untouched once v is assigned
      const int left = nq > 0 ? untouched_after(v) : 0;
      const int32_t floor_c = Cc * left;
      if (best < INF32 && g + (int32_t)(keys[0] >> 3) + floor_c >= best) {
        // rows are in ascending cost: every child is pruned on entry
        if (count_pruned(k)) { status = MPLD_BUDGET; break; }
        enter = false;
        continue;
      }
      work32 += (uint32_t)(k * (int)((dd & 0xFFFFu) + (dd >> 16)) + 5 * (1 + (int)(dd & 0xFFFFu)));
      if (level >= n) {
        // unreachable: each level covers one of the n columns (a guard for
        // the per-level arrays)
        if (lane == 0) atomicExch(a.err, MPLD_E_STATE);
        break;
      }
      // level record: {v | next row << 8 | v's field << 12, path cost,
      // degrees, cliques v touched, sorted row keys}
      if (lane == 0) {
        uint4 *r4 = (uint4 *)(rec + level * RS);
        r4[0] = make_uint4((uint32_t)v | (1u << 8) | (oldf << 12), (uint32_t)g, dd,
                           (uint32_t)(untouched - left));
        r4[1] = make_uint4(keys[0], MK > 1 ? keys[MK > 1 ? 1 : 0] : 0u,
                           MK > 2 ? keys[MK > 2 ? 2 : 0] : 0u, MK > 3 ? keys[MK > 3 ? 3 : 0] : 0u);
        if constexpr (MK == 8) r4[2] = make_uint4(keys[4 % MK], keys[5 % MK], keys[6 % MK], keys[7 % MK]);
      }
      // cover row (v, c): bit c of v's conflict neighbours, and v's field
      const int c = (int)(keys[0] & 7u);
      const uint32_t cb = ab & 0xFu, sb = ab >> 4;
      const uint32_t spc = spread_bits<FB>(cb);
      sav[level * 32 + lane] = (uint16_t)(gather_bits<FB>((w >> c) & spc) | (cb << 4) | (sb << 8));
      w &= ~(spc << c);
      move_counts(c, spread_bits<8>(cb), spread_bits<8>(sb), true);
      if (lane == src) {
        w &= ~(FMASK << (FB * jv));
        xw = (xw & ~(0xFFu << (8 * jv))) | ((uint32_t)c << (8 * jv));
      }
      if (nq > 0) {
        clique_move(v, 1);
        untouched = left;
      }
      g += (int32_t)(keys[0] >> 3);
      ++level;
      __syncwarp();
      continue;
    }
    // ---- backtrack: next row of the level above, or undo its column ----
    if (level == 0) break;
    --level;
    const uint32_t *r = rec + level * RS;
    const uint4 r0 = *(const uint4 *)r, r1 = *(const uint4 *)(r + 4);
    uint4 r2 = make_uint4(0u, 0u, 0u, 0u);
    if constexpr (MK == 8) r2 = *(const uint4 *)(r + 8);
    const uint32_t sv = sav[level * 32 + lane];
    // every lane has read the record before lane 0 rewrites its row index
    // below (the paths that led here may have left the warp diverged)
    __syncwarp();
    const int v = (int)(r0.x & 0xFFu);
    const int nxt = (int)((r0.x >> 8) & 0xFu);
    const int jv = v % P, src = v / P;
    // sorted row keys sit in words 4 .. 4+MK-1 of the record
    auto key_at = [&](int i) -> uint32_t {
      const uint32_t lo = i == 0 ? r1.x : i == 1 ? r1.y : i == 2 ? r1.z : r1.w;
      const uint32_t hi = i == 4 ? r2.x : i == 5 ? r2.y : i == 6 ? r2.z : r2.w;
      return i < 4 ? lo : hi;
    };
    const uint32_t klast = key_at(nxt - 1), knext = key_at(nxt < MK ? nxt : MK - 1);
    const int cl = (int)(klast & 7u);
    const uint32_t cb = (sv >> 4) & 0xFu, sb = sv >> 8;
    const uint32_t spc = spread_bits<FB>(cb);
    const uint32_t cb8 = spread_bits<8>(cb), sb8 = spread_bits<8>(sb);
    // take back the last row: its neighbours regain row bit cl, the counts
    // of mask cl lose v
    w |= spread_bits<FB>(sv & 0xFu) << cl;
    move_counts(cl, cb8, sb8, false);
    bool last = nxt >= k;
    if (!last && best < INF32 &&
        (int32_t)r0.y + (int32_t)(knext >> 3) + Cc * untouched >= best) {
      // this row and the ones after it cost at least as much: their nodes
      // are pruned on entry, so count them and undo the column
      if (count_pruned(k - nxt)) { status = MPLD_BUDGET; break; }
      last = true;
    }
    if (last) {
      // every row of this column tried: v's field and mask come back
      if (lane == src) {
        w |= (r0.x >> 12) << (FB * jv);
        xw |= 0xFFu << (8 * jv);
      }
      if (nq > 0) {
        clique_move(v, -1);
        untouched += (int)r0.w;   // the cliques v's assignment had touched
      }
      continue;
    }
    const int c = (int)(knext & 7u);
    g = (int32_t)r0.y + (int32_t)(knext >> 3);
    work32 += 5u * (1u + (r0.z & 0xFFFFu));
    sav[level * 32 + lane] = (uint16_t)(gather_bits<FB>((w >> c) & spc) | (sv & 0xFF0u));
    if (lane == 0) rec[level * RS] = (r0.x & ~0xF00u) | ((uint32_t)(nxt + 1) << 8);
    w &= ~(spc << c);
    move_counts(c, cb8, sb8, true);
    if (lane == src) xw = (xw & ~(0xFFu << (8 * jv))) | ((uint32_t)c << (8 * jv));
    ++level;
    enter = true;
    __syncwarp();
  }
  if (lane == 0) {
    d.res->cost = best == INF32 ? INT64_MAX : (int64_t)best;
    d.res->nodes = nodes;
    d.res->status = status;
    d.res->sub = (int32_t)best_sub;
    d.res->work = work + work32;
    if (a.split && status == MPLD_BUDGET) split_enlist(a, d, best, best_sub);
  }
  __syncwarp();
}

// ---- parallel exact search: the warps of a CTA split one instance --------
//
// For an exact search (no node budget) of an instance of at most 32 field
// words.  The canonical tree is cut at depth D into k^D subtrees, numbered in
// depth-first order: subtree s takes, at level i, the row whose place in the
// ascending (cost, mask) order is digit i of s in base k.  Warps take
// subtrees from a counter and search them as reg_search does.  They share the
// incumbent as one 64-bit key (cost << 32 | subtree): a leaf of cost c in
// subtree s improves it when (c, s) is smaller, so the answer is still the
// first minimum-cost leaf of the whole tree, and a node is pruned when its
// bound reaches cost* plus one if its subtree comes before the incumbent's.
// Node counts depend on when each warp sees a better incumbent.  The G
// warps are those of one CTA (context in shared memory) or of the whole grid
// (context in global memory); a warp re-reads the shared key every 16 nodes.
// Modes:
//   PAR_OWN    each warp keeps its best masks at `bestx` and, at the end, its
//              best key at wkey[gw] and its totals in the context;
//   PAR_QUEUE  totals are published after every subtree, then the subtree
//              is counted done; returns true in the warp that completes the
//              last one (it then recovers the masks by a replay);
//   PAR_REPLAY searches subtree s* alone with the bound of `replay_key`
//              (cost* << 32 | s* + 1, so leaves of cost <= cost* are taken)
//              and writes the first leaf it takes to d.mask: the first leaf
//              of cost cost* in s*, which is the split search's answer.
//   PAR_BUDGET budgeted split search, second phase: searches subtree
//              `it.sub` alone with its own budget and the incumbent of
//              `replay_key` (the first search's), keeps no masks, publishes
//              its best key and totals to the context and counts the subtree
//              done; returns true in the warp that completes the instance's
//              last subtree.
// Item of a call: PAR_BUDGET's subtree and budget; `build` = 0 when the
// warp's slot already holds this instance's adjacency; `split_cut` = the cut
// of the budgeted split search instead of the one for G warps (for
// PAR_BUDGET and its replay).
constexpr int PAR_OWN = 0, PAR_QUEUE = 1, PAR_REPLAY = 2, PAR_BUDGET = 3;
struct ParItem {
  uint32_t sub = 0;
  int64_t budget = 0;
  bool build = true;
  bool split_cut = false;
};

// Subtrees of the split search for G warps: k^D for the first depth D with
// k^D >= 16 G (the trees are skewed), never below the leaves.
__device__ __forceinline__ void par_cut(int n, int k, int G, int &D, uint32_t &ns) {
  D = 0;
  ns = 1;
  while (ns < 16u * (uint32_t)G && D < n) { ns *= (uint32_t)k; ++D; }
}

template <typename FT, int MK, int RULE>
__device__ __noinline__ bool par_search(const InstDesc &d, uint8_t *base, const LaunchArgs &a,
                                        int lane, int gw, int G, ParCtx *ctx,
                                        unsigned long long *wkey, int8_t *bestx, int mode,
                                        unsigned long long replay_key, const ParItem &it) {
  constexpr uint32_t FB = 8 * sizeof(FT);
  constexpr uint32_t FLAG = 1u << (FB - 1);
  constexpr uint32_t FMASK = (FB == 8) ? 0xFFu : 0xFFFFu;
  constexpr int P = 4 / (int)sizeof(FT);
  constexpr int RS = MK <= 4 ? 8 : 12;
  constexpr int NC = MK;
  const int n = d.n, k = d.k;
  const int Cc = d.cost_conflict, Cs = d.cost_stitch;
  const uint32_t kmask = (1u << k) - 1u;
  const RegLayout R = reg_layout(n, k, 0);
  uint8_t *adj = base + R.adj;
  uint32_t *deg = (uint32_t *)(base + R.deg);
  uint32_t *rec = (uint32_t *)(base + R.rec);
  uint16_t *sav = (uint16_t *)(base + R.sav);
  uint32_t rk = 0u;
  {
    const RoLayout Q = ro_layout(n, d.ne2, d.ns2);
    const int2 *ptr = (const int2 *)(d.ro + Q.ptr);
    const uint16_t *cnbr = (const uint16_t *)(d.ro + Q.cnbr);
    const uint16_t *snbr = (const uint16_t *)(d.ro + Q.snbr);
    const uint16_t *rank = (const uint16_t *)(d.ro + Q.rank);
    if (it.build) {
      uint32_t *adj32 = (uint32_t *)adj;
      for (int i = lane; i < 8 * n; i += 32) adj32[i] = 0u;
      __syncwarp();
      for (int v = lane; v < n; v += 32) {
        const int2 p0 = __ldcg(ptr + v), p1 = __ldcg(ptr + v + 1);
        uint8_t *row = adj + v * 32;
        for (int i = p0.x; i < p1.x; ++i) {
          const int u = __ldcg(cnbr + i);
          row[u / P] |= (uint8_t)(1u << (u % P));
        }
        for (int i = p0.y; i < p1.y; ++i) {
          const int u = __ldcg(snbr + i);
          row[u / P] |= (uint8_t)(1u << (4 + u % P));
        }
        deg[v] = (uint32_t)(p1.x - p0.x) | ((uint32_t)(p1.y - p0.y) << 16);
      }
    }
#pragma unroll
    for (int j = 0; j < P; ++j)
      if (RULE && lane * P + j < n) rk |= (uint32_t)__ldcg(rank + lane * P + j) << (8 * j);
  }
  __syncwarp();
  int D;
  uint32_t ns;
  if (it.split_cut) split_cut(n, k, D, ns);
  else par_cut(n, k, G, D, ns);
  int64_t nodes = 0, work = 0, nodes_pub = 0;
  uint32_t work32 = 0;
  bool timed_out = false, last_item = false, budget_hit = false, found = false;
  const int64_t budget = mode == PAR_BUDGET ? it.budget : 0;
  unsigned long long my_key = ~0ull;
  unsigned long long cached = (mode == PAR_REPLAY || mode == PAR_BUDGET) ? replay_key : ~0ull;
  // m children pruned on entry by their path cost: counted as the recursive
  // search counts them, stopping where the node budget does
  auto count_pruned = [&](int m) -> bool {
    const int64_t room = budget > 0 ? budget - nodes : (int64_t)m;
    nodes += room < m ? (room > 0 ? room : 0) : (int64_t)m;
    return room < m;
  };
  // the instance's start: the first warp to arrive sets it, and every warp
  // measures the time limit from there, so the limit bounds the instance's
  // wall time, not each warp's.  The replay, which runs once the instance
  // is done, has a limit of its own.
  uint64_t t0 = 0;
  if (lane == 0) {
    const uint64_t now = globaltimer();
    if (mode == PAR_REPLAY) {
      t0 = now;
    } else {
      const unsigned long long prev = atomicCAS(&ctx->t0, 0ull, (unsigned long long)now);
      t0 = prev != 0ull ? (uint64_t)prev : now;
    }
  }
  t0 = __shfl_sync(FULL, t0, 0);
  int64_t next_check = 1024;
  // the pruning threshold for subtree s: a leaf must cost less than it
  auto threshold = [&](uint32_t s) -> int32_t {
    const unsigned long long key = cached;
    if (key == ~0ull) return INF32;
    const int32_t c = (int32_t)(key >> 32);
    return c + (s < (uint32_t)(key & 0xFFFFFFFFull) ? 1 : 0);
  };
  for (bool first_pass = true;; first_pass = false) {
    uint32_t s = 0;
    if (mode == PAR_REPLAY) {
      if (!first_pass) break;
      s = (uint32_t)(replay_key & 0xFFFFFFFFull) - 1u;
    } else if (mode == PAR_BUDGET) {
      if (!first_pass) break;
      s = it.sub;
    } else {
      if (lane == 0) s = atomicAdd(&ctx->next, 1u);
      s = __shfl_sync(FULL, s, 0);
    }
    if (s >= ns) break;
    // a timed-out warp stops, except in the queue, where it still counts
    // the subtrees it takes as done
    if (timed_out && mode != PAR_QUEUE) break;
    // fresh state for the subtree
    uint32_t w = 0u, xw = 0xFFFFFFFFu;
    uint32_t cc[NC], sc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) cc[c] = sc[c] = 0u;
#pragma unroll
    for (int j = 0; j < P; ++j)
      if (lane * P + j < n) w |= (kmask | FLAG) << (FB * j);
    int32_t g = 0;
    int level = 0;
    auto move_counts = [&](int c, uint32_t cb8, uint32_t sb8, bool add) {
      const uint32_t dcw = add ? cb8 : 0u - cb8, dsw = add ? sb8 : 0u - sb8;
#pragma unroll
      for (int m = 0; m < NC; ++m) {
        const bool hit = m == c;
        cc[m] += hit ? dcw : 0u;
        sc[m] += hit ? dsw : 0u;
      }
    };
    // a leaf of cost g in subtree s
    auto take_leaf = [&]() {
      const unsigned long long key = ((unsigned long long)(uint32_t)g << 32) | s;
      if (lane == 0 && mode != PAR_REPLAY && mode != PAR_BUDGET) atomicMin(&ctx->key, key);
      my_key = key;
      found = true;
      cached = key < cached ? key : cached;
      int8_t *dst = mode == PAR_REPLAY ? d.mask : mode == PAR_BUDGET ? nullptr : bestx;
      if (dst) {
#pragma unroll
        for (int j = 0; j < P; ++j)
          if (lane * P + j < n) dst[lane * P + j] = (int8_t)((xw >> (8 * j)) & 0xFFu);
      }
      __syncwarp();
    };
    const uint32_t prefix = s;   // digit i, most significant first, is the row at level i
    uint32_t top = ns / (uint32_t)k;
    bool enter = true;
    const int floor_level = D;
    if (!timed_out) {
      for (;;) {
        if (enter) {
          if (mode != PAR_REPLAY && mode != PAR_BUDGET && (nodes & 15) == 0) {
            // one read of the shared key for the whole warp
            unsigned long long kk = 0ull;
            if (lane == 0) kk = *(volatile unsigned long long *)&ctx->key;
            kk = __shfl_sync(FULL, kk, 0);
            cached = kk < cached ? kk : cached;
          }
          // the node budget (an incumbent always exists here: the first
          // search's)
          if (budget > 0 && nodes >= budget) {
            budget_hit = true;
            break;
          }
          ++nodes;
          work32 += 2u * (uint32_t)(n - level);
          if (nodes >= next_check) {
            next_check = nodes + 1024;
            work += work32;
            work32 = 0;
            const uint64_t now = __shfl_sync(FULL, lane == 0 ? globaltimer() : 0ull, 0);
            if ((int64_t)(now - t0) > a.time_limit_ns) {
              timed_out = true;
              break;
            }
          }
          const int32_t thr = threshold(s);
          uint32_t key = 0xFFFFFFFFu;
  #pragma unroll
          for (int j = 0; j < P; ++j) {
            const uint32_t f = (w >> (FB * j)) & FMASK;
            const uint32_t cnt = (uint32_t)__popc(f & kmask);
            const uint32_t sg = (uint32_t)(lane * P + j);
            uint32_t kv;
            if constexpr (RULE == 0) kv = (cnt << 8) | sg;
            else kv = cnt == 1 ? sg : (0x10000u | (((rk >> (8 * j)) & 0xFFu) << 8) | sg);
            kv = (f & FLAG) ? kv : 0xFFFFFFFFu;
            key = min(key, kv);
          }
          key = __reduce_min_sync(FULL, key);
          if (key == 0xFFFFFFFFu) {
            // a leaf (always at level n >= D, so below the prefix)
            if (g < thr) {
              take_leaf();
              if (g == 0 || mode == PAR_REPLAY) break;
            }
            if (level <= floor_level) break;
            enter = false;
            continue;
          }
          if (thr < INF32) {
            uint32_t z = 0;
            if (RULE != 0 || key < 0x100u) {
  #pragma unroll
              for (int j = 0; j < P; ++j) {
                const uint32_t f = (w >> (FB * j)) & FMASK;
                z += (f & FLAG) && (f & kmask) == 0;
              }
              z = __reduce_add_sync(FULL, z);
            }
            if ((int64_t)g + (int64_t)Cc * z >= thr) {
              if (level < D) break;
              enter = false;
              continue;
            }
          }
          const int v = (int)(key & 0xFFu);
          const int jv = v % P, src = v / P;
          const uint32_t ab = adj[v * 32 + lane];
          const uint32_t dd = deg[v];
          const uint32_t sel = (uint32_t)jv | ((uint32_t)(jv + 4) << 4);
          auto ccr = [&](int m) -> uint32_t { return m < NC ? cc[m < NC ? m : 0] : 0u; };
          auto scr = [&](int m) -> uint32_t { return m < NC ? sc[m < NC ? m : 0] : 0u; };
          uint32_t cw0 = __shfl_sync(FULL, pick_bytes(ccr(0), ccr(1), ccr(2), ccr(3), sel), src);
          uint32_t sw0 = __shfl_sync(FULL, pick_bytes(scr(0), scr(1), scr(2), scr(3), sel), src);
          uint32_t cw1 = 0u, sw1 = 0u;
          if constexpr (NC == 8) {
            cw1 = __shfl_sync(FULL, pick_bytes(ccr(4), ccr(5), ccr(6), ccr(7), sel), src);
            sw1 = __shfl_sync(FULL, pick_bytes(scr(4), scr(5), scr(6), scr(7), sel), src);
          }
          const int stot = (int)(((sw0 * 0x01010101u) >> 24) + ((sw1 * 0x01010101u) >> 24));
          uint32_t keys[MK];
          uint32_t oldf = FLAG;
  #pragma unroll
          for (int c = 0; c < MK; ++c) {
            const uint32_t cwd = c < 4 ? cw0 : cw1, swd = c < 4 ? sw0 : sw1;
            const int sh = 8 * (c & 3);
            const int ncf = (int)((cwd >> sh) & 0xFFu);
            const int inc = Cc * ncf + Cs * (stot - (int)((swd >> sh) & 0xFFu));
            keys[c] = (MK == 8 && c >= k) ? 0xFFFFFFFFu : (((uint32_t)inc << 3) | (uint32_t)c);
            if (c < k && ncf == 0) oldf |= 1u << c;
          }
          sort_keys<MK>(keys);
          work32 += (uint32_t)(k * (int)((dd & 0xFFFFu) + (dd >> 16)) + 5 * (1 + (int)(dd & 0xFFFFu)));
          // the row to take: the prefix digit above the cut, the first below it
          int first = 0;
          if (level < D) {
            first = (int)((prefix / top) % (uint32_t)k);
            top /= (uint32_t)k;
          }
          uint32_t kf = keys[0];
  #pragma unroll
          for (int i = 1; i < MK; ++i) kf = i == first ? keys[i] : kf;
          if (thr < INF32 && g + (int32_t)(kf >> 3) >= thr) {
            // this row and the ones after it cannot improve: their nodes are
            // pruned on entry (above the cut only the forced row is taken)
            if (count_pruned(level < D ? 1 : k)) budget_hit = true;
            if (level < D || budget_hit) break;
            enter = false;
            continue;
          }
          if (level >= n) break;   // unreachable: each level covers a column
          if (level >= D && lane == 0) {
            uint4 *r4 = (uint4 *)(rec + level * RS);
            r4[0] = make_uint4((uint32_t)v | (1u << 8) | (oldf << 12), (uint32_t)g, dd, 0u);
            r4[1] = make_uint4(keys[0], MK > 1 ? keys[MK > 1 ? 1 : 0] : 0u,
                               MK > 2 ? keys[MK > 2 ? 2 : 0] : 0u, MK > 3 ? keys[MK > 3 ? 3 : 0] : 0u);
            if constexpr (MK == 8) r4[2] = make_uint4(keys[4 % MK], keys[5 % MK], keys[6 % MK], keys[7 % MK]);
          }
          const int c = (int)(kf & 7u);
          const uint32_t cb = ab & 0xFu, sb = ab >> 4;
          const uint32_t spc = spread_bits<FB>(cb);
          if (level >= D)
            sav[level * 32 + lane] = (uint16_t)(gather_bits<FB>((w >> c) & spc) | (cb << 4) | (sb << 8));
          w &= ~(spc << c);
          move_counts(c, spread_bits<8>(cb), spread_bits<8>(sb), true);
          if (lane == src) {
            w &= ~(FMASK << (FB * jv));
            xw = (xw & ~(0xFFu << (8 * jv))) | ((uint32_t)c << (8 * jv));
          }
          g += (int32_t)(kf >> 3);
          ++level;
          __syncwarp();
          continue;
        }
        // backtrack, never above the cut
        if (level <= floor_level) break;
        --level;
        const uint32_t *r = rec + level * RS;
        const uint4 r0 = *(const uint4 *)r, r1 = *(const uint4 *)(r + 4);
        uint4 r2 = make_uint4(0u, 0u, 0u, 0u);
        if constexpr (MK == 8) r2 = *(const uint4 *)(r + 8);
        const uint32_t sv = sav[level * 32 + lane];
        __syncwarp();
        const int v = (int)(r0.x & 0xFFu);
        const int nxt = (int)((r0.x >> 8) & 0xFu);
        const int jv = v % P, src = v / P;
        auto key_at = [&](int i) -> uint32_t {
          const uint32_t lo = i == 0 ? r1.x : i == 1 ? r1.y : i == 2 ? r1.z : r1.w;
          const uint32_t hi = i == 4 ? r2.x : i == 5 ? r2.y : i == 6 ? r2.z : r2.w;
          return i < 4 ? lo : hi;
        };
        const uint32_t klast = key_at(nxt - 1), knext = key_at(nxt < MK ? nxt : MK - 1);
        const int cl = (int)(klast & 7u);
        const uint32_t cb = (sv >> 4) & 0xFu, sb = sv >> 8;
        const uint32_t spc = spread_bits<FB>(cb);
        const uint32_t cb8 = spread_bits<8>(cb), sb8 = spread_bits<8>(sb);
        w |= spread_bits<FB>(sv & 0xFu) << cl;
        move_counts(cl, cb8, sb8, false);
        bool last = nxt >= k;
        const int32_t thr = threshold(s);
        if (!last && thr < INF32 && (int32_t)r0.y + (int32_t)(knext >> 3) >= thr) {
          // this row and the ones after it: children pruned on entry
          if (count_pruned(k - nxt)) {
            budget_hit = true;
            break;
          }
          last = true;
        }
        if (last) {
          if (lane == src) {
            w |= (r0.x >> 12) << (FB * jv);
            xw |= 0xFFu << (8 * jv);
          }
          continue;
        }
        const int c = (int)(knext & 7u);
        g = (int32_t)r0.y + (int32_t)(knext >> 3);
        work32 += 5u * (1u + (r0.z & 0xFFFFu));
        sav[level * 32 + lane] = (uint16_t)(gather_bits<FB>((w >> c) & spc) | (sv & 0xFF0u));
        if (lane == 0) rec[level * RS] = (r0.x & ~0xF00u) | ((uint32_t)(nxt + 1) << 8);
        w &= ~(spc << c);
        move_counts(c, cb8, sb8, true);
        if (lane == src) xw = (xw & ~(0xFFu << (8 * jv))) | ((uint32_t)c << (8 * jv));
        ++level;
        enter = true;
        __syncwarp();
      }
    }
    if (mode == PAR_BUDGET) {
      // publish this subtree's incumbent and totals, then count it done
      uint32_t fin = 0;
      if (lane == 0) {
        if (found) atomicMin(&ctx->key, my_key);
        atomicAdd(&ctx->nodes, (unsigned long long)nodes);
        atomicAdd(&ctx->work, (unsigned long long)(work + work32));
        if (timed_out) atomicExch(&ctx->timed_out, 1u);
        if (budget_hit) atomicExch(&ctx->pad, 1u);
        __threadfence();
        fin = atomicAdd(&ctx->done, 1u) == ns - 1u ? 1u : 0u;
      }
      if (__shfl_sync(FULL, fin, 0)) last_item = true;
    }
    if (mode == PAR_QUEUE) {
      // publish this subtree's totals, then count it done
      work += work32;
      work32 = 0;
      uint32_t fin = 0;
      if (lane == 0) {
        atomicAdd(&ctx->nodes, (unsigned long long)(nodes - nodes_pub));
        atomicAdd(&ctx->work, (unsigned long long)work);
        if (timed_out) atomicExch(&ctx->timed_out, 1u);
        __threadfence();
        fin = atomicAdd(&ctx->done, 1u) == ns - 1u ? 1u : 0u;
      }
      nodes_pub = nodes;
      work = 0;
      if (__shfl_sync(FULL, fin, 0)) last_item = true;
    }
  }
  if (mode == PAR_OWN) {
    if (lane == 0) {
      atomicAdd(&ctx->nodes, (unsigned long long)nodes);
      atomicAdd(&ctx->work, (unsigned long long)(work + work32));
      if (timed_out) atomicExch(&ctx->timed_out, 1u);
      wkey[gw] = my_key;
    }
  }
  __syncwarp();
  // the replay reports whether it took its leaf
  return mode == PAR_REPLAY ? found : last_item;
}

// par_search for the instance's field width, mask count and column rule.
__device__ __noinline__ bool par_dispatch(const InstDesc &d, uint8_t *base, const LaunchArgs &a,
                                          int lane, int gw, int G, ParCtx *ctx,
                                          unsigned long long *wkey, int8_t *bestx, int mode,
                                          unsigned long long replay_key,
                                          const ParItem &it = ParItem{}) {
#define MPLD_PAR(FT, MK)                                                                        \
  return a.rule ? par_search<FT, MK, 1>(d, base, a, lane, gw, G, ctx, wkey, bestx, mode, replay_key, it) \
                : par_search<FT, MK, 0>(d, base, a, lane, gw, G, ctx, wkey, bestx, mode, replay_key, it)
  if (d.k == 3) { MPLD_PAR(uint8_t, 3); }
  if (d.k == 4) { MPLD_PAR(uint8_t, 4); }
  if (d.k == 2) { MPLD_PAR(uint8_t, 2); }
  if (d.k <= 7) { MPLD_PAR(uint8_t, 8); }
  MPLD_PAR(uint16_t, 8);
#undef MPLD_PAR
}

// Initialise the state at `base` and search.  SM says at compile time
// whether `base` and `ro` point into shared memory.
template <typename FT, int MK, bool SM, typename Team, bool BK = false>
__device__ __forceinline__ void run_in(const InstDesc &d, uint8_t *base, const uint8_t *ro,
                                       const LaunchArgs &a, const Team &team,
                                       uint8_t *bk_mem = nullptr, uint32_t bk_room = 0) {
  using S = Search<FT, MK, SM, Team, BK>;
  const int lane = team.rank;
  const int ts = team.size();
  const int n = d.n;
  const StateLayout L = state_layout(n, d.ne2, d.k, d.nq);
  const RoLayout R = ro_layout(n, d.ne2, d.ns2, d.nq * (d.k + 1));
  S s;
  s.team = team;
  s.lv = (uint4 *)(base + L.lv);
  s.lvx = (int32_t *)(base + L.lvx);
  s.ccnt = (uint64_t *)(base + L.ccnt);
  s.scnt = (uint64_t *)(base + L.scnt);
  s.rows = (FT *)(base + L.rows);
  s.oldf = (FT *)(base + L.oldf);
  s.savf = (FT *)(base + L.savf);
  s.x = (int8_t *)(base + L.x);
  s.ptr = (const int2 *)(ro + R.ptr);
  s.cnbr = (const uint16_t *)(ro + R.cnbr);
  s.snbr = (const uint16_t *)(ro + R.snbr);
  s.rank = (const uint16_t *)(ro + R.rank);
  s.order = (const uint16_t *)(ro + R.order);
  s.qptr = (const int32_t *)(ro + R.qptr);
  s.qlist = (const uint16_t *)(ro + R.qlist);
  s.qcnt = base + L.qcnt;
  s.qlev = (int32_t *)(base + L.qlev);
  s.nq = d.nq;
  for (int i = lane; i < d.nq; i += ts) s.qcnt[i] = 0;
  s.rule = a.rule;
  s.n = n;
  s.k = d.k;
  s.Cc = d.cost_conflict;
  s.Cs = d.cost_stitch;
  s.kmask = (1u << d.k) - 1u;
  // initial state: every row active, every primary column uncovered, no
  // neighbour holds a mask; fields past n (word padding) stay zero
  const FT init = (FT)(s.kmask | S::FLAG);
  const int nfields = ((n + S::PER_WORD - 1) / S::PER_WORD) * S::PER_WORD;
  for (int i = lane; i < nfields; i += ts) s.rows[i] = i < n ? init : (FT)0;
  for (int i = lane; i < n; i += ts) s.x[i] = -1;
  for (int i = lane; i < n * S::CW; i += ts) {
    s.ccnt[i] = 0;
    s.scnt[i] = 0;
  }
  if constexpr (BK) {
    s.bk.carve(bk_mem, n, d.k);
    s.bk.init(n, lane);
    // the fields and masks too, when the room allows: the column choice and
    // the covers then touch no global memory for them
    const uint32_t fb = align16((uint32_t)sizeof(FT) * (uint32_t)nfields);
    const uint32_t at = align16(bucket_bytes(n, d.k));
    uint32_t off = at + 2u * fb + align16((uint32_t)n);
    if (off <= bk_room) {
      s.rows = (FT *)(bk_mem + at);
      s.oldf = (FT *)(bk_mem + at + fb);
      s.x = (int8_t *)(bk_mem + at + 2u * fb);
      for (int i = lane; i < nfields; i += ts) s.rows[i] = i < n ? init : (FT)0;
      for (int i = lane; i < n; i += ts) s.x[i] = -1;
      // then the counts and offsets, for k <= 4 when every degree is below
      // 256 (no 8-bit count can overflow, and a block of 64 segments spans
      // fewer than 65,536 list entries)
      const uint32_t cw = align16(4u * (uint32_t)n), ow = align16(2u * (uint32_t)(n + 1));
      const uint32_t bw = align16(4u * (uint32_t)((n >> 6) + 1));
      if (MK <= 4 && off + 2u * (cw + ow + bw) <= bk_room) {
        int dmax = 0;
        for (int i = lane; i < n; i += ts) {
          const int2 a0 = s.ptr[i], a1 = s.ptr[i + 1];
          dmax = max(dmax, max(a1.x - a0.x, a1.y - a0.y));
        }
        dmax = (int)__reduce_max_sync(FULL, (uint32_t)dmax);   // one warp
        if (dmax < 256) {
          s.bcc = (uint32_t *)(bk_mem + off);
          s.bsc = (uint32_t *)(bk_mem + off + cw);
          s.co16 = (uint16_t *)(bk_mem + off + 2u * cw);
          s.so16 = (uint16_t *)(bk_mem + off + 2u * cw + ow);
          s.cob = (int32_t *)(bk_mem + off + 2u * (cw + ow));
          s.sob = (int32_t *)(bk_mem + off + 2u * (cw + ow) + bw);
          for (int i = lane; i < n; i += ts) {
            s.bcc[i] = 0u;
            s.bsc[i] = 0u;
          }
          for (int i = lane; i <= n; i += ts) {
            const int2 q = s.ptr[i], b = s.ptr[i & ~63];
            s.co16[i] = (uint16_t)(q.x - b.x);
            s.so16[i] = (uint16_t)(q.y - b.y);
            if ((i & 63) == 0) {
              s.cob[i >> 6] = q.x;
              s.sob[i >> 6] = q.y;
            }
          }
        }
      }
    }
  }
  team.sync();
  int32_t best = INF32;
  int64_t nodes = 0, work = 0;
  SplitSpec sp;
  int64_t budget = a.budget;
  const bool split = a.split && n <= SPLIT_MAX_N;   // larger: one search, the whole budget
  if (split) {
    // budgeted split search, first phase: this search's share of the budget
    uint32_t S;
    split_cut(n, d.k, sp.cut, S);
    sp.track = sp.cut > 0;
    budget = split_search_budget(a.budget, S);
  }
  const int st = s.run(lane, budget, a.time_limit_ns, d.mask, best, nodes, work, sp);
  if (lane == 0) {
    d.res->cost = best == INF32 ? INT64_MAX : (int64_t)best;
    d.res->nodes = nodes;
    d.res->status = st;
    d.res->sub = (int32_t)sp.sub_out;
    d.res->work = work;
    if (split && st == MPLD_BUDGET) split_enlist(a, d, best, sp.sub_out);
  }
  team.sync();
}

template <typename FT, int MK>
__device__ __noinline__ bool run_instance(const InstDesc &d, uint32_t slot_off, int slot_bytes,
                                             uint64_t *bar, uint32_t &phase, const LaunchArgs &a,
                                             int lane) {
  if (reg_fits(d.n, d.k)) {
    // one call site per memory space, so that each copy knows where its
    // state lives; the column rule and the clique bound are template
    // arguments of the shared-memory copies
    if (slot_bytes > 0 && (int)reg_layout(d.n, d.k, d.nq).bytes <= slot_bytes) {
      uint8_t *slot = g_smem + slot_off;
      if (d.nq > 0) {
        if (a.rule) reg_search<FT, MK, 1, true>(d, slot, a, lane);
        else reg_search<FT, MK, 0, true>(d, slot, a, lane);
      } else {
        if (a.rule) reg_search<FT, MK, 1, false>(d, slot, a, lane);
        else reg_search<FT, MK, 0, false>(d, slot, a, lane);
      }
    } else {
      if (a.rule) reg_search<FT, MK, 1, true>(d, d.scratch, a, lane);
      else reg_search<FT, MK, 0, true>(d, d.scratch, a, lane);
    }
    return true;
  }
  const StateLayout L = state_layout(d.n, d.ne2, d.k, d.nq);
  const RoLayout R = ro_layout(d.n, d.ne2, d.ns2, d.nq * (d.k + 1));
  if (slot_bytes <= 0 || (int)(L.bytes + R.bytes) > slot_bytes) {
    run_in<FT, MK, false>(d, d.scratch, d.ro, a, WarpTeam{lane});
    return true;
  }
  uint8_t *slot = g_smem + slot_off;
  uint8_t *dst = slot + L.bytes;
  // the breadth-first tables and clique lists at the end of the block are
  // read under rule 1 / the clique bound only
  const uint32_t ro_copy = (a.rule || d.nq > 0) ? R.bytes : R.rank;
  if (ro_copy >= TMA_MIN_BYTES) {
    // one bulk copy of the read-only block into shared memory
    __syncwarp();
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar, ro_copy);
      bulk_copy_g2s(dst, d.ro, ro_copy, bar);
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
      run_in<FT, MK, false>(d, d.scratch, d.ro, a, WarpTeam{lane});
      return false;
    }
  } else {
    const uint4 *src = (const uint4 *)d.ro;
    uint4 *d4 = (uint4 *)dst;
    for (uint32_t i = lane; i < ro_copy / 16; i += 32) d4[i] = __ldcg(src + i);
  }
  run_in<FT, MK, true>(d, slot, dst, a, WarpTeam{lane});
  return true;
}

// ---- a search that its node budget ends at the first leaf ----------------
//
// With no incumbent nothing is pruned, so a search's first descent takes the
// first row of every column's order down to a leaf at node n + 1.  When the
// node budget is at most n + 1 the budget stops the search right there (the
// next row of the deepest level costs at least the leaf, so it is pruned and
// its count finds the budget spent), unless the leaf costs 0, which ends the
// search anyway.  The result is then that leaf, n + 1 nodes, status BUDGET
// (OK at cost 0), and the work of the descent alone.  Such a search needs no
// level record and no undo data: its state is the column classes (with
// exact summaries, and no class sizes), the fields and the masks, with a copy
// of the adjacency beside them as room allows, and a row's added cost comes
// from the masks of v's neighbours (Eq. 1) summed by one warp reduction per
// kind.  Giant instances under a
// small budget (a served layout whose simplified graph keeps a component of
// thousands of segments) take this form.

// Shared-memory layout of the descent: the column classes, the fields, the
// masks, then as room allows the adjacency offsets (16-bit, relative to the
// first segment of each block of 64), the conflict and stitch neighbour
// lists and the breadth-first ranks.
struct DescentLayout {
  uint32_t bk, rows, x, base;          // base: bytes of the part that must fit
  uint32_t co16, so16, cob, sob, offs_end;
  uint32_t cnbr, cnbr_end, snbr, snbr_end, rank, rank_end;
};
__device__ __forceinline__ DescentLayout descent_layout(int n, int k, int fb, int ne2, int ns2) {
  DescentLayout L;
  const int nfields = ((n + 3) / 4) * 4;
  uint32_t o = 0;
  L.bk = o; o += align16(bucket_bytes(n, k));
  L.rows = o; o += align16((uint32_t)fb * (uint32_t)nfields);
  L.x = o; o += align16((uint32_t)n);
  L.base = o;
  const uint32_t ow = align16(2u * (uint32_t)(n + 1)), bw = align16(4u * (uint32_t)((n >> 6) + 1));
  L.co16 = o; L.so16 = o + ow; L.cob = o + 2u * ow; L.sob = o + 2u * ow + bw;
  o += 2u * (ow + bw);
  L.offs_end = o;
  L.cnbr = o; o += align16(2u * (uint32_t)ne2);
  L.cnbr_end = o;
  L.snbr = o; o += align16(2u * (uint32_t)ns2);
  L.snbr_end = o;
  L.rank = o; o += align16(2u * (uint32_t)n);
  L.rank_end = o;
  return L;
}

// summary words per column class (two per lane of the column choice)
__device__ __forceinline__ int bk_summary_words(int n) { return (((n + 31) / 32) + 31) / 32; }

// 16-byte copy of `bytes` (a multiple of 16) from the read-only block in
// global memory into shared memory, by every thread of the CTA
__device__ __forceinline__ void cta_copy16(uint8_t *dst, const uint8_t *src, uint32_t bytes,
                                           int rank, int nthreads) {
  const uint4 *s = (const uint4 *)src;
  uint4 *d = (uint4 *)dst;
  for (uint32_t i = (uint32_t)rank; i < bytes / 16u; i += (uint32_t)nthreads) d[i] = __ldcg(s + i);
}

// The descent of instance d by warp 0 of the CTA (the other warps help set
// the state up).  `budget` is the search's budget (0 < budget <= n + 1);
// `split` / `sub`: the budgeted split search's first phase, whose leaf lies
// in subtree 0 (every level takes its first row).  Returns false, having
// done nothing, when the classes, fields and masks do not fit `room`.
template <typename FT, int MK>
__device__ __noinline__ bool run_descent(const InstDesc &d, const LaunchArgs &a,
                                         const CtaTeam &team, uint8_t *mem, uint32_t room,
                                         bool split) {
  constexpr uint32_t FLAG = 1u << (8 * sizeof(FT) - 1);
  const int n = d.n, k = d.k;
  const DescentLayout L = descent_layout(n, k, (int)sizeof(FT), d.ne2, d.ns2);
  if (L.base > room || n < 1 || bk_summary_words(n) > 64) return false;
  const RoLayout R = ro_layout(n, d.ne2, d.ns2, d.nq * (k + 1));
  const int2 *gptr = (const int2 *)(d.ro + R.ptr);
  const int rk = team.rank, nt = team.size();
  // the 16-bit offsets need every block of 64 segments to span fewer than
  // 65,536 entries of each list
  bool offs = L.offs_end <= room;
  if (offs) {
    bool wide = false;
    for (int b = rk * 64; b < n; b += nt * 64) {
      const int2 p0 = __ldcg(gptr + b), p1 = __ldcg(gptr + min(b + 64, n));
      wide |= (p1.x - p0.x) >= 65536 || (p1.y - p0.y) >= 65536;
    }
    offs = !__syncthreads_or(wide);
  }
  const bool cl = offs && L.cnbr_end <= room;
  const bool sl = cl && L.snbr_end <= room;
  const bool rl = sl && a.rule && L.rank_end <= room;
  Buckets bk;
  bk.carve(mem + L.bk, n, k);
  FT *rows = (FT *)(mem + L.rows);
  int8_t *x = (int8_t *)(mem + L.x);
  uint16_t *co16 = (uint16_t *)(mem + L.co16), *so16 = (uint16_t *)(mem + L.so16);
  int32_t *cob = (int32_t *)(mem + L.cob), *sob = (int32_t *)(mem + L.sob);
  const uint16_t *cnbr = cl ? (const uint16_t *)(mem + L.cnbr) : (const uint16_t *)(d.ro + R.cnbr);
  const uint16_t *snbr = sl ? (const uint16_t *)(mem + L.snbr) : (const uint16_t *)(d.ro + R.snbr);
  const uint16_t *rank = rl ? (const uint16_t *)(mem + L.rank) : (const uint16_t *)(d.ro + R.rank);
  const uint16_t *order = (const uint16_t *)(d.ro + R.order);
  // ---- state: every segment uncovered with k active rows, no mask ----
  const uint32_t kmask = (1u << k) - 1u;
  const int nfields = ((n + 3) / 4) * 4;
  for (int i = rk; i < nfields; i += nt) rows[i] = i < n ? (FT)(kmask | FLAG) : (FT)0;
  for (int i = rk; i < n; i += nt) x[i] = -1;
  {
    const int w32 = bk.w32, s32 = bk.s32;
    for (int i = rk; i < k * w32; i += nt) bk.cls[i] = 0u;
    for (int w = rk; w < w32; w += nt) {
      const int lo = 32 * w;
      const uint32_t bits = n - lo >= 32 ? 0xFFFFFFFFu : ((1u << (n - lo)) - 1u);
      bk.cls[k * w32 + w] = bits;
      bk.ur[w] = bits;
    }
    for (int j = rk; j < (k + 1) * s32; j += nt) {
      const int m = j / s32, jj = j % s32, left = w32 - 32 * jj;
      bk.sum[j] = m < k ? 0u : left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    }
    for (int jj = rk; jj < s32; jj += nt) {
      const int left = w32 - 32 * jj;
      bk.urs[jj] = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
    }
  }
  if (offs)
    for (int i = rk; i <= n; i += nt) {
      const int2 q = __ldcg(gptr + i), b = __ldcg(gptr + (i & ~63));
      co16[i] = (uint16_t)(q.x - b.x);
      so16[i] = (uint16_t)(q.y - b.y);
      if ((i & 63) == 0) {
        cob[i >> 6] = q.x;
        sob[i >> 6] = q.y;
      }
    }
  if (cl) cta_copy16(mem + L.cnbr, d.ro + R.cnbr, align16(2u * (uint32_t)d.ne2), rk, nt);
  if (sl) cta_copy16(mem + L.snbr, d.ro + R.snbr, align16(2u * (uint32_t)d.ns2), rk, nt);
  if (rl) cta_copy16(mem + L.rank, d.ro + R.rank, align16(2u * (uint32_t)n), rk, nt);
  __syncthreads();
  if ((rk >> 5) == 0) {
    const int lane = rk;
    const int Cc = d.cost_conflict, Cs = d.cost_stitch;
    const int w32 = bk.w32, s32 = bk.s32;
    // class membership moves.  Every summary here is exact (a bit per word of
    // the class that holds a segment): a cover first takes segments out of
    // their classes, clearing the summary bit of a word it empties, and only
    // after a warp barrier puts them into their new ones, so no word refills
    // while another lane judges it empty.
    auto cls_remove = [&](int m, int u) {
      const int w = u >> 5;
      const uint32_t b = 1u << (u & 31);
      const uint32_t old = atomicAnd(&bk.cls[m * w32 + w], ~b);
      if ((old & ~b) == 0u) atomicAnd(&bk.sum[m * s32 + (w >> 5)], ~(1u << (w & 31)));
    };
    auto cls_add = [&](int m, int u) {
      const int w = u >> 5;
      atomicOr(&bk.cls[m * w32 + w], 1u << (u & 31));
      atomicOr(&bk.sum[m * s32 + (w >> 5)], 1u << (w & 31));
    };
    int32_t g = 0, best = INF32;
    int64_t nodes = 0, work = 0, next_check = 1024;
    int status = MPLD_OK;
    const uint64_t t0 = __shfl_sync(FULL, lane == 0 ? globaltimer() : 0ull, 0);
    for (int level = 0;; ++level) {
      // ---- a node ----
      ++nodes;
      work += 2 * (int64_t)(n - level);
      if (nodes >= next_check) {
        next_check = nodes + 1024;
        const uint64_t now = __shfl_sync(FULL, lane == 0 ? globaltimer() : 0ull, 0);
        if ((int64_t)(now - t0) > a.time_limit_ns) { status = MPLD_TIMEOUT; break; }
      }
      // column choice, as the column classes give it to the full search:
      // the first class with a summary bit is the fewest-rows class, and
      // its lowest summary bit leads to its lowest segment (summary words
      // lane and lane + 32 of each class in this lane)
      uint32_t slo[MK + 1], shi[MK + 1];
      uint32_t have = 0u;
#pragma unroll
      for (int m = 0; m <= MK; ++m) {
        slo[m] = 0u;
        shi[m] = 0u;
        if (m <= k) {
          if (lane < s32) slo[m] = bk.sum[m * s32 + lane];
          if (lane + 32 < s32) shi[m] = bk.sum[m * s32 + lane + 32];
        }
        have |= (slo[m] | shi[m]) != 0u ? 1u << m : 0u;
      }
      have = __reduce_or_sync(FULL, have);
      if (have == 0u) {
        // leaf: every primary column covered
        best = g;
        for (int i = lane; i < n; i += 32) d.mask[i] = x[i];
        status = g == 0 ? MPLD_OK : MPLD_BUDGET;
        break;
      }
      int v = -1;
      const int m0 = a.rule == 0 ? __ffs(have) - 1 : ((have & 2u) ? 1 : -1);
      if (m0 >= 0) {
        uint32_t lo = slo[0], hi = shi[0];
#pragma unroll
        for (int m = 1; m <= MK; ++m)
          if (m == m0) {
            lo = slo[m];
            hi = shi[m];
          }
        const uint32_t nzl = __ballot_sync(FULL, lo != 0u), nzh = __ballot_sync(FULL, hi != 0u);
        const int l = nzl ? __ffs(nzl) - 1 : __ffs(nzh) - 1;
        const uint32_t sw = __shfl_sync(FULL, nzl ? lo : hi, l & 31);
        if (sw != 0u) {
          const int w = (nzl ? l : 32 + l) * 32 + __ffs(sw) - 1;
          v = w * 32 + __ffs(bk.cls[m0 * w32 + w]) - 1;
        }
      } else {
        const int r = bk.lowest(bk.ur, bk.urs, lane);
        if (r >= 0) v = (int)__ldcg(order + r);
      }
      // (never taken: every class and its summary agree after each cover)
      if ((unsigned)v >= (unsigned)n) { status = MPLD_TIMEOUT; break; }
      const uint32_t fv = (uint32_t)rows[v];
      int cb, dc, sb, ds;
      if (offs) {
        const int v1 = v + 1;
        cb = cob[v >> 6] + (int)co16[v];
        dc = cob[v1 >> 6] + (int)co16[v1] - cb;
        sb = sob[v >> 6] + (int)so16[v];
        ds = sob[v1 >> 6] + (int)so16[v1] - sb;
      } else {
        const int2 p0 = __ldcg(gptr + v), p1 = __ldcg(gptr + v + 1);
        cb = p0.x, dc = p1.x - p0.x, sb = p0.y, ds = p1.y - p0.y;
      }
      // masks held by v's neighbours: per mask, how many conflict / stitch
      // neighbours hold it (one-hot 8-bit lanes, masks 0-3 and 4-7, summed
      // over the warp)
      int cc[MK], sc[MK];
#pragma unroll
      for (int c = 0; c < MK; ++c) cc[c] = sc[c] = 0;
      auto onehot = [](int xu, uint32_t &lo, uint32_t &hi) {
        if (xu >= 0) {
          if (xu < 4) lo = 1u << (8 * xu);
          else hi = 1u << (8 * (xu - 4));
        }
      };
      auto tally = [&](int (&cnt)[MK], uint32_t lo, uint32_t hi) {
        lo = __reduce_add_sync(FULL, lo);
        if (MK > 4) hi = __reduce_add_sync(FULL, hi);
#pragma unroll
        for (int c = 0; c < MK; ++c) cnt[c] += (int)(((c < 4 ? lo : hi) >> (8 * (c & 3))) & 0xFFu);
      };
      int u0 = -1;   // this lane's conflict neighbour of the first pass and its field
      uint32_t f0 = 0u;
      if (dc + ds <= 32) {
        // one pass: lanes [0, dc) take the conflict neighbours, lanes
        // [dc, dc + ds) the stitch neighbours
        uint32_t clo = 0u, chi = 0u, tlo = 0u, thi = 0u;
        if (lane < dc) {
          u0 = cl ? (int)cnbr[cb + lane] : (int)__ldcg(cnbr + cb + lane);
          f0 = (uint32_t)rows[u0];
          onehot(x[u0], clo, chi);
        } else if (lane < dc + ds) {
          const int u = sl ? (int)snbr[sb + lane - dc] : (int)__ldcg(snbr + sb + lane - dc);
          onehot(x[u], tlo, thi);
        }
        tally(cc, clo, chi);
        tally(sc, tlo, thi);
      } else {
        for (int i0 = 0; i0 < dc; i0 += 32) {
          const int i = i0 + lane;
          uint32_t lo = 0u, hi = 0u;
          if (i < dc) {
            const int u = cl ? (int)cnbr[cb + i] : (int)__ldcg(cnbr + cb + i);
            if (i0 == 0) {
              u0 = u;
              f0 = (uint32_t)rows[u];
            }
            onehot(x[u], lo, hi);
          }
          tally(cc, lo, hi);
        }
        for (int i0 = 0; i0 < ds; i0 += 32) {
          const int i = i0 + lane;
          uint32_t lo = 0u, hi = 0u;
          if (i < ds) onehot(x[sl ? (int)snbr[sb + i] : (int)__ldcg(snbr + sb + i)], lo, hi);
          tally(sc, lo, hi);
        }
      }
      int stot = 0;
#pragma unroll
      for (int c = 0; c < MK; ++c) stot += sc[c];
      // the first row of v's order: the lowest added cost, lowest mask on ties
      int cbest = 0;
      int32_t ibest = INF32;
#pragma unroll
      for (int c = 0; c < MK; ++c) {
        const int32_t inc = Cc * cc[c] + Cs * (stot - sc[c]);
        if (c < k && inc < ibest) {
          ibest = inc;
          cbest = c;
        }
      }
      work += (int64_t)(k * (dc + ds) + 5 * (1 + dc));
      // ---- cover row (v, cbest), 32 conflict neighbours at a time ----
      const uint32_t bit = 1u << cbest;
      for (int i0 = 0; i0 == 0 || i0 < dc; i0 += 32) {
        const int i = i0 + lane;
        int u = -1;
        uint32_t f = 0u;
        if (i < dc) {
          if (i0 == 0) {
            u = u0;
            f = f0;
          } else {
            u = cl ? (int)cnbr[cb + i] : (int)__ldcg(cnbr + cb + i);
            f = (uint32_t)rows[u];
          }
        }
        if (i0 == 0 && lane == 0) {
          rows[v] = 0;
          x[v] = (int8_t)cbest;
          cls_remove(__popc(fv & kmask), v);
          if (a.rule) bk.rank_set(rl ? (int)rank[v] : (int)__ldcg(rank + v), false);
        }
        int mv = 0;
        if (u >= 0 && (f & FLAG) && (f & bit)) {
          rows[u] = (FT)(f & ~bit);
          mv = __popc(f & kmask);
          cls_remove(mv, u);
        }
        __syncwarp();
        if (mv > 0) cls_add(mv - 1, u);
        __syncwarp();
      }
      g += ibest;
    }
    if (lane == 0) {
      d.res->cost = best == INF32 ? INT64_MAX : (int64_t)best;
      d.res->nodes = nodes;
      d.res->status = status;
      d.res->sub = 0;
      d.res->work = work;
      if (split && status == MPLD_BUDGET) split_enlist(a, d, best, 0u);
    }
    __syncwarp();
  }
  __syncthreads();
  return true;
}

// One large instance searched by the CTA; its state stays in its global
// scratch region and its adjacency is read through L2.  When the CTA's
// slots hold its column classes (`bk_mem`, `bk_room` bytes), warp 0 searches
// it alone with them, so that a node costs its neighbours' updates rather
// than a scan of every segment; otherwise every thread of the CTA scans.
template <typename FT, int MK>
__device__ __noinline__ void run_instance_cta(const InstDesc &d, const LaunchArgs &a,
                                              const CtaTeam &team, uint8_t *bk_mem,
                                              uint32_t bk_room) {
  {
    // a search whose budget ends it at its first leaf: the descent alone
    const bool split = a.split && d.n <= SPLIT_MAX_N;
    int64_t b = a.budget;
    if (split) {
      int D;
      uint32_t S;
      split_cut(d.n, d.k, D, S);
      b = split_search_budget(a.budget, S);
    }
    if (b > 0 && b <= (int64_t)d.n + 1 && run_descent<FT, MK>(d, a, team, bk_mem, bk_room, split))
      return;
  }
  if (bucket_bytes(d.n, d.k) <= bk_room) {
    if ((team.rank >> 5) == 0)
      run_in<FT, MK, false, WarpTeam, true>(d, d.scratch, d.ro, a, WarpTeam{team.rank}, bk_mem,
                                            bk_room);
    __syncthreads();
    return;
  }
  run_in<FT, MK, false>(d, d.scratch, d.ro, a, team);
}

// Budgeted split search, second phase, for an instance beyond the register
// form: one subtree searched by one warp with the general search, its state
// in the warp's own global region (`state`), its adjacency read through L2.
// search: subtree s with budget b and the incumbent key1 (the first
// search's); publishes to the context as par_search's PAR_BUDGET does and
// returns true in the warp that completes the last subtree.  replay: the
// subtree and bound of `key1` (cost* << 32 | s* + 1), masks to d.mask;
// returns whether it took its leaf.
template <typename FT, int MK, bool SM>
__device__ __noinline__ bool split_general(const InstDesc &d, uint8_t *state, const uint8_t *ro,
                                           const LaunchArgs &a, int lane, ParCtx *ctx, uint32_t s,
                                           int cut, uint32_t S, int64_t b, unsigned long long key1,
                                           bool replay) {
  using Srch = Search<FT, MK, SM, WarpTeam>;
  const int n = d.n;
  const StateLayout L = state_layout(n, d.ne2, d.k, 0);
  const RoLayout R = ro_layout(n, d.ne2, d.ns2, 0);
  Srch sr;
  sr.team = WarpTeam{lane};
  sr.lv = (uint4 *)(state + L.lv);
  sr.lvx = (int32_t *)(state + L.lvx);
  sr.ccnt = (uint64_t *)(state + L.ccnt);
  sr.scnt = (uint64_t *)(state + L.scnt);
  sr.rows = (FT *)(state + L.rows);
  sr.oldf = (FT *)(state + L.oldf);
  sr.savf = (FT *)(state + L.savf);
  sr.x = (int8_t *)(state + L.x);
  sr.ptr = (const int2 *)(ro + R.ptr);
  sr.cnbr = (const uint16_t *)(ro + R.cnbr);
  sr.snbr = (const uint16_t *)(ro + R.snbr);
  sr.rank = (const uint16_t *)(ro + R.rank);
  sr.order = (const uint16_t *)(ro + R.order);
  sr.qptr = nullptr;
  sr.qlist = nullptr;
  sr.qcnt = state + L.qcnt;
  sr.qlev = (int32_t *)(state + L.qlev);
  sr.nq = 0;
  sr.rule = a.rule;
  sr.n = n;
  sr.k = d.k;
  sr.Cc = d.cost_conflict;
  sr.Cs = d.cost_stitch;
  sr.kmask = (1u << d.k) - 1u;
  const FT init = (FT)(sr.kmask | Srch::FLAG);
  const int nfields = ((n + Srch::PER_WORD - 1) / Srch::PER_WORD) * Srch::PER_WORD;
  for (int i = lane; i < nfields; i += 32) sr.rows[i] = i < n ? init : (FT)0;
  for (int i = lane; i < n; i += 32) sr.x[i] = -1;
  for (int i = lane; i < n * Srch::CW; i += 32) {
    sr.ccnt[i] = 0;
    sr.scnt[i] = 0;
  }
  __syncwarp();
  SplitSpec sp;
  sp.cut = cut;
  sp.forced = true;
  sp.replay = replay;
  const int32_t kc = (int32_t)(key1 >> 32);
  const uint32_t ks = (uint32_t)(key1 & 0xFFFFFFFFull);
  sp.prefix = replay ? ks - 1u : s;
  sp.init_best = replay ? kc + 1 : kc + (s < ks ? 1 : 0);
  // the time limit runs from the instance's start (the replay's from its own)
  uint64_t t0 = 0;
  if (lane == 0) {
    const uint64_t now = globaltimer();
    if (replay) {
      t0 = now;
    } else {
      const unsigned long long prev = atomicCAS(&ctx->t0, 0ull, (unsigned long long)now);
      t0 = prev != 0ull ? (uint64_t)prev : now;
    }
  }
  t0 = __shfl_sync(FULL, t0, 0);
  int32_t best = INF32;
  int64_t nodes = 0, work = 0;
  const int st = sr.run(lane, replay ? 0 : b, a.time_limit_ns, replay ? d.mask : nullptr, best,
                        nodes, work, sp, t0);
  if (replay) return sp.found;
  uint32_t fin = 0;
  if (lane == 0) {
    if (sp.found) atomicMin(&ctx->key, ((unsigned long long)(uint32_t)best << 32) | s);
    atomicAdd(&ctx->nodes, (unsigned long long)nodes);
    atomicAdd(&ctx->work, (unsigned long long)work);
    if (st == MPLD_TIMEOUT) atomicExch(&ctx->timed_out, 1u);
    if (st == MPLD_BUDGET) atomicExch(&ctx->pad, 1u);
    __threadfence();
    fin = atomicAdd(&ctx->done, 1u) == S - 1u ? 1u : 0u;
  }
  return __shfl_sync(FULL, fin, 0) != 0u;
}

// state: the search state (the warp's slot or its global region); ro: the
// instance's read-only block, copied into the slot after the state (ro_smem)
// or in the arena
template <bool SM>
__device__ __forceinline__ bool split_general_k(const InstDesc &d, uint8_t *state,
                                                const uint8_t *ro, const LaunchArgs &a, int lane,
                                                ParCtx *ctx, uint32_t s, int cut, uint32_t S,
                                                int64_t b, unsigned long long key1, bool replay) {
  if (d.k == 3)
    return split_general<uint8_t, 3, SM>(d, state, ro, a, lane, ctx, s, cut, S, b, key1, replay);
  if (d.k == 4)
    return split_general<uint8_t, 4, SM>(d, state, ro, a, lane, ctx, s, cut, S, b, key1, replay);
  if (d.k == 2)
    return split_general<uint8_t, 2, SM>(d, state, ro, a, lane, ctx, s, cut, S, b, key1, replay);
  if (d.k <= 7)
    return split_general<uint8_t, 8, SM>(d, state, ro, a, lane, ctx, s, cut, S, b, key1, replay);
  return split_general<uint16_t, 8, SM>(d, state, ro, a, lane, ctx, s, cut, S, b, key1, replay);
}
__device__ __noinline__ bool split_general_dispatch(const InstDesc &d, uint8_t *state,
                                                    const uint8_t *ro, bool ro_smem,
                                                    const LaunchArgs &a, int lane, ParCtx *ctx,
                                                    uint32_t s, int cut, uint32_t S, int64_t b,
                                                    unsigned long long key1, bool replay) {
  if (ro_smem) return split_general_k<true>(d, state, ro, a, lane, ctx, s, cut, S, b, key1, replay);
  return split_general_k<false>(d, state, ro, a, lane, ctx, s, cut, S, b, key1, replay);
}

// ---- per-lane search (budgeted split search, second phase) ---------------
//
// For instances of at most 64 segments and k <= 4 every lane searches a
// subtree of its own: the same canonical search as par_search's PAR_BUDGET
// (same column and row order, bound, node count and budget), with the
// instance's state in registers as one bit per segment (W: a 32- or 64-bit
// word):
//   unc      bit v: primary column P_v uncovered;
//   act[c]   bit v: row (v, c) still active (no conflict neighbour of v
//            holds mask c);
//   asg[c]   bit v: x_v = c;
//   uncr     (column rule 1) bit r: the segment of breadth-first rank r is
//            uncovered.
// The column choice counts each segment's active rows with a bit-sliced
// adder over act[], so the fewest-rows column is the lowest set bit of the
// first non-empty count class; a row's added cost (Eq. 1) is
// cost_conflict * popc(conflict nbrs & asg[c]) + cost_stitch *
// (assigned stitch nbrs - popc(stitch nbrs & asg[c])); the cover of row
// (v, c) is act[c] &= ~conflict nbrs(v) and the clearing of v's bits.  Each
// level below the cut keeps {v | row place << 8 | row order << 12}, the path
// cost and act[c] before the cover: for up to 32 segments in shared memory
// laid out [word][level][lane], for more in the thread's local memory.
struct LaneOut {
  int32_t best;
  bool found, hit, timed_out;
  int64_t nodes, work;
  unsigned long long m0, m1;   // found: the best leaf's masks, bit 0 and bit 1 per segment
  uint32_t sub;                // track > 0: subtree of the best leaf (its first `track` row places)
};

template <typename W> __device__ __forceinline__ int popcw(W x) {
  if constexpr (sizeof(W) == 4) return __popc(x);
  else return __popcll(x);
}
template <typename W> __device__ __forceinline__ int lowbit(W x) {
  if constexpr (sizeof(W) == 4) return __ffs(x) - 1;
  else return __ffsll((long long)x) - 1;
}

// per segment, whether its number of active rows among act[0..K) is m
template <int K, typename W>
__device__ __forceinline__ void row_count_classes(const W (&act)[K], W (&cls)[K + 1]) {
  if constexpr (K == 2) {
    const W s0 = act[0] ^ act[1], s1 = act[0] & act[1];
    cls[0] = ~(s0 | s1); cls[1] = s0; cls[2] = s1;
  } else if constexpr (K == 3) {
    const W s0 = act[0] ^ act[1] ^ act[2];
    const W s1 = (act[0] & act[1]) | (act[2] & (act[0] ^ act[1]));
    cls[0] = ~(s0 | s1); cls[1] = s0 & ~s1; cls[2] = ~s0 & s1; cls[3] = s0 & s1;
  } else {
    const W t0 = act[0] ^ act[1], u0 = act[0] & act[1];
    const W t1 = act[2] ^ act[3], u1 = act[2] & act[3];
    const W s0 = t0 ^ t1, cy = t0 & t1;
    const W s1 = u0 ^ u1 ^ cy, s2 = (u0 & u1) | (cy & (u0 ^ u1));
    cls[0] = ~(s0 | s1 | s2); cls[1] = s0 & ~s1 & ~s2; cls[2] = ~s0 & s1 & ~s2;
    cls[3] = s0 & s1 & ~s2; cls[4] = s2;   // four rows: s2 set, s0 = s1 = 0
  }
}

// The level records, in the thread's local memory.
template <typename W> struct LaneStack {
  static constexpr int N = 8 * (int)sizeof(W);
  uint32_t hh[N], gg[N];
  W ss[N];
  __device__ __forceinline__ uint32_t &h(int l) { return hh[l]; }
  __device__ __forceinline__ uint32_t &g(int l) { return gg[l]; }
  __device__ __forceinline__ W &s(int l) { return ss[l]; }
};

// cut / prefix: the forced levels of a subtree search (cut = 0: the whole
// tree); track: the whole tree's first search of the budgeted split search,
// whose best leaf's subtree (row places of the first `track` levels) is kept.
template <typename W, int K, int RULE>
__device__ __noinline__ void lane_search(const InstDesc &d, const uint8_t *ro, int cut,
                                         uint32_t prefix, int32_t thr0, int64_t budget,
                                         int64_t time_limit_ns, uint64_t t0, int track,
                                         LaneOut &o) {
  const int n = d.n;
  const int Cc = d.cost_conflict, Cs = d.cost_stitch;
  const RoLayout R = ro_layout(n, d.ne2, d.ns2, 0);
  const unsigned long long *cadj = (const unsigned long long *)(ro + R.bits);
  const unsigned long long *sadj = cadj + n;
  const uint16_t *rank = (const uint16_t *)(ro + R.rank);
  const uint16_t *order = (const uint16_t *)(ro + R.order);
  LaneStack<W> st;
  const W one = 1;
  const W all = n >= (int)(8 * sizeof(W)) ? ~(W)0 : ((one << n) - one);
  W unc = all, uncr = all, act[K], asg[K];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    act[c] = all;
    asg[c] = 0;
  }
  int32_t thr = thr0, g = 0;
  int level = 0;
  int64_t nodes = 0, work = 0, next_check = 1024;
  bool found = false, hit = false, tout = false;
  W m0 = 0, m1 = 0;
  uint32_t sub = 0;
  auto count_pruned = [&](int m) -> bool {
    const int64_t room = budget > 0 ? budget - nodes : (int64_t)m;
    nodes += room < m ? (room > 0 ? room : 0) : (int64_t)m;
    return room < m;
  };
  // added cost of row (v, c) against the current assignment
  auto row_cost = [&](W ca, W sa, int c) -> int32_t {
    const int stot = popcw<W>(sa & all & ~unc);
    return Cc * popcw<W>(ca & asg[c]) + Cs * (stot - popcw<W>(sa & asg[c]));
  };
  // Each pass: a lane that must backtrack pops levels until it covers the
  // next row of one (or its search ends), then every lane that is entering
  // a node expands it, so a warp's lanes meet in the node code whichever of
  // them backtracked.  Each lane takes the same steps in the same order as
  // a depth-first search of its own.
  bool enter = true;
  for (;;) {
    if (!enter) {
      // ---- backtrack: next row of the level above, or undo its column ----
      bool stop = false;
      for (;;) {
        if (level <= cut) {
          stop = true;
          break;
        }
        --level;
        const uint32_t h = st.h(level);
        const int32_t gl = (int32_t)st.g(level);
        const int v = (int)(h & 0xFFu), place = (int)((h >> 8) & 0xFu);
        const uint32_t ord = h >> 12;
        const W bit = one << v;
        const int cl = (int)((ord >> (2 * place)) & 3u);
        act[cl] = st.s(level);
        asg[cl] &= ~bit;
        unc |= bit;
        if (RULE) uncr |= one << rank[v];
        const int np = place + 1;
        if (np >= K) continue;   // the column is exhausted: keep popping
        const int c = (int)((ord >> (2 * np)) & 3u);
        const W ca = (W)cadj[v], sa = (W)sadj[v];
        const int32_t inc = row_cost(ca, sa, c);
        if (thr < INF32 && gl + inc >= thr) {
          // this row and the ones after it: children pruned on entry
          if (count_pruned(K - np)) {
            hit = true;
            stop = true;
            break;
          }
          continue;
        }
        work += 5 * (1 + popcw<W>(ca));
        st.h(level) = (h & ~0xF00u) | ((uint32_t)np << 8);
        st.s(level) = act[c];
        act[c] &= ~ca;
        unc &= ~bit;
        asg[c] |= bit;
        if (RULE) uncr &= ~(one << rank[v]);
        g = gl + inc;
        ++level;
        enter = true;
        break;
      }
      if (stop) break;
    }
    // ---- a node ----
    // the budget stops a search once it has an incumbent
    if (budget > 0 && thr < INF32 && nodes >= budget) { hit = true; break; }
    ++nodes;
    work += 2 * (n - level);
    if (nodes >= next_check) {
      next_check = nodes + 1024;
      if ((int64_t)(globaltimer() - t0) > time_limit_ns) { tout = true; break; }
    }
    if (unc == 0) {
      // leaf: every primary column covered
      if (g < thr) {
        // this leaf's masks: the leaf that sets the final bound is the
        // first one in depth-first order at that cost, the one a search of
        // this subtree bounded by that cost plus one would take first
        thr = g;
        found = true;
        m0 = asg[1];
        m1 = K > 2 ? asg[K > 2 ? 2 : 1] : (W)0;
        if constexpr (K == 4) {
          m0 |= asg[3];
          m1 |= asg[3];
        }
        if (track > 0) {
          sub = 0;
          for (int i = 0; i < track; ++i) sub = sub * (uint32_t)K + ((st.h(i) >> 8) & 0xFu);
        }
        if (g == 0) break;
      }
      if (level <= cut) break;
      enter = false;
      continue;
    }
    W cls[K + 1];
    row_count_classes<K, W>(act, cls);
    const W dead = unc & cls[0];
    int v;
    if constexpr (RULE == 0) {
      W cand = dead;
#pragma unroll
      for (int m = 1; m <= K; ++m) cand = cand ? cand : (unc & cls[m]);
      v = lowbit<W>(cand);
    } else {
      const W single = unc & cls[1];
      v = single ? lowbit<W>(single) : (int)order[lowbit<W>(uncr)];
    }
    if (thr < INF32 && g + Cc * popcw<W>(dead) >= thr) {
      if (level < cut) break;
      enter = false;
      continue;
    }
    const W ca = (W)cadj[v], sa = (W)sadj[v];
    uint32_t keys[K];
#pragma unroll
    for (int c = 0; c < K; ++c) keys[c] = ((uint32_t)row_cost(ca, sa, c) << 3) | (uint32_t)c;
    sort_keys<K>(keys);
    work += K * (popcw<W>(ca) + popcw<W>(sa)) + 5 * (1 + popcw<W>(ca));
    int place = 0;
    if (level < cut) {
      uint32_t pw = 1;
      for (int i = level + 1; i < cut; ++i) pw *= (uint32_t)K;
      place = (int)((prefix / pw) % (uint32_t)K);
    }
    uint32_t kp = keys[0];
#pragma unroll
    for (int i = 1; i < K; ++i) kp = i == place ? keys[i] : kp;
    if (thr < INF32 && g + (int32_t)(kp >> 3) >= thr) {
      // this row and the ones after it: their children are pruned on entry
      if (count_pruned(level < cut ? 1 : K)) { hit = true; break; }
      if (level < cut) break;
      enter = false;
      continue;
    }
    const int c = (int)(kp & 7u);
    if (level >= cut) {
      uint32_t ord = 0;
#pragma unroll
      for (int i = 0; i < K; ++i) ord |= (keys[i] & 3u) << (2 * i);
      st.h(level) = (uint32_t)v | ((uint32_t)place << 8) | (ord << 12);
      st.g(level) = (uint32_t)g;
      st.s(level) = act[c];
    }
    const W bit = one << v;
    act[c] &= ~ca;
    unc &= ~bit;
    asg[c] |= bit;
    if (RULE) uncr &= ~(one << rank[v]);
    g += (int32_t)(kp >> 3);
    ++level;
    continue;
  }
  o.best = thr;
  o.found = found;
  o.hit = hit;
  o.timed_out = tout;
  o.nodes = nodes;
  o.work = work;
  o.m0 = (unsigned long long)m0;
  o.m1 = (unsigned long long)m1;
  o.sub = sub;
}

template <typename W>
__device__ __forceinline__ void lane_dispatch_w(const InstDesc &d, int rule, int cut,
                                                uint32_t prefix, int32_t thr0, int64_t budget,
                                                int64_t tl, uint64_t t0, int track, LaneOut &o) {
  const uint8_t *ro = d.ro;
  if (d.k == 3) {
    if (rule) lane_search<W, 3, 1>(d, ro, cut, prefix, thr0, budget, tl, t0, track, o);
    else lane_search<W, 3, 0>(d, ro, cut, prefix, thr0, budget, tl, t0, track, o);
  } else if (d.k == 4) {
    if (rule) lane_search<W, 4, 1>(d, ro, cut, prefix, thr0, budget, tl, t0, track, o);
    else lane_search<W, 4, 0>(d, ro, cut, prefix, thr0, budget, tl, t0, track, o);
  } else {
    if (rule) lane_search<W, 2, 1>(d, ro, cut, prefix, thr0, budget, tl, t0, track, o);
    else lane_search<W, 2, 0>(d, ro, cut, prefix, thr0, budget, tl, t0, track, o);
  }
}

__device__ __noinline__ void lane_dispatch(const InstDesc &d, int rule, int cut, uint32_t prefix,
                                           int32_t thr0, int64_t budget, int64_t tl, uint64_t t0,
                                           int track, LaneOut &o) {
  if (d.n <= 32) lane_dispatch_w<uint32_t>(d, rule, cut, prefix, thr0, budget, tl, t0, track, o);
  else lane_dispatch_w<unsigned long long>(d, rule, cut, prefix, thr0, budget, tl, t0, track, o);
}

// The instance's result once its last subtree is done (one thread): the
// best (cost, subtree) with `ok` (false: its replay ran out of time, so the
// first search's incumbent and masks stand), nodes and work of both phases.
__device__ __forceinline__ void split_write_result(const InstDesc &d, ParCtx *ctx,
                                                   unsigned long long key, bool ok) {
  const int64_t nodes1 = d.res->nodes, work1 = d.res->work;
  const uint32_t to = *(volatile uint32_t *)&ctx->timed_out;
  const uint32_t bh = *(volatile uint32_t *)&ctx->pad;
  d.res->cost = (int64_t)(key >> 32);
  d.res->nodes = nodes1 + (int64_t)*(volatile unsigned long long *)&ctx->nodes;
  d.res->work = work1 + (int64_t)*(volatile unsigned long long *)&ctx->work;
  d.res->sub = (int32_t)(key & 0xFFFFFFFFull);
  d.res->status = (to || !ok) ? MPLD_TIMEOUT : bh ? MPLD_BUDGET : MPLD_OK;
}

// Budgeted split search, second phase (par == 4).  Items t = j * smax + s
// stand for hard-list entry j and subtree s (items past the entry's own
// subtree count are skipped).  First every warp takes items of the warps'
// list (instances beyond the per-lane search) from counter queue[0] and
// searches each subtree with the whole warp; then every lane takes items of
// the lanes' list from counter queue[1] on its own.  Each subtree has its own
// share of the budget and the first search's incumbent as its bound; the
// thread or warp that completes an instance's last subtree replays the
// winning subtree to write its masks (unless the first search's incumbent
// stands, whose masks are already written) and writes the result: the best
// (cost, subtree), nodes and work of both phases, status TIMEOUT / BUDGET /
// OK.
__device__ __noinline__ void run_split_phase2(const LaunchArgs &a, int lane, int warp, int nw,
                                              uint8_t *mine) {
  const int G = (int)gridDim.x * nw;
  const int gw = (int)blockIdx.x * nw + warp;
  uint8_t *wstate = a.split_scratch ? a.split_scratch + (size_t)gw * (size_t)a.split_state_bytes
                                    : nullptr;
  uint32_t HW = 0, HL = 0, HG = 0;
  if (lane == 0) {
    HW = (uint32_t)*(volatile int32_t *)a.hard;
    HL = (uint32_t)*(volatile int32_t *)(a.hard + 1);
    HG = (uint32_t)*(volatile int32_t *)(a.hard + 2);
  }
  HW = __shfl_sync(FULL, HW, 0);
  HL = __shfl_sync(FULL, HL, 0);
  HG = __shfl_sync(FULL, HG, 0);
  const int32_t *list_w = a.hard + 4;
  const int32_t *list_g = a.hard + 4 + 2 * a.hard_cap;
  // warps with a general-state region first take the subtrees of instances
  // beyond the register form (counter queue[2]), then every warp those of
  // the register form (queue[0])
  const bool gen_warp = gw < a.split_gen_warps;
  bool gen_phase = gen_warp && HG > 0;
  int built = -1;   // instance whose adjacency the slot holds (register form)
  int gro = -1;     // instance whose read-only block the slot holds (general form)
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(a.queue + (gen_phase ? 2 : 0), 1u);
    t = __shfl_sync(FULL, t, 0);
    if ((uint64_t)t >= (uint64_t)(gen_phase ? HG : HW) * (uint64_t)a.smax) {
      if (gen_phase) {
        gen_phase = false;
        continue;
      }
      break;
    }
    const uint32_t j = t / (uint32_t)a.smax, s = t % (uint32_t)a.smax;
    const int di = __ldcg((gen_phase ? list_g : list_w) + j);
    const InstDesc d = a.desc[di];
    int D;
    uint32_t S;
    split_cut(d.n, d.k, D, S);
    if (s >= S) continue;
    ParCtx *ctx = (ParCtx *)(a.par_buf + (size_t)di * 64);
    const int64_t b = split_search_budget(a.budget, S);
    const int64_t c1 = __ldcg(&d.res->cost);
    const uint32_t s1 = (uint32_t)__ldcg(&d.res->sub);
    const unsigned long long key1 = ((unsigned long long)(uint32_t)c1 << 32) | s1;
    const bool reg = reg_fits(d.n, d.k) && a.slot_bytes >= (int)reg_layout(d.n, d.k, 0).bytes;
    // the general form keeps its state in the warp's slot when it fits, and
    // its read-only block after it when that fits too; else its state is in
    // the warp's global region
    uint8_t *gstate = wstate;
    const uint8_t *gro_ptr = d.ro;
    bool ro_smem = false;
    if (!reg) {
      const uint32_t sb = align16(state_layout(d.n, d.ne2, d.k, 0).bytes);
      const RoLayout R = ro_layout(d.n, d.ne2, d.ns2, 0);
      const uint32_t ro_copy = a.rule ? R.bytes : R.rank;
      if ((uint32_t)a.slot_bytes >= sb) {
        gstate = mine;
        built = -1;
        if ((uint32_t)a.slot_bytes >= sb + ro_copy) {
          ro_smem = true;
          gro_ptr = mine + sb;
          if (gro != di) {
            const uint4 *src = (const uint4 *)d.ro;
            uint4 *dst = (uint4 *)(mine + sb);
            for (uint32_t i = lane; i < ro_copy / 16u; i += 32u) dst[i] = __ldcg(src + i);
            __syncwarp();
            gro = di;
          }
        }
      } else if (!wstate || a.split_state_bytes < d.state_bytes) {
        // the host sizes the slots or the per-warp regions for every instance
        if (lane == 0) atomicExch(a.err, MPLD_E_STATE);
        return;
      }
    }
    bool fin;
    if (reg) {
      gro = -1;
      ParItem it;
      it.sub = s;
      it.budget = b;
      it.build = built != di;
      it.split_cut = true;
      fin = par_dispatch(d, mine, a, lane, gw, G, ctx, nullptr, nullptr, PAR_BUDGET, key1, it);
      built = di;
    } else {
      fin = split_general_dispatch(d, gstate, gro_ptr, ro_smem, a, lane, ctx, s, D, S, b, key1,
                                   false);
    }
    if (!fin) continue;
    // every subtree of the instance is done: its best key is final
    __threadfence();
    unsigned long long key = 0ull;
    if (lane == 0) key = *(volatile unsigned long long *)&ctx->key;
    key = __shfl_sync(FULL, key, 0);
    bool ok = true;
    if (key != key1) {
      const unsigned long long rk = (key & ~0xFFFFFFFFull) | ((key & 0xFFFFFFFFull) + 1ull);
      if (reg) {
        ParItem it;
        it.build = false;
        it.split_cut = true;
        ok = par_dispatch(d, mine, a, lane, gw, G, ctx, nullptr, nullptr, PAR_REPLAY, rk, it);
      } else {
        ok = split_general_dispatch(d, gstate, gro_ptr, ro_smem, a, lane, ctx, 0, D, S, 0, rk,
                                    true);
      }
      if (!ok) key = key1;
    }
    if (lane == 0) split_write_result(d, ctx, key, ok);
    __syncwarp();
  }
}

// Every warp of the grid splits the instances desc[order[0..n_inst)] one
// after another: a warp takes subtrees of the first instance that still has
// some.  Contexts are 64 bytes apart in par_buf.  The warp that completes an
// instance's last subtree replays the winning subtree to write its masks,
// then writes its result.
__device__ __noinline__ void run_grid_queue(const LaunchArgs &a, int lane, int warp, int nw,
                                            uint8_t *mine) {
  const int G = (int)gridDim.x * nw;
  const int gw = (int)blockIdx.x * nw + warp;
  for (int j = 0; j < a.n_inst; ++j) {
    const InstDesc d = a.desc[a.order[j]];
    ParCtx *ctx = (ParCtx *)(a.par_buf + (size_t)j * 64);
    int D;
    uint32_t ns;
    par_cut(d.n, d.k, G, D, ns);
    uint32_t taken = 0;
    if (lane == 0) taken = *(volatile uint32_t *)&ctx->next;
    if (__shfl_sync(FULL, taken, 0) >= ns) continue;   // all handed out
    if (!reg_fits(d.n, d.k) || a.slot_bytes < (int)reg_layout(d.n, d.k, 0).bytes) {
      // the host queues only register-resident instances
      if (lane == 0) atomicExch(a.err, MPLD_E_STATE);
      return;
    }
    if (!par_dispatch(d, mine, a, lane, gw, G, ctx, nullptr, nullptr, PAR_QUEUE, 0ull)) continue;
    __threadfence();
    unsigned long long key = 0ull;
    if (lane == 0) key = *(volatile unsigned long long *)&ctx->key;
    key = __shfl_sync(FULL, key, 0);
    if (key != ~0ull)
      par_dispatch(d, mine, a, lane, gw, G, ctx, nullptr, nullptr, PAR_REPLAY,
                   (key & ~0xFFFFFFFFull) | ((key & 0xFFFFFFFFull) + 1ull));
    if (lane == 0) {
      d.res->cost = key == ~0ull ? INT64_MAX : (int64_t)(key >> 32);
      d.res->nodes = (int64_t)*(volatile unsigned long long *)&ctx->nodes;
      d.res->status = *(volatile uint32_t *)&ctx->timed_out ? MPLD_TIMEOUT : MPLD_OK;
      d.res->work = (int64_t)*(volatile unsigned long long *)&ctx->work;
    }
    __syncwarp();
  }
}

// Every warp of the grid splits the one instance desc[0]; the last warp to
// finish writes the result.
__device__ __noinline__ void run_grid_split(const LaunchArgs &a, int lane, int warp, int nw,
                                            uint8_t *mine) {
  const InstDesc d = a.desc[0];
  const int G = (int)gridDim.x * nw;
  const int gw = (int)blockIdx.x * nw + warp;
  const ParLayout PL = par_layout(G, d.n);
  ParCtx *ctx = (ParCtx *)(a.par_buf + PL.ctx);
  unsigned long long *wkey = (unsigned long long *)(a.par_buf + PL.wkey);
  int8_t *bx = (int8_t *)(a.par_buf + PL.bestx + (size_t)gw * PL.row);
  if (!reg_fits(d.n, d.k) || a.slot_bytes < (int)reg_layout(d.n, d.k, 0).bytes) {
    // the host launches this form only for register-resident instances
    if (threadIdx.x == 0) atomicExch(a.err, MPLD_E_STATE);
    return;
  }
  par_dispatch(d, mine, a, lane, gw, G, ctx, wkey, bx, PAR_OWN, 0ull);
  // publish this warp's masks, key and totals, then count it finished
  __threadfence();
  __syncwarp();
  uint32_t last = 0;
  if (lane == 0) last = atomicAdd(&ctx->done, 1u) == (uint32_t)(G - 1) ? 1u : 0u;
  last = __shfl_sync(FULL, last, 0);
  if (last) {
    __threadfence();
    const unsigned long long key = *(volatile unsigned long long *)&ctx->key;
    int win = -1;
    for (int i = lane; i < G; i += 32)
      if (__ldcg(wkey + i) == key) win = i;
    win = __reduce_max_sync(FULL, (uint32_t)(win + 1)) - 1;
    if (win >= 0) {
      const int8_t *wb = (const int8_t *)(a.par_buf + PL.bestx + (size_t)win * PL.row);
      for (int i = lane; i < d.n; i += 32) d.mask[i] = __ldcg(wb + i);
    }
    if (lane == 0) {
      d.res->cost = key == ~0ull ? INT64_MAX : (int64_t)(key >> 32);
      d.res->nodes = (int64_t)*(volatile unsigned long long *)&ctx->nodes;
      d.res->status = *(volatile uint32_t *)&ctx->timed_out ? MPLD_TIMEOUT : MPLD_OK;
      d.res->work = (int64_t)*(volatile unsigned long long *)&ctx->work;
    }
  }
}

__global__ void __launch_bounds__(512, 1) mpld_search_kernel(const LaunchArgs a) {
  // a launch after this one that reads nothing it writes (the per-lane
  // first searches) may take SMs as its blocks finish
  launch_dependents();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  uint32_t *team_red = (uint32_t *)g_smem;
  uint64_t *bars = (uint64_t *)(g_smem + TEAM_BYTES);
  const uint32_t bar_bytes = kernel_head_bytes(nw);
  const uint32_t slot_off =
      bar_bytes + (uint32_t)warp * (uint32_t)(a.slot_bytes > 0 ? a.slot_bytes : 0);
  int slot_bytes = a.slot_bytes;
  uint64_t *bar = bars + warp;
  if (lane == 0) mbar_init(bar);
  __syncwarp();
  if (lane == 0) fence_proxy_async();
  __syncwarp();
  uint32_t phase = 0;

  if (a.par == 2) {
    run_grid_split(a, lane, warp, nw, g_smem + slot_off);
    return;
  }
  if (a.par == 3) {
    run_grid_queue(a, lane, warp, nw, g_smem + slot_off);
    return;
  }
  if (a.par == 4) {
    run_split_phase2(a, lane, warp, nw, g_smem + slot_off);
    // this launch may have started beside the lanes' kernel before it (its
    // blocks take SMs as the lanes' blocks finish): it completes only after
    // that kernel, so what follows on the stream sees both
    wait_prerequisites();
    return;
  }

  // the first blocks search the large instances (the first n_large of the
  // order) as whole-CTA teams, taking them from the second work counter;
  // then they join the warps on the rest
  if ((int)blockIdx.x < a.n_large) {
    const CtaTeam team{(int)threadIdx.x, (int)blockDim.x, team_red};
    for (int t = (int)blockIdx.x;;) {
      if (a.queue) {
        if (threadIdx.x == 0) team_red[18] = atomicAdd(a.queue + 1, 1u);
        __syncthreads();
        t = (int)team_red[18];
        __syncthreads();
      }
      if (t >= a.n_large) break;
      const InstDesc d = a.desc[a.order ? a.order[t] : t];
      if (a.par && reg_fits(d.n, d.k) && a.slot_bytes >= (int)reg_layout(d.n, d.k, 0).bytes) {
        // exact search with the warps splitting the subtrees of one instance
        ParCtx *ctx = (ParCtx *)(g_smem + PAR_CTX_OFF);
        unsigned long long *wkey = (unsigned long long *)(g_smem + PAR_WKEY_OFF);
        if (threadIdx.x == 0) {
          ctx->key = ~0ull;
          ctx->nodes = 0;
          ctx->work = 0;
          ctx->next = 0;
          ctx->timed_out = 0;
          ctx->done = 0;
          ctx->t0 = 0;
        }
        __syncthreads();
        uint8_t *mine = g_smem + slot_off;
        int8_t *bx = (int8_t *)(mine + reg_layout(d.n, d.k, 0).bestx);
        par_dispatch(d, mine, a, lane, warp, nw, ctx, wkey, bx, PAR_OWN, 0ull);
        __syncthreads();
        // the warp holding the winning leaf writes its masks
        const unsigned long long key = ctx->key;
        if (wkey[warp] == key)
          for (int i = lane; i < d.n; i += 32) d.mask[i] = bx[i];
        if (threadIdx.x == 0) {
          d.res->cost = key == ~0ull ? INT64_MAX : (int64_t)(key >> 32);
          d.res->nodes = (int64_t)ctx->nodes;
          d.res->status = ctx->timed_out ? MPLD_TIMEOUT : MPLD_OK;
          d.res->work = (int64_t)ctx->work;
        }
        __syncthreads();
      } else {
        // the CTA's slots, free while it searches this instance
        uint8_t *bkm = g_smem + bar_bytes;
        const uint32_t room = (uint32_t)nw * (uint32_t)(a.slot_bytes > 0 ? a.slot_bytes : 0);
        if (d.k == 3) run_instance_cta<uint8_t, 3>(d, a, team, bkm, room);
        else if (d.k == 4) run_instance_cta<uint8_t, 4>(d, a, team, bkm, room);
        else if (d.k == 2) run_instance_cta<uint8_t, 2>(d, a, team, bkm, room);
        else if (d.k <= 7) run_instance_cta<uint8_t, 8>(d, a, team, bkm, room);
        else run_instance_cta<uint16_t, 8>(d, a, team, bkm, room);
      }
      if (!a.queue) break;
    }
  }

  const int n_small = a.n_inst - a.n_large;
  int idx = a.queue ? 0 : blockIdx.x * nw + warp - a.n_large * nw;
  for (;;) {
    if (a.queue) {
      uint32_t t = 0;
      if (lane == 0) t = atomicAdd(a.queue, 1u);
      idx = (int)__shfl_sync(FULL, t, 0);
    }
    if (idx < 0 || idx >= n_small) break;
    const int pos = a.n_large + idx;
    const InstDesc d = a.desc[a.order ? a.order[pos] : pos];
    bool ok;
    if (d.k == 3) ok = run_instance<uint8_t, 3>(d, slot_off, slot_bytes, bar, phase, a, lane);
    else if (d.k == 4) ok = run_instance<uint8_t, 4>(d, slot_off, slot_bytes, bar, phase, a, lane);
    else if (d.k == 2) ok = run_instance<uint8_t, 2>(d, slot_off, slot_bytes, bar, phase, a, lane);
    else if (d.k <= 7) ok = run_instance<uint8_t, 8>(d, slot_off, slot_bytes, bar, phase, a, lane);
    else ok = run_instance<uint16_t, 8>(d, slot_off, slot_bytes, bar, phase, a, lane);
    if (!ok) slot_bytes = 0;
    if (!a.queue) break;
  }
}

// Largest dynamic shared memory size already granted to the kernel; the
// attribute is only raised, and only outside stream capture (the shape is
// chosen, and the attribute set, before any capture begins).  Callers on
// several threads (the server's, the user's) raise it under one lock, so it
// never goes down.
int g_smem_granted = 48 * 1024;
std::mutex g_smem_mu;

int ensure_smem(size_t smem) {
  std::lock_guard<std::mutex> lk(g_smem_mu);
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
  const size_t smem = mpld::kernel_head_bytes(warps_per_cta) +
                      (size_t)warps_per_cta * (size_t)(a->slot_bytes > 0 ? a->slot_bytes : 0);
  if (mpld::ensure_smem(smem) != MPLD_OK) return MPLD_E_CUDA;
  mpld::mpld_search_kernel<<<ctas, warps_per_cta * 32, smem, (cudaStream_t)stream>>>(*a);
  return cudaGetLastError() == cudaSuccess ? MPLD_OK : MPLD_E_CUDA;
}

// The same launch, allowed to start before the kernel before it on the stream
// completes (programmatic stream serialization): its blocks are scheduled as
// that kernel's blocks leave SMs.  Only for a kernel that reads nothing the
// previous one writes and waits for it before it exits (par == 4).
extern "C" int mpld_internal_launch_overlapped(const LaunchArgs *a, int ctas, int warps_per_cta,
                                              void *stream) {
  const size_t smem = mpld::kernel_head_bytes(warps_per_cta) +
                      (size_t)warps_per_cta * (size_t)(a->slot_bytes > 0 ? a->slot_bytes : 0);
  if (mpld::ensure_smem(smem) != MPLD_OK) return MPLD_E_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3((unsigned)(warps_per_cta * 32));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const LaunchArgs args = *a;
  return cudaLaunchKernelEx(&cfg, mpld::mpld_search_kernel, args) == cudaSuccess ? MPLD_OK
                                                                                 : MPLD_E_CUDA;
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
  const int avail = optin - (int)mpld::kernel_head_bytes(warps_per_cta);
  return (avail / warps_per_cta) & ~15;
}

extern "C" int mpld_internal_ctas_per_sm(int warps_per_cta, int slot_bytes) {
  const size_t smem =
      mpld::kernel_head_bytes(warps_per_cta) + (size_t)warps_per_cta * (size_t)slot_bytes;
  if (mpld::ensure_smem(smem) != MPLD_OK) return 0;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, mpld::mpld_search_kernel,
                                                    warps_per_cta * 32, smem) != cudaSuccess)
    return 0;
  return blocks;
}

// ---- budgeted split search: the lanes' subtrees ---------------------------
//
// A kernel of its own, so that its threads can have fewer registers than the
// warp searches need and twice as many warps fit an SM: every thread takes
// (hard-list entry, subtree) items of the lanes' list from counter queue[1]
// and searches each subtree alone (lane_search); the thread that completes an
// instance's last subtree replays the winning subtree and writes the result.

namespace mpld {
namespace {

// threads per block and resident blocks per SM the lane kernel is built for
constexpr int LANE_BLOCK = 1024, LANE_BLOCKS_PER_SM = 1;

__global__ void __launch_bounds__(LANE_BLOCK, LANE_BLOCKS_PER_SM)
    mpld_lane_kernel(const LaunchArgs a) {
  if (a.lane_phase1) {
    // the budgeted split search's first search of the per-lane instances
    // desc[order[0..n_inst)], one per thread: instance l * W + w goes to lane
    // l of warp w (W warps in the grid), so each warp holds about n_inst / W
    // of them; written as the warps' first search writes them.  This launch
    // may run beside the warps' first searches launched before it, and
    // completes only after them.
    const uint32_t W = gridDim.x * (blockDim.x >> 5);
    const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (uint32_t i = (threadIdx.x & 31u) * W + gw; i < (uint32_t)a.n_inst; i += 32u * W) {
      const InstDesc d = a.desc[a.order[i]];
      int D;
      uint32_t S;
      split_cut(d.n, d.k, D, S);
      LaneOut o;
      lane_dispatch(d, a.rule, 0, 0u, INF32, split_search_budget(a.budget, S), a.time_limit_ns,
                    globaltimer(), D, o);
      if (o.found)
        for (int v = 0; v < d.n; ++v)
          d.mask[v] = (int8_t)(((o.m0 >> v) & 1ull) | (((o.m1 >> v) & 1ull) << 1));
      const int st = o.timed_out ? MPLD_TIMEOUT : o.hit ? MPLD_BUDGET : MPLD_OK;
      d.res->cost = o.found ? (int64_t)o.best : INT64_MAX;
      d.res->nodes = o.nodes;
      d.res->status = st;
      d.res->sub = (int32_t)o.sub;
      d.res->work = o.work;
      if (st == MPLD_BUDGET) split_enlist(a, d, o.best, o.sub);
    }
    wait_prerequisites();
    return;
  }
  // the warps' subtree launch that follows may take SMs as these blocks finish
  launch_dependents();
  uint32_t HL = (uint32_t)*(volatile int32_t *)(a.hard + 1);
  if (HL == 0) return;
  const int32_t *list_l = a.hard + 4 + a.hard_cap;
  const uint64_t total = (uint64_t)HL * (uint64_t)a.smax;
  for (;;) {
    const uint32_t t = atomicAdd(a.queue + 1, 1u);
    if ((uint64_t)t >= total) break;
    const uint32_t j = t / (uint32_t)a.smax, s = t % (uint32_t)a.smax;
    const int di = __ldcg(list_l + j);
    const InstDesc d = a.desc[di];
    int D;
    uint32_t S;
    split_cut(d.n, d.k, D, S);
    if (s >= S) continue;
    ParCtx *ctx = (ParCtx *)(a.par_buf + (size_t)di * 64);
    const int64_t b = split_search_budget(a.budget, S);
    const int64_t c1 = __ldcg(&d.res->cost);
    const uint32_t s1 = (uint32_t)__ldcg(&d.res->sub);
    const unsigned long long key1 = ((unsigned long long)(uint32_t)c1 << 32) | s1;
    // the time limit runs from the instance's start
    const uint64_t now = globaltimer();
    const unsigned long long prev = atomicCAS(&ctx->t0, 0ull, (unsigned long long)now);
    const uint64_t t0 = prev != 0ull ? (uint64_t)prev : now;
    LaneOut o;
    lane_dispatch(d, a.rule, D, s, (int32_t)c1 + (s < s1 ? 1 : 0), b, a.time_limit_ns, t0, 0, o);
    unsigned long long *slot = a.lane_masks + 2u * ((size_t)j * (size_t)a.smax + s);
    if (o.found) {
      slot[0] = o.m0;
      slot[1] = o.m1;
      atomicMin(&ctx->key, ((unsigned long long)(uint32_t)o.best << 32) | s);
    }
    atomicAdd(&ctx->nodes, (unsigned long long)o.nodes);
    atomicAdd(&ctx->work, (unsigned long long)o.work);
    if (o.timed_out) atomicExch(&ctx->timed_out, 1u);
    if (o.hit) atomicExch(&ctx->pad, 1u);
    __threadfence();
    if (atomicAdd(&ctx->done, 1u) != S - 1u) continue;
    // this thread completed the instance's last subtree
    __threadfence();
    const unsigned long long key = *(volatile unsigned long long *)&ctx->key;
    if (key != key1) {
      // the winning subtree's leaf (its item wrote the slot before counting
      // itself done): mask of segment v = bit v of word 0 + 2 * bit v of word 1
      const unsigned long long *w =
          a.lane_masks + 2u * ((size_t)j * (size_t)a.smax + (size_t)(key & 0xFFFFFFFFull));
      const unsigned long long w0 = __ldcg(w), w1 = __ldcg(w + 1);
      for (int v = 0; v < d.n; ++v)
        d.mask[v] = (int8_t)(((w0 >> v) & 1ull) | (((w1 >> v) & 1ull) << 1));
    }
    split_write_result(d, ctx, key, true);
  }
}

}  // namespace
}  // namespace mpld

namespace {
int lane_blocks() {
  static int blocks = 0;   // resident blocks of the lane kernel (one query per process)
  if (blocks == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mpld::mpld_lane_kernel,
                                                      mpld::LANE_BLOCK, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    blocks = per_sm * std::max(1, mpld_internal_num_sms());
  }
  return blocks;
}
}  // namespace

extern "C" int mpld_internal_launch_lanes(const LaunchArgs *a, void *stream) {
  mpld::mpld_lane_kernel<<<lane_blocks(), mpld::LANE_BLOCK, 0, (cudaStream_t)stream>>>(*a);
  return cudaGetLastError() == cudaSuccess ? MPLD_OK : MPLD_E_CUDA;
}

// The lane kernel allowed to start before the kernel before it completes
// (programmatic stream serialization; the per-lane first searches beside
// the warps' first searches, which read and write other instances), with
// `blocks` blocks (0: one per resident place).
extern "C" int mpld_internal_launch_lanes_overlapped(const LaunchArgs *a, int blocks,
                                                    void *stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(blocks > 0 ? blocks : lane_blocks()));
  cfg.blockDim = dim3((unsigned)mpld::LANE_BLOCK);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const LaunchArgs args = *a;
  return cudaLaunchKernelEx(&cfg, mpld::mpld_lane_kernel, args) == cudaSuccess ? MPLD_OK
                                                                               : MPLD_E_CUDA;
}

// ---- search of one instance without allocating --------------------------
//
// For callers that may not allocate device memory (see
// mpld_search_instance_noalloc in mpld.h).  The packed instance and its
// search state live in one file-scope device array; the host half below
// looks its device address up once per device and passes it to the kernel.
// Layout of the array: [0, 256) status word; then the read-only block of
// the instance; then its mutable search state.

#include <stddef.h>

namespace mpld {
namespace {

static __device__ __align__(256) uint8_t g_noalloc_scratch[MPLD_NOALLOC_SCRATCH_BYTES];

constexpr uint32_t NOALLOC_CTRL = 256;

__host__ __device__ __forceinline__ uint32_t align256(uint32_t x) { return (x + 255u) & ~255u; }

static_assert(sizeof(mpld_instance_result) == sizeof(InstResult), "result layout");
static_assert(offsetof(mpld_instance_result, cost) == offsetof(InstResult, cost), "result layout");
static_assert(offsetof(mpld_instance_result, nodes) == offsetof(InstResult, nodes), "result layout");
static_assert(offsetof(mpld_instance_result, status) == offsetof(InstResult, status), "result layout");
static_assert(offsetof(mpld_instance_result, device_error) == offsetof(InstResult, sub), "result layout");
static_assert(offsetof(mpld_instance_result, work) == offsetof(InstResult, work), "result layout");

// One warp: check and pack the caller's adjacency into the array, then run
// the same instance search as the batched and plain kernels.
__global__ void __launch_bounds__(32, 1)
    mpld_noalloc_kernel(const mpld_device_instance inst, uint8_t *scratch, int8_t *mask_out,
                        InstResult *res_out, int64_t budget, int64_t time_limit_ns,
                        int slot_bytes) {
  const int lane = threadIdx.x & 31;
  const int n = inst.n, ne2 = inst.n_conf_entries, ns2 = inst.n_stitch_entries;
  const RoLayout R = ro_layout(n, ne2, ns2);
  uint8_t *ro = scratch + NOALLOC_CTRL;
  uint8_t *state = ro + align256(R.bytes);
  int32_t *err = (int32_t *)scratch;
  if (lane == 0) *err = 0;
  int2 *ptr = (int2 *)(ro + R.ptr);
  uint16_t *cn = (uint16_t *)(ro + R.cnbr);
  uint16_t *sn = (uint16_t *)(ro + R.snbr);
  bool bad = false;
  for (int v = lane; v <= n; v += 32) {
    const int c0 = inst.conf_ptr[v], s0 = inst.st_ptr[v];
    ptr[v] = make_int2(c0, s0);
    if (c0 < 0 || c0 > ne2 || s0 < 0 || s0 > ns2) bad = true;
    if (v == 0 && (c0 != 0 || s0 != 0)) bad = true;
    if (v == n && (c0 != ne2 || s0 != ns2)) bad = true;
    if (v == n || bad) continue;
    const int c1 = inst.conf_ptr[v + 1], s1 = inst.st_ptr[v + 1];
    if (c1 < c0 || c1 > ne2 || s1 < s0 || s1 > ns2) { bad = true; continue; }
    int prev = -1;
    for (int i = c0; i < c1; ++i) {   // ascending, in range, no self-loop
      const int u = inst.conf_nbr[i];
      if (u <= prev || u >= n || u == v) { bad = true; break; }
      cn[i] = (uint16_t)u;
      prev = u;
    }
    prev = -1;
    for (int i = s0; i < s1; ++i) {
      const int u = inst.st_nbr[i];
      if (u <= prev || u >= n || u == v) { bad = true; break; }
      sn[i] = (uint16_t)u;
      prev = u;
    }
  }
  // every edge must be listed from both ends: each entry u of v's list
  // needs v in u's list (binary search in the packed copies, whose ranges
  // and order were checked above)
  if (!__any_sync(FULL, bad)) {
    __syncwarp();
    for (int v = lane; v < n && !bad; v += 32) {
      const int2 p0 = ptr[v], p1 = ptr[v + 1];
      for (int i = p0.x; i < p1.x && !bad; ++i) {
        const int u = cn[i];
        int lo = ptr[u].x, hi = ptr[u + 1].x;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((int)cn[mid] < v) lo = mid + 1;
          else hi = mid;
        }
        bad = lo >= ptr[u + 1].x || (int)cn[lo] != v;
      }
      for (int i = p0.y; i < p1.y && !bad; ++i) {
        const int u = sn[i];
        int lo = ptr[u].y, hi = ptr[u + 1].y;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((int)sn[mid] < v) lo = mid + 1;
          else hi = mid;
        }
        bad = lo >= ptr[u + 1].y || (int)sn[lo] != v;
      }
    }
  }
  if (__any_sync(FULL, bad)) {
    if (lane == 0) {
      res_out->cost = INT64_MAX;
      res_out->nodes = 0;
      res_out->status = MPLD_E_INVALID;
      res_out->sub = 0;
      res_out->work = 0;
    }
    return;
  }
  // the packed block is read next by the bulk-copy engine (async proxy)
  __threadfence();
  asm volatile("fence.proxy.async;" ::: "memory");
  __syncwarp();
  uint64_t *bar = (uint64_t *)g_smem;
  if (lane == 0) mbar_init(bar);
  __syncwarp();
  if (lane == 0) fence_proxy_async();
  __syncwarp();
  InstDesc d;
  d.ro = ro;
  d.scratch = state;
  d.mask = mask_out;
  d.res = res_out;
  d.n = n;
  d.maxdeg = 0x7FFFFFFF;   // unknown: no small-instance specialisation
  d.ne2 = ne2;
  d.ns2 = ns2;
  d.ro_bytes = (int32_t)R.bytes;
  d.state_bytes = (int32_t)search_state_bytes(n, ne2, inst.k);
  d.k = inst.k;
  d.cost_conflict = inst.cost_conflict;
  d.cost_stitch = inst.cost_stitch;
  d.nq = 0;
  d.idx = 0;
  d.pad1 = 0;
  LaunchArgs a;
  a.desc = nullptr;
  a.order = nullptr;
  a.n_inst = 1;
  a.slot_bytes = slot_bytes;
  a.queue = nullptr;
  a.err = err;
  a.budget = budget;
  a.time_limit_ns = time_limit_ns;
  a.rule = 0;
  a.n_large = 0;
  a.par = 0;
  a.split = 0;
  a.par_buf = nullptr;
  uint32_t phase = 0;
  const uint32_t slot_off = align16(8u);
  if (d.k == 3) run_instance<uint8_t, 3>(d, slot_off, slot_bytes, bar, phase, a, lane);
  else if (d.k == 4) run_instance<uint8_t, 4>(d, slot_off, slot_bytes, bar, phase, a, lane);
  else if (d.k == 2) run_instance<uint8_t, 2>(d, slot_off, slot_bytes, bar, phase, a, lane);
  else if (d.k <= 7) run_instance<uint8_t, 8>(d, slot_off, slot_bytes, bar, phase, a, lane);
  else run_instance<uint16_t, 8>(d, slot_off, slot_bytes, bar, phase, a, lane);
  // the status word (a bulk copy that did not land in time: the search then
  // ran from the array instead, and its result stands)
  __syncwarp();
  if (lane == 0) res_out->sub = *(volatile int32_t *)err;
}

// Per-device set-up of the allocation-free path: the array's device address
// and the kernel's shared-memory limit.
struct NoallocDevice {
  bool ready = false;
  uint8_t *scratch = nullptr;
  int max_slot = 0;
};
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

}  // namespace
}  // namespace mpld

extern "C" int mpld_search_instance_noalloc(const mpld_device_instance *inst,
                                            const mpld_params *prm, int8_t *mask_out,
                                            mpld_instance_result *result_out, void *stream) {
  using namespace mpld;
  if (!inst || !mask_out || !result_out || !inst->conf_ptr || !inst->st_ptr) return MPLD_E_INVALID;
  if (prm && (prm->flags & MPLD_COLUMN_BFS)) return MPLD_E_INVALID;  // no breadth-first ranks here
  if (prm && (prm->flags & MPLD_PARALLEL_EXACT)) return MPLD_E_INVALID;  // one warp per instance
  if (prm && (prm->flags & MPLD_SPLIT_BUDGET)) return MPLD_E_INVALID;    // no second launch here
  const int n = inst->n, k = inst->k, ne2 = inst->n_conf_entries, ns2 = inst->n_stitch_entries;
  if (n < 1 || k < 2 || k > 8 || ne2 < 0 || ns2 < 0) return MPLD_E_INVALID;
  if ((ne2 > 0 && !inst->conf_nbr) || (ns2 > 0 && !inst->st_nbr)) return MPLD_E_INVALID;
  if (inst->cost_conflict < 0 || inst->cost_conflict > 10000 || inst->cost_stitch < 0 ||
      inst->cost_stitch > 10000)
    return MPLD_E_INVALID;
  if (n > MPLD_MAX_INSTANCE_SEGMENTS) return MPLD_E_TOO_LARGE;
  // every adjacency entry takes at least two bytes of the array: larger
  // entry counts cannot fit, and below this bound the 32-bit layout sums
  // further down cannot wrap
  if ((int64_t)ne2 > (int64_t)(MPLD_NOALLOC_SCRATCH_BYTES / 2) ||
      (int64_t)ns2 > (int64_t)(MPLD_NOALLOC_SCRATCH_BYTES / 2))
    return MPLD_E_TOO_LARGE;
  // row keys and path costs are 32-bit in the kernel (bound without degrees)
  if ((int64_t)inst->cost_conflict * ne2 + (int64_t)inst->cost_stitch * ns2 >= ((int64_t)1 << 28))
    return MPLD_E_TOO_LARGE;
  const RoLayout R = ro_layout(n, ne2, ns2);
  if ((uint64_t)NOALLOC_CTRL + align256(R.bytes) + search_state_bytes(n, ne2, k) >
      (uint64_t)MPLD_NOALLOC_SCRATCH_BYTES)
    return MPLD_E_TOO_LARGE;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MPLD_E_CUDA;
  NoallocDevice *nd;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    nd = &g_noalloc_dev[dev];
    if (!nd->ready) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return MPLD_E_CUDA;
      }
      int optin = 0;
      if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
              cudaSuccess ||
          cudaFuncSetAttribute(mpld_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin) != cudaSuccess) {
        cudaGetLastError();
        return MPLD_E_CUDA;
      }
      nd->scratch = (uint8_t *)p;
      nd->max_slot = (optin - (int)align16(8u)) & ~15;
      nd->ready = true;
    }
  }
  const uint32_t fp = align16(search_footprint(n, ne2, ns2, k));
  const int slot = (int)fp <= nd->max_slot ? (int)fp : 0;   // else state stays in the array
  const int64_t budget = prm ? (prm->node_budget > 0 ? prm->node_budget : 0) : 0;
  const int64_t tl = (prm && prm->time_limit_ms > 0 ? prm->time_limit_ms : 60000) * 1000000ll;
  // an error left pending by earlier work of the caller stays the caller's:
  // nothing is launched, and the error is not consumed here
  if (cudaPeekAtLastError() != cudaSuccess) return MPLD_E_CUDA;
  mpld_noalloc_kernel<<<1, 32, align16(8u) + (size_t)slot, (cudaStream_t)stream>>>(
      *inst, nd->scratch, mask_out, reinterpret_cast<InstResult *>(result_out), budget, tl, slot);
  return cudaGetLastError() == cudaSuccess ? MPLD_OK : MPLD_E_CUDA;
}
