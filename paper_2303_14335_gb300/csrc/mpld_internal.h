// mpld_internal.h -- layout shared by the host builder (mpld_host.cpp) and the
// search kernels (mpld_search.cu).  Not part of the public ABI.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define MPLD_HD __host__ __device__ __forceinline__
#else
#define MPLD_HD inline
#endif

namespace mpld {

// Rows of the EC matrix (Sec. 2.3): the activeRows bitset holds one field of
// FB bits per segment v (FB = 8 for k <= 7, 16 for k = 8).  Bit c < k of
// field v is row (v, c); the top bit of the field is set while primary
// column P_v is uncovered (the column-header bit).  The k row bits of field
// v are the row set of P_v; secondary column S_{e,c} of conflict edge
// e = (u, w) is bit c of fields u and w.  Columns are therefore one- or
// two-bit masks generated from the conflict adjacency below, which is the
// block-sparse form of the column-major bitset matrix colRows[j][W].
MPLD_HD int field_bytes_for(int k) { return k <= 7 ? 1 : 2; }
MPLD_HD int mk_for(int k) { return k <= 4 ? 4 : 8; }   // width of the row sort
MPLD_HD uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// Read-only block of one instance, 16-byte aligned in the device arena and
// copied as one piece into shared memory (cp.async.bulk for large blocks):
//   ptr[n+1]  int2    {conflict CSR offset, stitch CSR offset} per segment
//   cnbr[ne2] uint16  conflict neighbours (component-local), ascending
//   snbr[ns2] uint16  stitch neighbours, ascending
//   rank[n]   uint16  breadth-first rank of each segment over conflict and
//                     stitch edges (roots ascending, neighbours ascending)
//   order[n]  uint16  segment of each breadth-first rank
//   qptr[n+1] int32   (nq > 0 only) each segment's range in qlist
//   qlist[nq*(k+1)] uint16  the bound's cliques holding each segment
//   bits[2n]  uint64  (n <= 64 only) each segment's conflict neighbours as a
//                     bit mask, then its stitch neighbours (the per-lane search)
// (rank / order serve the paper's column rule, Algorithm 1: a column with a
// single row left, else the first uncovered column in BFS order of G; the
// clique lists serve the second bound mode.)
struct RoLayout {
  uint32_t ptr, cnbr, snbr, rank, order, qptr, qlist, bits, bytes;
};
constexpr int LANE_MAX_N = 64;   // the per-lane search's largest instance
MPLD_HD RoLayout ro_layout(int n, int ne2, int ns2, int nqe = 0) {
  RoLayout L;
  uint32_t o = 0;
  L.ptr = o; o += align16(8u * (uint32_t)(n + 1));
  L.cnbr = o; o += align16(2u * (uint32_t)ne2);
  L.snbr = o; o += align16(2u * (uint32_t)ns2);
  L.rank = o; o += align16(2u * (uint32_t)n);
  L.order = o; o += align16(2u * (uint32_t)n);
  L.qptr = o; o += nqe > 0 ? align16(4u * (uint32_t)(n + 1)) : 0u;
  L.qlist = o; o += align16(2u * (uint32_t)nqe);
  L.bits = o; o += n <= LANE_MAX_N ? align16(16u * (uint32_t)n) : 0u;
  L.bytes = o;
  return L;
}
// Shared memory of the column classes a giant instance is searched with
// (one warp): per count class a bit per segment, its summary and its size,
// and the breadth-first rank map with its summary.
MPLD_HD uint32_t bucket_bytes(int n, int k) {
  const uint32_t w = (uint32_t)(n + 31) / 32u, sw = (w + 31u) / 32u;
  return 4u * ((uint32_t)(k + 1) * (w + sw + 1u) + w + sw);
}

// Instances the second phase of the budgeted split search gives to single
// lanes (a subtree per lane, the whole state in registers as one bit per
// segment); larger ones, or k > 4, to whole warps.
MPLD_HD bool lane_fits(int n, int k) { return n <= LANE_MAX_N && k <= 4; }


// Mutable search state of one instance (shared memory, or the instance's
// global scratch region when it does not fit the warp's slot).  The DFS
// depth is at most n; undo data is kept per segment and per adjacency entry
// because each segment appears at most once on the current path.
//   lv[n]       32-byte level record {path cost, v | rows tried << 16,
//               visiting order (4 bits per row), conflict offset, conflict
//               degree | stitch degree << 16, stitch offset, added cost of
//               rows 1 and 2}
//   lvx[n*mk]   added cost of rows 3.. in visiting order
//   ccnt[n*cw]  per segment, 16-bit counts of conflict neighbours holding
//               each mask (cw = mk/4 64-bit words)
//   scnt[n*cw]  the same for stitch neighbours
//   rows[n]     FB-bit fields: activeRows + uncovered-column bits (padded
//               with zero fields to a multiple of 4 bytes)
//   oldf[n]     field of v before v's row was covered
//   x[n]        i8   current mask per segment (-1 = none)
//   savf[ne2]   field of neighbour u before v's row cleared its bit (the
//               undo record of the cover, one per adjacency entry of v)
//   qcnt[nq]    u8 per clique of the second bound mode: members assigned
//   qlev[n]     (nq > 0 only) per level, the cliques its segment's
//               assignment took out of the untouched count
struct StateLayout {
  uint32_t lv, lvx, ccnt, scnt, rows, oldf, x, savf, qcnt, qlev, bytes;
};
MPLD_HD StateLayout state_layout(int n, int ne2, int k, int nq = 0) {
  const uint32_t fb = (uint32_t)field_bytes_for(k), mk = (uint32_t)mk_for(k), cw = mk / 4u;
  StateLayout L;
  uint32_t o = 0;
  L.lv = o; o += 32u * (uint32_t)n;
  L.lvx = o; o += align16(4u * mk * (uint32_t)n);
  L.ccnt = o; o += align16(8u * cw * (uint32_t)n);
  L.scnt = o; o += align16(8u * cw * (uint32_t)n);
  L.rows = o; o += align16(fb * (uint32_t)n);
  L.oldf = o; o += align16(fb * (uint32_t)n);
  L.x = o; o += align16((uint32_t)n);
  L.savf = o; o += align16(fb * (uint32_t)ne2);
  L.qcnt = o; o += align16((uint32_t)nq);
  L.qlev = o; o += nq > 0 ? align16(4u * (uint32_t)n) : 0u;
  L.bytes = o;
  return L;
}

// Register-resident search, for instances of at most 32 words of fields
// (n <= 128 for byte fields, n <= 64 for k = 8): lane l keeps the fields of
// segments 4l..4l+3 (2l..2l+1 for k = 8) in one register, so the column
// scan and the covers touch no memory.  Per-warp state:
//   adj[n*32]    u8   per (segment v, lane l): bit j = segment l*P+j is a
//                     conflict neighbour of v; bit 4+j = a stitch neighbour
//   deg[n]       u32  conflict degree | stitch degree << 16
//   rec[(n+1)*rs]     level record {v | next row << 8 | v's field << 12,
//                     path cost, degrees, -, sorted row keys}; rs = 32 bytes
//                     for k <= 4, else 48
//   sav[(n+1)*32] u16 per (level, lane): which neighbour fields of the lane
//                     lost a row bit to the level's cover (bits 0-3), and
//                     the lane's conflict (bits 4-7) and stitch (bits 8-11)
//                     neighbour bits of the level's segment
//   qptr[n+1]    u16  (nq > 0 only) clique ranges, copied from the block
//   qlist[nq*(k+1)] u16  cliques holding each segment
//   qcnt[nq]     u8   members of each clique assigned
//   bestx[n]     i8   parallel exact search: this warp's best masks
struct RegLayout {
  uint32_t adj, deg, rec, sav, qptr, qlist, qcnt, bestx, bytes;
};
MPLD_HD bool reg_fits(int n, int k) { return n <= 32 * (4 / field_bytes_for(k)); }
MPLD_HD RegLayout reg_layout(int n, int k, int nq = 0) {
  const uint32_t rs = k <= 4 ? 32u : 48u;
  const uint32_t nqe = (uint32_t)nq * (uint32_t)(k + 1);
  RegLayout L;
  uint32_t o = 0;
  L.adj = o; o += align16(32u * (uint32_t)n);
  L.deg = o; o += align16(4u * (uint32_t)n);
  L.rec = o; o += rs * (uint32_t)(n + 1);
  L.sav = o; o += 64u * (uint32_t)(n + 1);
  L.qptr = o; o += nq > 0 ? align16(2u * (uint32_t)(n + 1)) : 0u;
  L.qlist = o; o += align16(2u * nqe);
  L.qcnt = o; o += align16((uint32_t)nq);
  L.bestx = o; o += align16((uint32_t)n);
  L.bytes = o;
  return L;
}

// Global scratch an instance needs when its state does not fit a slot, and
// its shared-memory footprint when it does (nq: cliques of the second bound
// mode, 0 without it).  The scratch holds either layout: an instance small
// enough for the register search is still searched with the general layout
// when a whole CTA takes it.
MPLD_HD uint32_t search_state_bytes(int n, int ne2, int k, int nq = 0) {
  const uint32_t general = state_layout(n, ne2, k, nq).bytes;
  const uint32_t reg = reg_fits(n, k) ? reg_layout(n, k, nq).bytes : 0u;
  return general > reg ? general : reg;
}
MPLD_HD uint32_t search_footprint(int n, int ne2, int ns2, int k, int nq = 0) {
  return reg_fits(n, k) ? reg_layout(n, k, nq).bytes
                        : state_layout(n, ne2, k, nq).bytes +
                              ro_layout(n, ne2, ns2, nq * (k + 1)).bytes;
}

// One search instance, as the kernel sees it (absolute device pointers so
// that instances of several problems can share one launch).
struct __align__(16) InstDesc {
  const uint8_t *ro;       // read-only block (16-byte aligned)
  uint8_t *scratch;        // global state region (state_bytes), used when spilled
  int8_t *mask;            // n bytes: best assignment found
  struct InstResult *res;  // result record
  int32_t n, maxdeg, ne2, ns2;   // maxdeg: largest conflict degree | largest stitch degree << 16
  int32_t ro_bytes, state_bytes;
  int32_t k, cost_conflict;
  int32_t cost_stitch, nq;   // nq: cliques of the second bound mode (0: none)
  int32_t idx;               // position in the launch's descriptor array
  int32_t pad1;
};

struct InstResult {
  int64_t cost;
  int64_t nodes;
  int32_t status;   // MPLD_OK / MPLD_BUDGET / MPLD_TIMEOUT, -1 = not run
  int32_t sub;      // budgeted split search: subtree of the incumbent's leaf
  // algorithmic integer operations of the search: 2 per uncovered column at
  // every node that scans the columns (AND + popcount of the column choice;
  // a node pruned by its path cost alone scans nothing), k per neighbour
  // when a node's rows are costed, 5 per column of every covered row
  // (AND-NOT, undo record, restore) -- the work the method must do,
  // independent of how the kernel packs it
  int64_t work;
};

struct LaunchArgs {
  const InstDesc *desc;
  const int32_t *order;    // instance indices, largest first
  int32_t n_inst;
  int32_t slot_bytes;      // shared memory per warp
  uint32_t *queue;         // work counters [small, large]; NULL = static assignment
  int32_t *err;            // device status word (0 = fine)
  int64_t budget;
  int64_t time_limit_ns;
  int32_t rule;            // column rule: 0 fewest rows, 1 single row else BFS order
  int32_t n_large;         // the first n_large instances of the order are searched by whole
                           // CTAs (blocks 0..n_large-1 first; counter queue[1])
  int32_t par;             // 1: those CTAs search exactly, their warps splitting subtrees;
                           // 2: every warp of the grid splits the one instance desc[0];
                           // 3: the grid splits desc[order[0..n_inst)] one after another;
                           // 4: budgeted split search, second phase: the warps of the
                           //    grid search the subtrees of the instances on the hard list
  int32_t split = 0;       // 1: budgeted split search, first phase: each instance searched
                           // with its per-search budget; one that stops on it goes on the
                           // hard list with a fresh context
  uint8_t *par_buf;        // par == 2: the split context in global memory (ParLayout);
                           // par == 3: one 64-byte context per queued instance;
                           // split / par == 4: one 64-byte context per descriptor index
  int32_t *hard = nullptr; // split / par == 4: entry counts of the three hard lists (warps,
                           // lanes, warps with general state) at [0..2], then hard_cap
                           // descriptor indices of each list from [4] on (instances that
                           // stopped on their first-phase budget); contexts are per
                           // descriptor index
  int32_t hard_cap = 0;
  int32_t split_gen_warps = 0;   // par == 4: warps with a general-state region (the first)
  uint8_t *split_scratch = nullptr;  // par == 4: per-warp global search state for instances
                                     // beyond the register form (split_state_bytes per warp)
  int32_t smax = 0;        // par == 4: item numbers per hard-list entry (>= its subtrees)
  // par == 4: per item of the lanes' list (entry * smax + subtree), the masks
  // of its best leaf, two bits per segment as two words (bit 0, bit 1)
  unsigned long long *lane_masks = nullptr;
  // lane kernel: 1 = the budgeted split search's first search of the
  // per-lane instances desc[order[0..n_inst)] (0 = their subtrees)
  int32_t lane_phase1 = 0;
  int32_t split_state_bytes = 0;
};

// Budgeted split search (MPLD_SPLIT_BUDGET): an instance's search tree is cut
// at depth D, the first depth with k^D >= SPLIT_TARGET (at most n and 8),
// into S = k^D subtrees; the first search and every subtree search get
// b = ceil(B / (S + 1)) nodes of the instance's budget B.
constexpr int SPLIT_TARGET = 64;
// Instances of more than SPLIT_MAX_N segments are not split: one search with
// the whole budget (every subtree search would first descend through all
// their levels).
constexpr int SPLIT_MAX_N = 4096;
// Hard list of an instance: 1 = a lane per subtree, 0 = a warp per subtree
// with the register form, 2 = a warp with a general-state region.
MPLD_HD int split_list_of(int n, int k) { return lane_fits(n, k) ? 1 : reg_fits(n, k) ? 0 : 2; }
MPLD_HD void split_cut(int n, int k, int &D, uint32_t &S) {
  D = 0;
  S = 1;
  while (S < (uint32_t)SPLIT_TARGET && D < n && D < 8) {
    S *= (uint32_t)k;
    ++D;
  }
}
MPLD_HD int64_t split_search_budget(int64_t B, uint32_t S) {
  return B > 0 ? (B + (int64_t)S) / ((int64_t)S + 1) : 0;
}

// Shared state of a split exact search: the incumbent as one 64-bit key
// (cost << 32 | subtree; ~0 = none), the next subtree to hand out, and
// totals.  In shared memory for a CTA's warps, in global memory for a grid.
struct ParCtx {
  unsigned long long key;
  unsigned long long nodes, work;
  uint32_t next;
  uint32_t timed_out;
  uint32_t done;           // warps (or, in the queue, subtrees) finished
  uint32_t pad;
  unsigned long long t0;   // %globaltimer when the first warp started on the
                           // instance (0 = not yet): the time limit runs from
                           // there for every warp, however late it joins
};
static_assert(sizeof(ParCtx) <= 64, "queue contexts are 64 bytes apart");

// Global-memory block of the grid form for G warps and an n-segment
// instance: each warp's best key, the context, each warp's best masks.
struct ParLayout {
  uint32_t wkey, ctx, bestx, row, bytes;
};
MPLD_HD ParLayout par_layout(int G, int n) {
  ParLayout L;
  L.wkey = 0;
  L.ctx = (uint32_t)align16(8u * (uint32_t)G);
  L.bestx = L.ctx + (uint32_t)align16(sizeof(ParCtx));
  L.row = (uint32_t)align16((uint32_t)n);
  L.bytes = L.bestx + (uint32_t)G * L.row;
  return L;
}

}  // namespace mpld

// Host-side launch wrappers implemented in mpld_search.cu.
extern "C" int mpld_internal_launch(const mpld::LaunchArgs *a, int ctas, int warps_per_cta,
                                    void *stream);
extern "C" int mpld_internal_max_slot_bytes(int warps_per_cta);
extern "C" int mpld_internal_ctas_per_sm(int warps_per_cta, int slot_bytes);
extern "C" int mpld_internal_num_sms(void);
// The budgeted split search's per-lane subtree searches (the lanes' hard list).
extern "C" int mpld_internal_launch_lanes(const mpld::LaunchArgs *a, void *stream);
extern "C" int mpld_internal_launch_lanes_overlapped(const mpld::LaunchArgs *a, int blocks,
                                                    void *stream);
extern "C" int mpld_internal_launch_overlapped(const mpld::LaunchArgs *a, int ctas,
                                              int warps_per_cta, void *stream);
