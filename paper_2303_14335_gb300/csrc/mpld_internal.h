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

// Rows of the EC matrix (Sec. 2.3): row (v, c) is bit v*KP + c of the
// activeRows bitset, KP = 4 for k <= 4 and 8 for 5 <= k <= 8.  The KP bits
// of segment v form the row set of primary column P_v and always sit inside
// one 64-bit word; secondary column S_{e,c} of conflict edge e = (u, w) is
// the two bits u*KP + c and w*KP + c.  The columns are therefore one- or
// two-word masks generated from the conflict adjacency below, which is the
// block-sparse form of the column-major bitset matrix colRows[j][W].
MPLD_HD int kp_for(int k) { return k <= 4 ? 4 : 8; }
MPLD_HD int words_for(int n, int kp) { return (n * kp + 63) >> 6; }
MPLD_HD uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// Read-only block of one instance, 16-byte aligned in the device arena and
// copied as one piece into shared memory (cp.async.bulk for large blocks):
//   cptr[n+1] int32   conflict CSR offsets (component-local ids)
//   sptr[n+1] int32   stitch CSR offsets
//   cnbr[ne2] uint16  conflict neighbours, ascending per segment
//   snbr[ns2] uint16  stitch neighbours
struct RoLayout {
  uint32_t cptr, sptr, cnbr, snbr, bytes;
};
MPLD_HD RoLayout ro_layout(int n, int ne2, int ns2) {
  RoLayout L;
  uint32_t o = 0;
  L.cptr = o; o += align16(4u * (uint32_t)(n + 1));
  L.sptr = o; o += align16(4u * (uint32_t)(n + 1));
  L.cnbr = o; o += align16(2u * (uint32_t)ne2);
  L.snbr = o; o += align16(2u * (uint32_t)ns2);
  L.bytes = o;
  return L;
}

// Mutable search state of one instance (shared memory, or the instance's
// global scratch region when it does not fit the warp's slot).  The DFS
// depth is at most n, so every per-level array has n entries; undo data is
// kept per segment / per adjacency entry because each segment appears at
// most once on the current path.
//   active[W]   u64  activeRows
//   unas[W]     u64  KP-bit field all ones while segment v is uncovered
//   lv_g[n]     i64  path cost at each level
//   lv_inc[n*KP] i32 added cost of the level's rows, in visiting order
//   lv_ord[n]   u32  visiting order of the masks, 4 bits each
//   lv_v[n]     i32  segment (column) chosen at each level
//   lv_next[n]  u8   rows of the level already visited
//   x[n]        i8   current mask per segment (-1 = none)
//   oldnib[n]   u8   active rows of P_v before v's row was covered
//   clrb[ne2]   u8   1 if covering v's row cleared neighbour row (u, c)
struct StateLayout {
  uint32_t active, unas, lv_g, lv_inc, lv_ord, lv_v, lv_next, x, oldnib, clrb, bytes;
};
MPLD_HD StateLayout state_layout(int n, int W, int ne2, int kp) {
  StateLayout L;
  uint32_t o = 0;
  L.active = o; o += align16(8u * (uint32_t)W);
  L.unas = o; o += align16(8u * (uint32_t)W);
  L.lv_g = o; o += align16(8u * (uint32_t)n);
  L.lv_inc = o; o += align16(4u * (uint32_t)(n * kp));
  L.lv_ord = o; o += align16(4u * (uint32_t)n);
  L.lv_v = o; o += align16(4u * (uint32_t)n);
  L.lv_next = o; o += align16((uint32_t)n);
  L.x = o; o += align16((uint32_t)n);
  L.oldnib = o; o += align16((uint32_t)n);
  L.clrb = o; o += align16((uint32_t)ne2);
  L.bytes = o;
  return L;
}

// One search instance, as the kernel sees it (absolute device pointers so
// that instances of several problems can share one launch).
struct InstDesc {
  const uint8_t *ro;       // read-only block (16-byte aligned)
  uint8_t *scratch;        // global state region (state_bytes), used when spilled
  int8_t *mask;            // n bytes: best assignment found
  struct InstResult *res;  // result record
  int32_t n, W, ne2, ns2;
  int32_t ro_bytes, state_bytes;
  int32_t k, cost_conflict;
  int32_t cost_stitch, pad0;
  int64_t pad1;
};

struct InstResult {
  int64_t cost;
  int64_t nodes;
  int32_t status;   // MPLD_OK / MPLD_BUDGET / MPLD_TIMEOUT, -1 = not run
  int32_t pad0;
  // algorithmic integer operations of the search: 2 per uncovered column at
  // every node (AND + popcount of the column choice), k per neighbour when a
  // node's rows are costed, 5 per column of every covered row (AND-NOT,
  // undo record, restore) -- the work the method must do, independent of
  // how the kernel packs it
  int64_t work;
};

struct LaunchArgs {
  const InstDesc *desc;
  const int32_t *order;    // instance indices, largest first
  int32_t n_inst;
  int32_t slot_bytes;      // shared memory per warp
  uint32_t *queue;         // work counter; NULL = static assignment
  int32_t *err;            // device status word (0 = fine)
  int64_t budget;
  int64_t time_limit_ns;
};

}  // namespace mpld

// Host-side launch wrappers implemented in mpld_search.cu.
extern "C" int mpld_internal_launch(const mpld::LaunchArgs *a, int ctas, int warps_per_cta,
                                    void *stream);
extern "C" int mpld_internal_max_slot_bytes(int warps_per_cta);
extern "C" int mpld_internal_ctas_per_sm(int warps_per_cta, int slot_bytes);
extern "C" int mpld_internal_num_sms(void);
