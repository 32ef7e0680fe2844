// mpld_problem.h -- the problem handle of libmpld, shared by the host
// builder / launcher (mpld_host.cpp) and the serving loop (mpld_serve.cpp).
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <stdint.h>

#include <vector>

#include "../../include/mpld.h"
#include "mpld_internal.h"

namespace mpld {

struct GraphKey {
  int nw = 0, slot = 0, ctas = 0;
  int64_t budget = 0, tl = 0;
  int rule = 0, n_large = 0;
  int queue_ctas = 0, queue_slot = 0;  // the split-search queue launch before it (0 = none)
  int split_nw = 0, split_ctas = 0;    // the budgeted split search's second launch (0 = none)
  bool operator==(const GraphKey &o) const {
    return nw == o.nw && slot == o.slot && ctas == o.ctas && budget == o.budget && tl == o.tl &&
           rule == o.rule && n_large == o.n_large && queue_ctas == o.queue_ctas &&
           queue_slot == o.queue_slot && split_nw == o.split_nw && split_ctas == o.split_ctas;
  }
};

// Budgeted split search (MPLD_SPLIT_BUDGET): the device block and the second
// launch of a batched call (mpld_host.cpp; used by the server too).
struct SplitPlan {
  bool on = false;
  int nw = 0, slot = 0, ctas = 0;   // second launch
  int smax = 1;                     // item numbers per hard-list entry
  int state_bytes = 0;              // general-state region per warp (0: no such instance)
  int gen_warps = 0;                // warps with such a region (all warps when every
                                    // general-form state fits the slot)
  int cap = 0;                      // entries of each hard list (the launch's descriptors)
  size_t o_hard = 0, o_ctx = 0, o_state = 0, bytes = 0;
  size_t o_lmask = 0;               // best-leaf masks of the lanes' items (16 bytes each)
};
// Plan for the descriptors of one launch; the general-state regions take at
// most gen_cap_bytes (fewer warps get one).  on = false unless prm asks for
// the split search.
SplitPlan split_plan(const InstDesc *desc, int n_inst, const mpld_params *prm,
                     size_t gen_cap_bytes);
void split_phase1_args(LaunchArgs &a, const SplitPlan &q, uint8_t *buf);
int split_reset(const SplitPlan &q, uint8_t *buf, cudaStream_t st);
int split_phase2_launch(const LaunchArgs &a1, const InstDesc *desc, const SplitPlan &q,
                        uint8_t *buf, uint32_t *queue, cudaStream_t st);
// First phase: how many leading entries of the largest-first order h_order
// the warps' forms take (at least the n_large whole-CTA instances); every
// later entry is an instance of the per-lane form.  n when the order does
// not split that way (then the warps take every instance).
int split_warp_prefix(const InstDesc *h_desc, const int32_t *h_order, int n, int n_large);
// First phase over desc[order[0..a.n_inst)]: the warps' searches of the first
// n_w entries (at most ctas CTAs of nw warps), and the lane kernel's of the
// rest beside them.
int split_phase1_launch(const LaunchArgs &a, int ctas, int nw, int n_w, cudaStream_t st);

}  // namespace mpld

struct mpld_problem {
  int n_seg = 0, k = 0;
  int64_t Cc = 10, Cs = 1;
  uint32_t flags = 0;
  // normalised input
  std::vector<int32_t> cu, cv, su, sv;
  std::vector<int32_t> cptr, cadj;  // global conflict adjacency
  // simplification
  std::vector<int32_t> unit_of, uptr, useg, removed_order;
  int64_t n_removed_segments = 0;
  // sub-graphs (search instances)
  int n_comp = 0;
  std::vector<int32_t> comp_ptr, comp_seg, comp_of;
  std::vector<int32_t> inst_attach;   // biconnected blocks: attach segment's index, -1 first
  std::vector<int32_t> inst_ne2;
  std::vector<int32_t> inst_nq;       // cliques of the second bound mode per instance
  int max_component = 0;
  int64_t instance_segments = 0;
  // packed instances
  std::vector<uint8_t> h_arena;        // host copy of the read-only blocks
  std::vector<uint64_t> ro_off;
  std::vector<uint32_t> footprint;     // state + read-only bytes
  std::vector<mpld::InstDesc> h_desc;  // sizes filled; device pointers only when uploaded
  std::vector<int32_t> h_order;        // largest first
  // device memory: one allocation
  uint8_t *d_base = nullptr;
  size_t d_bytes = 0;
  uint8_t *d_arena = nullptr, *d_scratch = nullptr;
  size_t arena_bytes = 0, scratch_bytes = 0;
  mpld::InstDesc *d_desc = nullptr;
  int32_t *d_order = nullptr;
  mpld::InstResult *d_res = nullptr;
  int8_t *d_masks = nullptr;
  uint32_t *d_queue = nullptr;
  uint8_t *d_par = nullptr;           // grid-wide split search context (grown on demand)
  size_t par_bytes = 0;
  bool queue_ready = false;           // the queue's index arrays are in d_par
  uint8_t *d_split = nullptr;         // budgeted split search: hard list, contexts and the
  size_t split_bytes = 0;             // per-warp state of the second launch (grown on demand)
  int32_t *d_err = nullptr;
  // pinned host mirrors of the results
  mpld::InstResult *h_res = nullptr;
  int8_t *h_masks = nullptr;
  int32_t *h_err = nullptr;
  size_t mask_bytes = 0;
  bool searched = false;      // a search was enqueued since the last fetch
  bool have_results = false;  // a fetch completed
  bool results_copied = false;  // the enqueued work already copies results back
  std::vector<int64_t> r_nodes, r_cost;
  std::vector<int32_t> r_status;
  // captured launch sequence
  cudaGraphExec_t gexec = nullptr;
  mpld::GraphKey gkey;
  void *gstream = nullptr;
};

// Scatter per-instance results (instance order) into the layout, recover
// the removed segments, count conflicts and stitches; `err` is the device
// status word of the search.
int mpld_internal_finish(mpld_problem *p, const mpld::InstResult *res, const int8_t *masks,
                         int32_t err, int8_t *mask_out, mpld_result *out);
