// lrs_internal.h -- host-side structures shared by the translation units of
// liblrs (analysis, factorization, solve).  Not part of the public ABI.
#pragma once

#include <atomic>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lrs.h"

namespace lrs {

// Node naming (Def. Htree).  A node belongs to one cluster of the nested
// partitioning, named by its heap index h = 2^level + j.  At level i of
// Algorithm 1 the live nodes all belong to clusters of P_{i-1}: super-node
// s_j^[i], black-node b_j^[i] and red-node P(b_j^[i]) share cluster j of
// P_{i-1}.  The exported id is 4 h + kind with kind 0 red, 1 super, 2 black.
enum Kind : int { kRed = 0, kSuper = 1, kBlack = 2 };

inline int32_t heap_of(int level, int32_t j) { return (int32_t(1) << level) + j; }
inline int32_t export_id(int32_t heap, int kind) { return heap * 4 + kind; }

// Within level i the runtime names nodes locally: 3 j + slot, slot 0 for the
// super-node, 1 for the black-node, 2 for the red parent of cluster j.
enum Slot : int { kSlotS = 0, kSlotB = 1, kSlotP = 2 };
inline int32_t local_node(int32_t j, int slot) { return 3 * j + slot; }
inline int32_t local_cluster(int32_t v) { return v / 3; }
inline int local_slot(int32_t v) { return v % 3; }

struct LevelPlan {
  int level = 0;                                // i, from l down to 1
  int32_t nsuper = 0;                           // 2^(i-1)
  // super-super interaction edges when the level starts (after the merge),
  // as pairs of cluster indices (a, b), a != b, each unordered pair once
  std::vector<std::pair<int32_t, int32_t>> merge_edges;
  std::vector<std::vector<int32_t>> batches;    // cluster indices j of each batch
  // per super-node j (local node names):
  std::vector<std::vector<int32_t>> ws;         // well-separated neighbours at Compress
  std::vector<std::vector<int32_t>> nbs;        // neighbours of s at Eliminate(s)
  std::vector<std::vector<int32_t>> nbb;        // neighbours of b at Eliminate(b)
};

}  // namespace lrs

struct lrs_plan {
  int64_t n = 0, nnz = 0;
  int dim = 0;
  int depth = 0;                                // l
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colind;
  std::vector<int32_t> perm;                    // position -> original index
  std::vector<int32_t> pos;                     // original index -> position
  std::vector<int32_t> leaf_off;                // 2^l + 1
  std::vector<int32_t> leaf_of;                 // original index -> leaf cluster
  // cluster adjacency of every level, CSR over clusters (Def. adj)
  std::vector<std::vector<int32_t>> cadj_ptr, cadj;
  std::vector<lrs::LevelPlan> levels;           // levels[0] is level l
  // leaf assembly: for nonzero e, the leaf super-node block (index into
  // levels[0] block list, see factor) and the element offset inside it
  std::vector<int32_t> nz_block;
  std::vector<int32_t> nz_elem;
  // for entry e = (i, j): the index of entry (j, i); empty when the pattern
  // is not symmetric
  std::vector<int64_t> tpos;
  // instances of the batched form (one for lrs_analyze): rows
  // [inst_row_off[k], inst_row_off[k+1]) of the union are instance k, whose
  // depth inst_depth[k] subtree has leaves from inst_leaf_base[k]
  std::vector<int64_t> inst_row_off;
  std::vector<int64_t> inst_leaf_base;
  std::vector<int> inst_depth;
  int min_dist = 2;                             // well-separated: cluster distance >= this
  // references: the caller's handle plus one per factor built on the plan
  // (a factor reads the plan until it is destroyed); freed at zero
  mutable std::atomic<int> refs{1};
  bool cluster_adjacent(int level, int32_t a, int32_t b) const;
  bool well_separated(int level, int32_t a, int32_t b) const;
};

namespace lrs {
// Drops one reference of a plan; the last one frees it.
inline void unref_plan(const lrs_plan* plan) {
  if (plan && plan->refs.fetch_sub(1, std::memory_order_acq_rel) == 1) delete plan;
}
// analyze.cpp
int analyze(const lrs_csr* A, const lrs_analyze_opts* opts, lrs_plan** out);
int analyze_batch(int count, const lrs_csr* A, const lrs_analyze_opts* opts, lrs_plan** out);
void export_plan(const lrs_plan& p, int what, std::vector<int32_t>& v);
int32_t export_local(int level, int32_t local);  // local node of level i -> export id
}  // namespace lrs
