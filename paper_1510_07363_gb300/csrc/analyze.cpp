// analyze.cpp -- host analysis: nested partitioning (Sec. 3), cluster
// adjacency (Def. adj) and the symbolic run of Algorithm 1 that fixes the
// elimination order, the well-separated sets of every Compress (Def. wellSep,
// or the distance-3 variant) and the neighbour sets of every Eliminate; and
// the batched form's union of instance subtrees.  No GPU work happens here.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>
#include <thread>
#include <utility>

#include "lrs_internal.h"

bool lrs_plan::cluster_adjacent(int level, int32_t a, int32_t b) const {
  if (a == b) return true;
  const auto& ptr = cadj_ptr[level];
  const auto& idx = cadj[level];
  return std::binary_search(idx.begin() + ptr[a], idx.begin() + ptr[a + 1], b);
}

// Well-separated clusters (Def. wellSep, Def. distance): cluster distance at
// least min_dist in the level's cluster graph -- 2: not adjacent; 3: not
// adjacent and no cluster adjacent to both (the sorted adjacency lists of a
// and b share no entry).
bool lrs_plan::well_separated(int level, int32_t a, int32_t b) const {
  if (cluster_adjacent(level, a, b)) return false;
  if (min_dist <= 2) return true;
  const auto& ptr = cadj_ptr[level];
  const auto& idx = cadj[level];
  auto i = idx.begin() + ptr[a], ie = idx.begin() + ptr[a + 1];
  auto j = idx.begin() + ptr[b], je = idx.begin() + ptr[b + 1];
  while (i != ie && j != je) {
    if (*i < *j) ++i;
    else if (*j < *i) ++j;
    else return false;
  }
  return true;
}

namespace lrs {
namespace {

// Recursive coordinate bisection: the cluster is split along the axis of
// largest coordinate extent (lowest axis on ties), ordered by (coordinate,
// original index); the first floor(|S|/2) entries form child 0.  That order is
// a strict total order, so a split needs only the set of the floor(|S|/2)
// smallest entries (a selection, linear time): the next level orders each
// child again.  Only the last split sorts both halves, whose order the leaves
// keep.  The result is the one full sorts at every level would give.
void build_partition(lrs_plan& p, const double* coords) {
  const int L = p.depth, dim = p.dim;
  std::vector<int32_t> order(p.n);
  std::iota(order.begin(), order.end(), 0);
  // bounds[c] .. bounds[c+1] delimit cluster c of the current level in `order`
  std::vector<int64_t> bounds = {0, p.n};
  for (int level = 0; level < L; ++level) {
    std::vector<int64_t> next;
    next.reserve(bounds.size() * 2);
    next.push_back(0);
    for (size_t c = 0; c + 1 < bounds.size(); ++c) {
      int32_t* first = order.data() + bounds[c];
      int32_t* last = order.data() + bounds[c + 1];
      int axis = 0;
      if (first != last) {
        double best = -1.0;
        for (int d = 0; d < dim; ++d) {
          double lo = coords[(int64_t)first[0] * dim + d], hi = lo;
          for (int32_t* it = first; it != last; ++it) {
            double x = coords[(int64_t)(*it) * dim + d];
            lo = std::min(lo, x);
            hi = std::max(hi, x);
          }
          if (hi - lo > best) { best = hi - lo; axis = d; }
        }
      }
      auto less = [&](int32_t a, int32_t b) {
        double xa = coords[(int64_t)a * dim + axis], xb = coords[(int64_t)b * dim + axis];
        return xa < xb || (xa == xb && a < b);
      };
      const int64_t half = (bounds[c + 1] - bounds[c]) / 2;
      std::nth_element(first, first + half, last, less);
      if (level + 1 == L) {
        std::sort(first, first + half, less);
        std::sort(first + half, last, less);
      }
      next.push_back(bounds[c] + half);
      next.push_back(bounds[c + 1]);
    }
    bounds.swap(next);
  }
  p.perm = order;
  p.leaf_off.assign(bounds.begin(), bounds.end());
}

// Cluster adjacency of every level as sorted CSR lists (Def. adj): leaf
// clusters touch when a stored entry couples them in either direction; a
// coarse pair touches when a pair of leaf descendants does.
void build_adjacency(lrs_plan& p) {
  const int L = p.depth;
  std::vector<std::pair<int32_t, int32_t>> pairs;
  for (int64_t row = 0; row < p.n; ++row)
    for (int64_t e = p.rowptr[row]; e < p.rowptr[row + 1]; ++e) {
      int32_t a = p.leaf_of[row], b = p.leaf_of[p.colind[e]];
      if (a != b) {
        pairs.emplace_back(a, b);
        pairs.emplace_back(b, a);
      }
    }
  p.cadj_ptr.assign(L + 1, {});
  p.cadj.assign(L + 1, {});
  for (int level = L; level >= 0; --level) {
    if (level < L)
      for (auto& pr : pairs) { pr.first >>= 1; pr.second >>= 1; }
    pairs.erase(std::remove_if(pairs.begin(), pairs.end(),
                               [](const std::pair<int32_t, int32_t>& x) { return x.first == x.second; }),
                pairs.end());
    std::sort(pairs.begin(), pairs.end());
    pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
    const int32_t nc = int32_t(1) << level;
    auto& ptr = p.cadj_ptr[level];
    auto& idx = p.cadj[level];
    ptr.assign(nc + 1, 0);
    for (auto& pr : pairs) ptr[pr.first + 1]++;
    for (int32_t c = 0; c < nc; ++c) ptr[c + 1] += ptr[c];
    idx.resize(pairs.size());
    for (size_t k = 0; k < pairs.size(); ++k) idx[k] = pairs[k].second;
  }
}

// Sorted-vector set helpers for the symbolic graph.
void add_sorted(std::vector<int32_t>& v, int32_t x) {
  auto it = std::lower_bound(v.begin(), v.end(), x);
  if (it == v.end() || *it != x) v.insert(it, x);
}
void del_sorted(std::vector<int32_t>& v, int32_t x) {
  auto it = std::lower_bound(v.begin(), v.end(), x);
  if (it != v.end() && *it == x) v.erase(it);
}

// Symbolic Algorithm 1.  The graph of level i has 3 * 2^(i-1) local nodes
// (super, black, red parent per cluster of P_{i-1}); red_adj carries the
// edges among the red-nodes of level i left by level i+1.
void symbolic(lrs_plan& p) {
  const int L = p.depth;
  // red-node edges at level l: leaf cluster adjacency
  std::vector<std::vector<int32_t>> red_adj(size_t(1) << L);
  for (int32_t c = 0; c < (int32_t(1) << L); ++c)
    red_adj[c].assign(p.cadj[L].begin() + p.cadj_ptr[L][c], p.cadj[L].begin() + p.cadj_ptr[L][c + 1]);
  p.levels.clear();
  for (int i = L; i >= 1; --i) {
    LevelPlan lp;
    lp.level = i;
    const int32_t ns = int32_t(1) << (i - 1);
    lp.nsuper = ns;
    std::vector<std::vector<int32_t>> g(3 * (size_t)ns);
    // MergeRedNodes: red c of level i belongs to super c / 2
    for (int32_t c = 0; c < 2 * ns; ++c)
      for (int32_t d : red_adj[c]) {
        int32_t a = c >> 1, b = d >> 1;
        if (a != b) add_sorted(g[local_node(a, kSlotS)], local_node(b, kSlotS));
      }
    for (int32_t a = 0; a < ns; ++a)
      for (int32_t v : g[local_node(a, kSlotS)]) {
        int32_t b = local_cluster(v);
        if (a < b) lp.merge_edges.emplace_back(a, b);
      }
    lp.ws.assign(ns, {});
    lp.nbs.assign(ns, {});
    lp.nbb.assign(ns, {});
    std::vector<char> done(ns, 0);
    int32_t left = ns;
    auto eliminate = [&](int32_t x, std::vector<int32_t>& rec) {
      rec = g[x];
      for (size_t u = 0; u < rec.size(); ++u) {
        del_sorted(g[rec[u]], x);
        for (size_t v = 0; v < rec.size(); ++v)
          if (u != v) add_sorted(g[rec[u]], rec[v]);
      }
      g[x].clear();
    };
    std::vector<char> in_batch(ns, 0);
    while (left > 0) {
      // j joins when no super-node already in the batch is its neighbour
      std::vector<int32_t> batch;
      for (int32_t j = 0; j < ns; ++j) {
        if (done[j]) continue;
        bool free = true;
        for (int32_t v : g[local_node(j, kSlotS)])
          if (local_slot(v) == kSlotS && in_batch[local_cluster(v)]) { free = false; break; }
        if (free) { batch.push_back(j); in_batch[j] = 1; }
      }
      for (int32_t j : batch) in_batch[j] = 0;
      for (int32_t j : batch) {
        const int32_t s = local_node(j, kSlotS), b = local_node(j, kSlotB), P = local_node(j, kSlotP);
        // Compress(s): neighbours whose cluster (in P_{i-1}) is not adjacent
        std::vector<int32_t>& ws = lp.ws[j];
        for (int32_t v : g[s])
          if (p.well_separated(i - 1, j, local_cluster(v))) ws.push_back(v);
        for (int32_t v : ws) {
          del_sorted(g[s], v);
          del_sorted(g[v], s);
          add_sorted(g[v], P);
          add_sorted(g[P], v);
        }
        add_sorted(g[s], b);
        add_sorted(g[b], s);
        add_sorted(g[b], P);
        add_sorted(g[P], b);
        eliminate(s, lp.nbs[j]);
        eliminate(b, lp.nbb[j]);
        done[j] = 1;
        --left;
      }
      lp.batches.push_back(batch);
    }
    // red-nodes of level i-1 and their edges survive into the next level
    std::vector<std::vector<int32_t>> next(ns);
    for (int32_t j = 0; j < ns; ++j)
      for (int32_t v : g[local_node(j, kSlotP)]) next[j].push_back(local_cluster(v));
    red_adj.swap(next);
    p.levels.push_back(std::move(lp));
  }
}

// Leaf assembly map: every stored entry goes to one block of a leaf
// super-node pair.  Blocks of level l are numbered: self block of super a at
// index a, then for merge edge e = (a, b): (a, b) at ns + 2e, (b, a) at
// ns + 2e + 1.
void leaf_assembly(lrs_plan& p) {
  const LevelPlan& lp = p.levels[0];
  const int32_t ns = lp.nsuper;
  std::vector<std::vector<std::pair<int32_t, int32_t>>> edge_of(ns);  // (other super, block index)
  for (size_t e = 0; e < lp.merge_edges.size(); ++e) {
    auto [a, b] = lp.merge_edges[e];
    edge_of[a].emplace_back(b, ns + 2 * (int32_t)e);
    edge_of[b].emplace_back(a, ns + 2 * (int32_t)e + 1);
  }
  for (auto& v : edge_of) std::sort(v.begin(), v.end());
  auto super_off = [&](int32_t leaf) { return p.leaf_off[leaf] - p.leaf_off[leaf & ~1]; };
  auto super_size = [&](int32_t sj) { return p.leaf_off[2 * sj + 2] - p.leaf_off[2 * sj]; };
  p.nz_block.assign(p.nnz, 0);
  p.nz_elem.assign(p.nnz, 0);
  for (int64_t row = 0; row < p.n; ++row)
    for (int64_t e = p.rowptr[row]; e < p.rowptr[row + 1]; ++e) {
      int32_t col = p.colind[e];
      int32_t lr = p.leaf_of[row], lc = p.leaf_of[col];
      int32_t sa = lr >> 1, sb = lc >> 1;
      int32_t blk = sa;
      if (sa != sb) {
        auto& v = edge_of[sa];
        auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(sb, INT32_MIN));
        blk = it->second;
      }
      int32_t r = p.pos[row] - p.leaf_off[lr] + super_off(lr);
      int32_t c = p.pos[col] - p.leaf_off[lc] + super_off(lc);
      p.nz_elem[e] = c * super_size(sa) + r;
      p.nz_block[e] = blk;
    }
}

}  // namespace

int32_t export_local(int level, int32_t v) {
  const int32_t j = local_cluster(v);
  const int32_t h = heap_of(level - 1, j);
  switch (local_slot(v)) {
    case kSlotS: return export_id(h, kSuper);
    case kSlotB: return export_id(h, kBlack);
    default: return export_id(h, kRed);
  }
}

namespace {

// Checks one input matrix; returns its tree depth (> 0) or an LRS_ERR_* code
// negated.
int check_input(const lrs_csr* A, const lrs_analyze_opts* opts) {
  if (!A || A->n < 1 || !A->rowptr || !A->colind || !A->coords) return -LRS_ERR_INVALID_ARG;
  if (opts->separation != 0 && opts->separation != 2 && opts->separation != 3) return -LRS_ERR_INVALID_ARG;
  if (A->dim < 1 || A->dim > 8 || A->n > INT32_MAX) return -LRS_ERR_INVALID_ARG;
  int depth = opts->depth;
  if (depth <= 0) {
    if (opts->leaf_size < 1) return -LRS_ERR_INVALID_ARG;
    depth = 0;
    while (((int64_t)opts->leaf_size << depth) < A->n) ++depth;
    depth = std::max(depth, 1);
  }
  if (depth > 24) return -LRS_ERR_INVALID_ARG;
  if (A->rowptr[0] != 0) return -LRS_ERR_INVALID_ARG;
  for (int64_t i = 0; i < A->n * A->dim; ++i)
    if (!std::isfinite(A->coords[i])) return -LRS_ERR_INVALID_ARG;
  for (int64_t r = 0; r < A->n; ++r)
    if (A->rowptr[r + 1] < A->rowptr[r]) return -LRS_ERR_INVALID_ARG;
  std::vector<int32_t> seen(A->n, -1);
  for (int64_t r = 0; r < A->n; ++r)
    for (int64_t e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e) {
      const int32_t c = A->colind[e];
      if (c < 0 || c >= A->n || seen[c] == (int32_t)r) return -LRS_ERR_INVALID_ARG;
      seen[c] = (int32_t)r;
    }
  return depth;
}

// Position of the transposed entry of every stored entry when the pattern is
// symmetric (for the test of numerical symmetry at factor time); empty
// otherwise.  The entries are bucketed by column with ascending rows, and
// entry (c, r) is looked up among the entries of column r.
void build_tpos(lrs_plan& p) {
  std::vector<int64_t> cptr(p.n + 1, 0);
  for (int64_t e = 0; e < p.nnz; ++e) cptr[p.colind[e] + 1]++;
  for (int64_t c = 0; c < p.n; ++c) cptr[c + 1] += cptr[c];
  std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1), cent(p.nnz);
  std::vector<int32_t> crow(p.nnz);
  for (int64_t r = 0; r < p.n; ++r)
    for (int64_t e = p.rowptr[r]; e < p.rowptr[r + 1]; ++e) {
      const int64_t k = fill[p.colind[e]]++;
      crow[k] = (int32_t)r;
      cent[k] = e;
    }
  p.tpos.assign(p.nnz, -1);
  for (int64_t r = 0; r < p.n; ++r)
    for (int64_t e = p.rowptr[r]; e < p.rowptr[r + 1]; ++e) {
      const int32_t c = p.colind[e];
      const auto first = crow.begin() + cptr[r], last = crow.begin() + cptr[r + 1];
      const auto it = std::lower_bound(first, last, c);
      if (it == last || *it != c) { p.tpos.clear(); return; }
      p.tpos[e] = cent[it - crow.begin()];
    }
}

void set_positions(lrs_plan& p) {
  p.pos.assign(p.n, 0);
  p.leaf_of.assign(p.n, 0);
  for (int64_t k = 0; k < p.n; ++k) p.pos[p.perm[k]] = (int32_t)k;
  for (size_t c = 0; c + 1 < p.leaf_off.size(); ++c)
    for (int64_t k = p.leaf_off[c]; k < p.leaf_off[c + 1]; ++k) p.leaf_of[p.perm[k]] = (int32_t)c;
}

void finish(lrs_plan& p) {
  build_tpos(p);
  build_adjacency(p);
  symbolic(p);
  leaf_assembly(p);
}

}  // namespace

int analyze(const lrs_csr* A, const lrs_analyze_opts* opts, lrs_plan** out) {
  if (!A || !opts || !out) return LRS_ERR_INVALID_ARG;
  const int depth = check_input(A, opts);
  if (depth < 0) return -depth;
  lrs_plan* p = new (std::nothrow) lrs_plan();
  if (!p) return LRS_ERR_OOM;
  p->n = A->n;
  p->nnz = A->rowptr[A->n];
  p->dim = A->dim;
  p->depth = depth;
  p->min_dist = opts->separation == 3 ? 3 : 2;
  p->rowptr.assign(A->rowptr, A->rowptr + A->n + 1);
  p->colind.assign(A->colind, A->colind + p->nnz);
  p->inst_row_off = {0, p->n};
  p->inst_leaf_base = {0};
  p->inst_depth = {depth};
  build_partition(*p, A->coords);
  set_positions(*p);
  finish(*p);
  *out = p;
  return LRS_OK;
}

// The batched form: instance k keeps the partitioning lrs_analyze would give
// it alone (depth d_k), and its 2^(d_k) leaves take an aligned range of the
// union's 2^l leaves -- instances placed by descending depth (ascending index
// on ties), so every range starts at a multiple of its length, as in a buddy
// allocator.  Each instance is then one cluster of P_(l - d_k); clusters that
// hold no instance are empty.  Since no entry couples two instances, no
// cluster ever holds live unknowns of two instances: every Compress and
// Eliminate of the union is one of an instance's own, and the instances'
// eliminations at one level share its batches and launches.
int analyze_batch(int count, const lrs_csr* A, const lrs_analyze_opts* opts, lrs_plan** out) {
  if (count < 1 || !A || !opts || !out) return LRS_ERR_INVALID_ARG;
  std::vector<int> depth(count);
  int64_t n = 0, nnz = 0, leaves = 0;
  for (int k = 0; k < count; ++k) {
    depth[k] = check_input(&A[k], opts);
    if (depth[k] < 0) return -depth[k];
    n += A[k].n;
    nnz += A[k].rowptr[A[k].n];
    leaves += int64_t(1) << depth[k];
  }
  int L = 1;
  while ((int64_t(1) << L) < leaves) ++L;
  if (n > INT32_MAX || L > 24) return LRS_ERR_INVALID_ARG;
  lrs_plan* p = new (std::nothrow) lrs_plan();
  if (!p) return LRS_ERR_OOM;
  p->n = n;
  p->nnz = nnz;
  p->dim = A[0].dim;
  p->depth = L;
  p->min_dist = opts->separation == 3 ? 3 : 2;
  p->rowptr.assign(1, 0);
  p->colind.reserve(nnz);
  p->inst_row_off.assign(1, 0);
  for (int k = 0; k < count; ++k) {
    const int64_t r0 = p->inst_row_off.back(), e0 = p->rowptr.back();
    for (int64_t r = 0; r < A[k].n; ++r) p->rowptr.push_back(e0 + A[k].rowptr[r + 1]);
    for (int64_t e = 0; e < A[k].rowptr[A[k].n]; ++e) p->colind.push_back((int32_t)(r0 + A[k].colind[e]));
    p->inst_row_off.push_back(r0 + A[k].n);
  }
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return depth[a] > depth[b]; });
  p->inst_leaf_base.assign(count, 0);
  p->inst_depth = depth;
  p->perm.assign(n, 0);
  p->leaf_off.assign((size_t(1) << L) + 1, (int32_t)n);
  // the instances' partitions are independent: up to 16 host threads take
  // them in turn (the calling thread always works; a worker that cannot be
  // started or that fails leaves its instances to the others or to the error)
  std::vector<lrs_plan> parts(count);
  {
    std::atomic<int> next{0};
    std::atomic<bool> failed{false};
    auto work = [&] {
      try {
        for (int k; (k = next.fetch_add(1)) < count;) {
          parts[k].n = A[k].n;
          parts[k].dim = A[k].dim;
          parts[k].depth = depth[k];
          build_partition(parts[k], A[k].coords);
        }
      } catch (...) {
        failed = true;
        next = count;
      }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = (int)std::min<unsigned>({(unsigned)count, 16u, hw});
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) {
      try {
        pool.emplace_back(work);
      } catch (...) {
        break;
      }
    }
    work();
    for (std::thread& t : pool) t.join();
    if (failed) {
      delete p;
      return LRS_ERR_OOM;
    }
  }
  int64_t leaf0 = 0, pos0 = 0;
  for (int k : order) {
    lrs_plan& one = parts[k];
    const int32_t r0 = (int32_t)p->inst_row_off[k];
    for (int64_t t = 0; t < one.n; ++t) p->perm[pos0 + t] = r0 + one.perm[t];
    for (int64_t c = 0; c < (int64_t(1) << depth[k]); ++c) p->leaf_off[leaf0 + c] = (int32_t)(pos0 + one.leaf_off[c]);
    std::vector<int32_t>().swap(one.perm);
    p->inst_leaf_base[k] = leaf0;
    leaf0 += int64_t(1) << depth[k];
    pos0 += one.n;
  }
  set_positions(*p);
  finish(*p);
  *out = p;
  return LRS_OK;
}

void export_plan(const lrs_plan& p, int what, std::vector<int32_t>& v) {
  v.clear();
  if (what == 0) v = p.perm;
  if (what == 1) v = p.leaf_off;
  if (what == 2)
    for (const LevelPlan& lp : p.levels) {
      v.push_back(lp.level);
      v.push_back((int32_t)lp.batches.size());
      for (const auto& b : lp.batches) {
        v.push_back((int32_t)b.size());
        for (int32_t j : b) v.push_back(export_local(lp.level, local_node(j, kSlotS)));
      }
    }
  auto push_sorted = [&](int level, int32_t node, const std::vector<int32_t>& nb) {
    std::vector<int32_t> ids;
    for (int32_t x : nb) ids.push_back(export_local(level, x));
    std::sort(ids.begin(), ids.end());
    v.push_back(export_local(level, node));
    v.push_back((int32_t)ids.size());
    v.insert(v.end(), ids.begin(), ids.end());
  };
  if (what == 3)
    for (const LevelPlan& lp : p.levels)
      for (const auto& b : lp.batches)
        for (int32_t j : b) push_sorted(lp.level, local_node(j, kSlotS), lp.ws[j]);
  if (what == 5)
    for (size_t k = 0; k + 1 < p.inst_row_off.size(); ++k) {
      v.push_back((int32_t)p.inst_row_off[k]);
      v.push_back((int32_t)(p.inst_row_off[k + 1] - p.inst_row_off[k]));
      v.push_back((int32_t)p.inst_leaf_base[k]);
      v.push_back(p.inst_depth[k]);
    }
  if (what == 4)
    for (const LevelPlan& lp : p.levels)
      for (const auto& b : lp.batches)
        for (int32_t j : b) {
          push_sorted(lp.level, local_node(j, kSlotS), lp.nbs[j]);
          push_sorted(lp.level, local_node(j, kSlotB), lp.nbb[j]);
        }
}

}  // namespace lrs
