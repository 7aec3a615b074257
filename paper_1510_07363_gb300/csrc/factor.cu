// factor.cu -- Algorithm 1 on the GPU.
//
// The host walks the symbolic program of lrs_analyze level by level and batch
// by batch and launches one grid per step over all super-nodes of a batch
// (batch members share no edge, so their Compress and Eliminate steps are
// independent; updates to a block shared by several members are summed by
// one CTA per output tile in batch order, without atomics).  Per batch:
//   C  Gram matrices of the stacked well-separated blocks and their spectra
//      (tridiagonal reduction, multisection, inverse iteration); the ranks
//      come back to the host (one sync per batch: block sizes of the new
//      black / red-nodes depend on them)
//   A  R_k = A_k V, Q_k^T = V^T B_k^T, V, V^T, -I blocks (Sec. 4.3 edge rules)
//   S  Eliminate(s): pivot inverse, A_ss^{-1} A_{s,k}, Schur updates
//   B  Eliminate(b): the same for the black-nodes
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <memory>

#include "runtime.h"

namespace lrs {
namespace {

inline uint64_t key(int32_t r, int32_t c) { return (uint64_t(uint32_t(r)) << 32) | uint32_t(c); }
inline int ntiles(int x) { return (x + kTile - 1) / kTile; }

struct Blk {
  double* p;
  int rows, cols;
};

// The live blocks of a level keyed by (row node, column node): an
// open-addressing hash table with linear probing and backward-shift deletion
// (flat arrays; the factorization of a batched plan performs tens of millions
// of lookups, inserts and erasures, for which node-based maps were the bulk of
// the host time).  Given the number of row names (reset), the slots of a row
// form a window of cap / rows slots with the column hashed inside it: the
// loops that walk blocks in row order then sweep the table instead of missing
// the cache on every access.  Linear probing keeps it correct whatever the
// rows hold; the windows double with the table.
class BlockMap {
 public:
  Blk* find(uint64_t k) {
    if (keys_.empty()) return nullptr;
    for (size_t i = slot(k);; i = (i + 1) & mask_) {
      if (keys_[i] == k) return &vals_[i];
      if (keys_[i] == kEmpty) return nullptr;
    }
  }
  const Blk* find(uint64_t k) const { return const_cast<BlockMap*>(this)->find(k); }
  bool count(uint64_t k) const { return find(k) != nullptr; }
  Blk& operator[](uint64_t k) {
    bool inserted;
    return find_or_insert(k, inserted);
  }
  // the entry of k; a new one ({nullptr, 0, 0}, inserted = true) if k had none
  Blk& find_or_insert(uint64_t k, bool& inserted) {
    if (2 * (n_ + 1) > keys_.size()) rehash(std::max<size_t>(16, 2 * keys_.size()));
    size_t i = slot(k);
    while (keys_[i] != kEmpty && keys_[i] != k) i = (i + 1) & mask_;
    inserted = keys_[i] == kEmpty;
    if (inserted) {
      keys_[i] = k;
      vals_[i] = Blk{nullptr, 0, 0};
      ++n_;
    }
    return vals_[i];
  }
  void erase(uint64_t k) {
    if (keys_.empty()) return;
    size_t i = slot(k);
    while (keys_[i] != k) {
      if (keys_[i] == kEmpty) return;
      i = (i + 1) & mask_;
    }
    // move later entries of the probe run back over the hole while their home
    // slot does not lie cyclically in (hole, position]
    for (size_t j = (i + 1) & mask_; keys_[j] != kEmpty; j = (j + 1) & mask_) {
      const size_t h = slot(keys_[j]);
      const bool stays = (i <= j) ? (i < h && h <= j) : (i < h || h <= j);
      if (stays) continue;
      keys_[i] = keys_[j];
      vals_[i] = vals_[j];
      i = j;
    }
    keys_[i] = kEmpty;
    --n_;
  }
  // empty, with room for n entries whose row names are below `rows` (no
  // rehashing until then)
  void reset(size_t n, size_t rows) {
    size_t cap = 16;
    while (cap < 2 * n) cap <<= 1;
    row_bits_ = 0;
    while ((size_t(1) << row_bits_) < rows) ++row_bits_;
    keys_.assign(cap, kEmpty);
    vals_.resize(cap);                           // set when a key is inserted
    n_ = 0;
    size_for(cap);
  }
  size_t size() const { return n_; }
  std::vector<uint64_t> key_list() const {
    std::vector<uint64_t> out;
    out.reserve(n_);
    for (uint64_t k : keys_)
      if (k != kEmpty) out.push_back(k);
    return out;
  }
  void swap(BlockMap& o) {
    keys_.swap(o.keys_);
    vals_.swap(o.vals_);
    std::swap(mask_, o.mask_);
    std::swap(n_, o.n_);
    std::swap(row_bits_, o.row_bits_);
    std::swap(win_bits_, o.win_bits_);
  }

 private:
  static constexpr uint64_t kEmpty = ~0ull;      // never a key: node names are non-negative
  std::vector<uint64_t> keys_;
  std::vector<Blk> vals_;
  size_t mask_ = 0, n_ = 0;
  int row_bits_ = 0;                             // rows below 2^row_bits_ (0: not given)
  int win_bits_ = 0;                             // slots per row window: 2^win_bits_ (0: no windows)
  size_t slot(uint64_t k) const {
    if (win_bits_) {                             // the row's window, the column hashed (Fibonacci) inside
      const uint64_t c = (k & 0xffffffffull) * 0x9E3779B97F4A7C15ull;
      return (size_t)(((k >> 32) << win_bits_) + (c >> (64 - win_bits_))) & mask_;
    }
    k ^= k >> 33;                                // 64-bit finaliser of MurmurHash3
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (size_t)k & mask_;
  }
  void size_for(size_t cap) {
    mask_ = cap - 1;
    int cap_bits = 0;
    while ((size_t(1) << cap_bits) < cap) ++cap_bits;
    // windows of at least 16 slots, else the plain hash
    win_bits_ = (row_bits_ > 0 && cap_bits - row_bits_ >= 4) ? cap_bits - row_bits_ : 0;
  }
  void rehash(size_t cap) {
    std::vector<uint64_t> ok;
    std::vector<Blk> ov;
    ok.swap(keys_);
    ov.swap(vals_);
    keys_.assign(cap, kEmpty);
    vals_.assign(cap, Blk{nullptr, 0, 0});
    n_ = 0;
    size_for(cap);
    for (size_t i = 0; i < ok.size(); ++i)
      if (ok[i] != kEmpty) (*this)[ok[i]] = ov[i];
  }
};

// Stable LSD radix sort of entries by their 64-bit key (11-bit digits, only
// as many passes as the largest key needs).
template <class E>
void radix_sort_pairs(std::vector<E>& v, uint64_t kmax) {
  constexpr int kBits = 11, kBuckets = 1 << kBits;
  std::vector<E> tmp(v.size());
  for (int shift = 0; shift < 64 && (kmax >> shift) != 0; shift += kBits) {
    size_t count[kBuckets + 1] = {};
    for (const E& e : v) ++count[((e.key >> shift) & (kBuckets - 1)) + 1];
    for (int b = 0; b < kBuckets; ++b) count[b + 1] += count[b];
    for (const E& e : v) tmp[count[(e.key >> shift) & (kBuckets - 1)]++] = e;
    v.swap(tmp);
  }
}

// The Schur targets of one elimination phase, from the neighbour lists alone
// (no sizes): one (target, pivot a, neighbours u, v) entry per pair, stably
// radix-sorted by target key so each target's entries keep the pivots' order
// (the summation order of its products).  Built before the batch's sync, while
// the device computes the spectra.
struct SchurGroups {
  struct Pair {
    uint64_t key;
    int32_t a, u, v;
  };
  std::vector<Pair> pairs;
  std::vector<std::pair<int32_t, int32_t>> order;   // targets (q, k), ascending key
  std::vector<int> first;                          // entry ranges [first[o], first[o + 1])
  void build(const std::vector<const std::vector<int32_t>*>& nbrs) {
    pairs.clear();
    order.clear();
    first.clear();
    size_t npairs = 0;
    for (const auto* nb : nbrs) npairs += nb->size() * nb->size();
    pairs.reserve(npairs);
    uint64_t kmax = 0;
    for (size_t a = 0; a < nbrs.size(); ++a) {
      const auto& nb = *nbrs[a];
      for (size_t u = 0; u < nb.size(); ++u)
        for (size_t v = 0; v < nb.size(); ++v) {
          const uint64_t kk = ((uint64_t)(uint32_t)nb[u] << 32) | (uint32_t)nb[v];
          kmax = std::max(kmax, kk);
          pairs.push_back(Pair{kk, (int32_t)a, (int32_t)u, (int32_t)v});
        }
    }
    radix_sort_pairs(pairs, kmax);
    for (size_t e = 0; e < pairs.size(); ++e)
      if (e == 0 || pairs[e].key != pairs[e - 1].key) {
        first.push_back((int)e);
        order.emplace_back((int32_t)(pairs[e].key >> 32), (int32_t)(pairs[e].key & 0xffffffffu));
      }
    first.push_back((int)pairs.size());
  }
};

struct Factorizer {
  lrs_factor_t* F;
  const lrs_plan& P;
  cudaStream_t st;
  int level = 0;                                    // current level i
  std::vector<int> sz;                              // sizes of local nodes of level i
  BlockMap blocks;                                  // live blocks, keyed by local names
  // product tiles and their terms per engine: FP64 FMAs (64 x 64 tiles), FP64
  // emulated on the tensor cores (128 x 64), TF32 split (precision form, 128 x 128)
  enum Engine { kSimt = 0, kEmu = 1, kTf32 = 2, kEngines = 3 };
  std::vector<GemmTask> gt[kEngines];
  std::vector<GemmTerm> gm[kEngines];
  std::vector<CopyTask> ct;
  double flops = 0.0, flops32 = 0.0;
  double pend_flops[kEngines] = {}, pend_bytes[kEngines] = {};   // of the launches being built
  double copy_bytes = 0.0;

  Factorizer(lrs_factor_t* f) : F(f), P(*f->plan), st(f->stream) {}
  bool sym = false;                   // the symmetric path (A = A^T): half the products, transposes for the rest
  bool lowp = false;                  // the precision form: block products on the tensor cores
  bool lowp_gram = false;             // ... and the Gram matrices too (eps >= LRS_PREC_FP32_GRAM_EPS)

  bool is_red(int32_t v) const { return local_slot(v) == kSlotP; }
  Arena& arena_for(int32_t r, int32_t c) {
    return (is_red(r) && is_red(c)) ? F->trans[level & 1] : F->persist;
  }
  Blk& get(int32_t r, int32_t c) {
    Blk* b = blocks.find(key(r, c));
    if (!b) fail(LRS_ERR_STATE, "missing block");
    return *b;
  }
  Blk make(int32_t r, int32_t c) {
    Blk b{arena_for(r, c).take((size_t)sz[r] * sz[c]), sz[r], sz[c]};
    blocks[key(r, c)] = b;
    return b;
  }

  // Add the tiles of C (rows x cols) = init + sign * sum(terms) to the task
  // list of an engine (lower_only: a symmetric C, only tiles holding entries
  // on or below the diagonal).  f32: the precision form's TF32 products;
  // otherwise FP64, emulated on the tensor cores unless the factor asks for
  // FP64 FMAs or the contraction is too long for the emulation's integer sums.
  void add_gemm(double* C, int ldc, const double* D, int ldd, int rows, int cols, int mode,
                const std::vector<GemmTerm>& terms, bool lower_only = false, bool f32 = false) {
    add_gemm(C, ldc, D, ldd, rows, cols, mode, terms.data(), terms.size(), lower_only, f32);
  }
  // one term (no temporary vector: the host plans millions of these on a batched plan)
  void add_gemm(double* C, int ldc, const double* D, int ldd, int rows, int cols, int mode,
                const GemmTerm& term, bool lower_only = false, bool f32 = false) {
    add_gemm(C, ldc, D, ldd, rows, cols, mode, &term, 1, lower_only, f32);
  }
  void add_gemm(double* C, int ldc, const double* D, int ldd, int rows, int cols, int mode,
                const GemmTerm* terms_p, size_t nterms, bool lower_only = false, bool f32 = false) {
    if (rows <= 0 || cols <= 0) return;
    int eng = f32 ? kTf32 : kSimt;
    if (!f32 && F->gemm_emu) {
      // the emulation pays for its split and its fixed cost per tile from about
      // 64^3 multiply-adds on; smaller products stay on FP64 FMAs
      const int chunks = gemm_emu_chunks(terms_p, (int)nterms);
      double ksum = 0.0;
      for (size_t i = 0; i < nterms; ++i) ksum += terms_p[i].k;
      if (chunks <= kEmuMaxChunks && (double)rows * cols * ksum >= kEmuMinWork) eng = kEmu;
    }
    std::vector<GemmTask>& tl = gt[eng];
    std::vector<GemmTerm>& ml = gm[eng];
    const int t0 = (int)ml.size();
    ml.insert(ml.end(), terms_p, terms_p + nterms);
    const GemmTerm* terms_end = terms_p + nterms;
    double frac_rows = 0.0;                          // share of C's entries actually computed
    const int tm = eng == kEmu ? kEmuTileM : eng == kTf32 ? kTcTile : kTile;
    const int tn = eng == kEmu ? kEmuTileN : eng == kTf32 ? kTcTile : kTile;
    const int nr = (rows + tm - 1) / tm, nc = (cols + tn - 1) / tn;
    for (int tj = 0; tj < nc; ++tj)
      for (int ti = lower_only ? (tj * tn) / tm : 0; ti < nr; ++ti) {   // rows of tile ti reach column tj tn
        tl.push_back(GemmTask{C, D, ldc, ldd, rows, cols, ti, tj, t0, (int)nterms, mode});
        frac_rows += (double)std::min(tm, rows - ti * tm) * std::min(tn, cols - tj * tn);
      }
    const double frac = frac_rows / ((double)rows * cols);
    for (const GemmTerm* tp = terms_p; tp != terms_end; ++tp) {
      const GemmTerm& t = *tp;
      flops += frac * 2.0 * rows * cols * t.k;
      if (f32) flops32 += frac * 2.0 * rows * cols * t.k;
      pend_flops[eng] += frac * 2.0 * rows * cols * t.k;
      pend_bytes[eng] += 8.0 * ((double)rows * t.k + (double)t.k * cols);
    }
    pend_bytes[eng] += frac * 8.0 * rows * cols * ((D || (mode & kAccumulate)) ? 2 : 1);
  }
  // the emulated products of one launch: every distinct operand split once
  // into the launch's workspace (reused by the next launch of the stream),
  // then the product kernel
  void launch_emu(int n, const GemmTask* d_tasks) {
    EmuPlan plan = plan_gemm_emu(gt[kEmu].data(), n, gm[kEmu].data(), (int)gm[kEmu].size());
    F->emu_ws.reset();
    uint8_t* work = reinterpret_cast<uint8_t*>(F->emu_ws.take((plan.bytes + 7) / 8));
    plan.bind(work);
    if (plan.bad_bytes) cuda_check(cudaMemsetAsync(work + plan.bad_off, 0, plan.bad_bytes, st), "emulation flags");
    const EmuSplitTask* d_split = F->stager.put(plan.split);
    const EmuTerm* d_eterms = F->stager.put(plan.eterms);
    cuda_check(launch_gemm_emu(plan, d_split, d_tasks, n, d_eterms, F->status, st), "emulated FP64 gemm");
  }
  void flush_gemm() {
    for (int eng = 0; eng < kEngines; ++eng) {
      if (gt[eng].empty()) continue;
      const GemmTerm* d_terms = F->stager.put(gm[eng]);
      const GemmTask* d_tasks = F->stager.put(gt[eng]);
      const int n = (int)gt[eng].size();
      cudaEvent_t e = F->prof.start();
      if (eng == kSimt) launch_gemm(d_tasks, n, d_terms, st);
      else if (eng == kEmu) launch_emu(n, d_tasks);
      else cuda_check(launch_gemm_tc(d_tasks, n, d_terms, F->status, st), "tensor-core gemm");
      const int cls = eng == kSimt ? LRS_PROF_FACTOR_GEMM : eng == kEmu ? LRS_PROF_FACTOR_GEMM_EMU
                                                                        : LRS_PROF_FACTOR_GEMM_F32;
      F->prof.stop(cls, e, pend_flops[eng], pend_bytes[eng], 0, 0, n);
      gt[eng].clear();
      gm[eng].clear();
      pend_flops[eng] = pend_bytes[eng] = 0.0;
    }
  }
  void flush_copy() {
    if (!ct.empty()) {
      for (const CopyTask& c : ct) copy_bytes += 8.0 * c.rows * c.cols * (c.mode == 2 ? 1 : 2);
      // one CTA per 64-column piece of a block (the in-place mirror stays whole:
      // its tiles are defined relative to the block's diagonal)
      std::vector<CopyTask> pieces;
      for (const CopyTask& c : ct) {
        if (c.mode == 3 || c.cols <= 64) { pieces.push_back(c); continue; }
        for (int j0 = 0; j0 < c.cols; j0 += 64) {
          CopyTask q = c;
          q.cols = std::min(64, c.cols - j0);
          q.dst = c.dst + (size_t)j0 * c.ldd;
          if (c.mode == 0) {
            q.src = c.src + (size_t)j0 * c.lds;                          // columns j0.. of src
          } else if (c.mode == 1) {
            q.src = c.src + j0;                                          // rows j0.. of src
          } else {                                                       // alpha * I: its diagonal
            q.mode = 4;                                                  // entries (j0 + j, j0 + j)
            q.lds = j0;
          }
          pieces.push_back(q);
        }
      }
      ct.swap(pieces);
      const CopyTask* d = F->stager.put(ct);
      cudaEvent_t e = F->prof.start();
      launch_copy(d, (int)ct.size(), st);
      F->prof.stop(LRS_PROF_COPY, e, 0.0, copy_bytes);
    }
    ct.clear();
    copy_bytes = 0.0;
  }

  void assemble_leaf(const double* d_val);
  void merge(const BlockMap& old, const std::vector<int>& redsz);
  // eq. curOff6: add the squared Frobenius norms of every block of the level
  // as it starts (after the merge) to the running ||all levels below||_F^2;
  // blocks in key order, pieces of at most 64 columns, summed in a fixed order
  void add_level_norm() {
    flush_copy();
    std::vector<uint64_t> keys = blocks.key_list();
    std::sort(keys.begin(), keys.end());
    std::vector<SumSqTask> tasks;
    for (uint64_t k : keys) {
      const Blk& b = *blocks.find(k);
      if (!b.p || b.rows <= 0 || b.cols <= 0) continue;
      for (int j0 = 0; j0 < b.cols; j0 += 64)
        tasks.push_back(SumSqTask{b.p + (size_t)j0 * b.rows, b.rows, std::min(64, b.cols - j0), b.rows});
    }
    if (tasks.empty()) return;
    const SumSqTask* d_tasks = F->stager.put(tasks);
    double* partial = F->workspace.take(tasks.size());
    launch_sumsq(d_tasks, (int)tasks.size(), partial, &F->status->below_sq, st);
    cuda_check(cudaGetLastError(), "level norm");
  }
  void batch(const LevelPlan& lp, const std::vector<int32_t>& js);
  void eliminate(const std::vector<int32_t>& nodes, const std::vector<const std::vector<int32_t>*>& nbrs,
                 bool pre_inverted, const SchurGroups& groups);
  // defer: the large (resident) inverses are not launched but kept in
  // deferred_inv / deferred_mirror, to run beside the batch's reductions
  void launch_inverses(const std::vector<int32_t>& nodes, cudaStream_t s, bool side, bool defer = false);
  std::vector<InvTask> deferred_inv;
  std::vector<CopyTask> deferred_mirror;
  void launch_deferred_inverses();
  void run(const double* d_val);
};

// Initialize(l) + MergeRedNodes at the leaf level: the stored entries of A
// are scattered straight into the blocks of the leaf super-nodes.
void Factorizer::assemble_leaf(const double* d_val) {
  const LevelPlan& lp = P.levels[0];
  const int32_t ns = lp.nsuper;
  std::vector<int32_t> ra, ca;
  for (int32_t a = 0; a < ns; ++a) { ra.push_back(a); ca.push_back(a); }
  for (auto [a, b] : lp.merge_edges) {
    ra.push_back(a); ca.push_back(b);
    ra.push_back(b); ca.push_back(a);
  }
  std::vector<int64_t> base(ra.size());
  int64_t total = 0;
  for (size_t k = 0; k < ra.size(); ++k) {
    base[k] = total;
    total += ((int64_t)sz[local_node(ra[k], kSlotS)] * sz[local_node(ca[k], kSlotS)] + 31) & ~int64_t(31);
  }
  double* region = F->persist.take((size_t)std::max<int64_t>(total, 1));
  cuda_check(cudaMemsetAsync(region, 0, (size_t)total * sizeof(double), st), "zero leaf blocks");
  for (size_t k = 0; k < ra.size(); ++k) {
    const int32_t r = local_node(ra[k], kSlotS), c = local_node(ca[k], kSlotS);
    blocks[key(r, c)] = Blk{region + base[k], sz[r], sz[c]};
  }
  std::vector<int64_t> dst(P.nnz);
  for (int64_t e = 0; e < P.nnz; ++e) dst[e] = base[P.nz_block[e]] + P.nz_elem[e];
  int64_t* d_dst = reinterpret_cast<int64_t*>(F->scratch.take((size_t)P.nnz));
  cuda_check(cudaMemcpyAsync(d_dst, dst.data(), dst.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st),
             "leaf map");
  cudaEvent_t e = F->prof.start();
  launch_scatter(d_val, d_dst, P.nnz, region, st);
  launch_amax(d_val, P.nnz, F->status, st);
  F->prof.stop(LRS_PROF_ASSEMBLE, e, 0.0, 8.0 * P.nnz * 4);
  cuda_check(cudaStreamSynchronize(st), "leaf assembly");   // dst is pageable host memory
}

// MergeRedNodes (Sec. 4.2): super-node blocks are the 2 x 2 concatenations of
// the blocks between their red-nodes; a missing red block is zero.
void Factorizer::merge(const BlockMap& old, const std::vector<int>& redsz) {
  const LevelPlan& lp = P.levels[P.depth - level];
  std::vector<std::pair<int32_t, int32_t>> pairs;
  for (int32_t a = 0; a < lp.nsuper; ++a) pairs.emplace_back(a, a);
  for (auto [a, b] : lp.merge_edges) {
    pairs.emplace_back(a, b);
    pairs.emplace_back(b, a);
  }
  for (auto [a, b] : pairs) {
    Blk d = make(local_node(a, kSlotS), local_node(b, kSlotS));
    if (d.rows == 0 || d.cols == 0) continue;
    for (int x = 0; x < 2; ++x)
      for (int y = 0; y < 2; ++y) {
        const int32_t c = 2 * a + x, e = 2 * b + y;
        const int rows = redsz[c], cols = redsz[e];
        if (rows == 0 || cols == 0) continue;
        double* dst = d.p + (x ? redsz[2 * a] : 0) + (size_t)(y ? redsz[2 * b] : 0) * d.rows;
        const Blk* ob = old.find(key(local_node(c, kSlotP), local_node(e, kSlotP)));
        if (ob) ct.push_back(CopyTask{ob->p, dst, rows, d.rows, rows, cols, 0, 0.0});
        else ct.push_back(CopyTask{nullptr, dst, 0, d.rows, rows, cols, 2, 0.0});
      }
  }
  flush_copy();
}

// Pivot inverses of a set of nodes: small blocks one CTA each (on stream s);
// large ones resident in shared memory on teams of CTAs, in waves on the main
// stream (a kernel whose CTAs wait on one another never runs beside another
// such kernel), or, when a block is too large for that, on a cluster each or
// the whole GPU.  On the side stream the task arrays live in the scratch arena
// (the staging ring may be reused before that stream reads them).
void Factorizer::launch_inverses(const std::vector<int32_t>& nodes, cudaStream_t s, bool side, bool defer) {
  std::vector<InvTask> inv[2];
  int max_m[2] = {0, 0};
  double inv_flops[2] = {0.0, 0.0}, inv_bytes[2] = {0.0, 0.0};
  for (int32_t p : nodes) {
    const int m = sz[p];
    if (m == 0) continue;
    if (m > kInvMaxM) fail(LRS_ERR_INVALID_ARG, "a pivot block exceeds the largest the inverse kernels take");
    const int g = m >= kInvClusterMin;
    inv[g].push_back(InvTask{get(p, p).p, g ? F->scratch.take(inv_resident_workspace(m)) : nullptr, m, m});
    max_m[g] = std::max(max_m[g], m);
    flops += 2.0 * m * m * (double)m;
    inv_flops[g] += 2.0 * m * m * (double)m;
    inv_bytes[g] += 16.0 * m * m;
  }
  auto put = [&](const std::vector<InvTask>& v) -> const InvTask* {
    if (!side) return F->stager.put(v);
    InvTask* d = reinterpret_cast<InvTask*>(F->scratch.take((v.size() * sizeof(InvTask) + 7) / 8));
    cuda_check(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(InvTask), cudaMemcpyHostToDevice, st), "inverse tasks");
    return d;
  };
  // large blocks resident in shared memory, in waves on the main stream
  std::vector<std::pair<int, int>> waves;
  if (!inv[1].empty()) {
    std::vector<int> ms, c0(inv[1].size()), cw(inv[1].size());
    for (const InvTask& t : inv[1]) ms.push_back(t.m);
    waves = plan_resident_waves(ms.data(), (int)ms.size(), false, c0.data(), cw.data());
    for (size_t i = 0; i < inv[1].size(); ++i) { inv[1][i].cta0 = c0[i]; inv[1][i].cw = cw[i]; }
  }
  const bool resident = !inv[1].empty() && !waves.empty();
  const bool deferred = resident && defer;
  std::vector<std::pair<const InvTask*, InvTask>> grid_tasks;
  const InvTask* d_small = inv[0].empty() ? nullptr : put(inv[0]);
  const InvTask* d_large = nullptr;
  const InvTask* d_res = resident && !deferred ? F->stager.put(inv[1]) : nullptr;
  // not resident: a few large blocks one whole-GPU launch each, always on the
  // main stream (a cooperative grid never runs beside another stream's work);
  // many: clusters
  const bool large_grid = (int)inv[1].size() <= kGridTeamMaxTasks;
  if (!inv[1].empty() && !resident) {
    if (large_grid)
      for (const InvTask& t : inv[1]) grid_tasks.emplace_back(F->stager.put(std::vector<InvTask>{t}), t);
    else d_large = put(inv[1]);
  }
  // symmetric path: the computed inverse of a symmetric pivot block is
  // symmetric only to rounding; its lower triangle is mirrored onto the upper
  // one so that every later product (and the transposes standing in for half
  // of them) uses one and the same A_pp^{-1}.  mirror_s: the blocks inverted
  // on stream s; mirror_m: those inverted on the main stream.
  std::vector<CopyTask> mirror_s, mirror_m;
  if (sym) {
    for (const InvTask& t : inv[0]) mirror_s.push_back(CopyTask{t.A, t.A, t.lda, t.lda, t.m, t.m, 3, 0.0});
    for (const InvTask& t : inv[1])
      (d_large ? mirror_s : mirror_m).push_back(CopyTask{t.A, t.A, t.lda, t.lda, t.m, t.m, 3, 0.0});
  }
  const CopyTask* d_mirror_s = nullptr;
  if (!mirror_s.empty()) {
    if (side) {
      CopyTask* d = reinterpret_cast<CopyTask*>(F->scratch.take((mirror_s.size() * sizeof(CopyTask) + 7) / 8));
      cuda_check(cudaMemcpyAsync(d, mirror_s.data(), mirror_s.size() * sizeof(CopyTask), cudaMemcpyHostToDevice, st),
                 "mirror tasks");
      d_mirror_s = d;
    } else {
      d_mirror_s = F->stager.put(mirror_s);
    }
  }
  if (deferred) {
    deferred_inv.insert(deferred_inv.end(), inv[1].begin(), inv[1].end());
    deferred_mirror.insert(deferred_mirror.end(), mirror_m.begin(), mirror_m.end());
    waves.clear();
    mirror_m.clear();
  }
  const CopyTask* d_mirror_m = mirror_m.empty() ? nullptr : F->stager.put(mirror_m);
  if (side) {                                       // the side stream starts after the tasks are on the device
    cuda_check(cudaEventRecord(F->ev_fork, st), "fork");
    cuda_check(cudaStreamWaitEvent(s, F->ev_fork, 0), "fork wait");
  }
  if (d_small) {
    cudaEvent_t e = F->prof.start(s);
    cuda_check(launch_invert(d_small, (int)inv[0].size(), max_m[0], TeamKind::Cta, 1, F->status, s), "invert launch");
    F->prof.stop(LRS_PROF_INVERT, e, inv_flops[0], inv_bytes[0], max_m[0], 0, (int)inv[0].size(), s);
  }
  if (d_large) {
    cudaEvent_t e = F->prof.start(s);
    cuda_check(launch_invert(d_large, (int)inv[1].size(), max_m[1], TeamKind::Cluster, kDenseCluster, F->status, s),
               "invert launch");
    F->prof.stop(LRS_PROF_INVERT, e, inv_flops[1], inv_bytes[1], max_m[1], 1, (int)inv[1].size(), s);
  }
  if (d_mirror_s) launch_copy(d_mirror_s, (int)mirror_s.size(), s);
  if (side) cuda_check(cudaEventRecord(F->ev_join, s), "join");
  for (auto [b, e] : waves) {
    double fl = 0.0, by = 0.0;
    int mm = 0;
    for (int i = b; i < e; ++i) {
      const double m = inv[1][i].m;
      fl += 2.0 * m * m * m;
      by += 16.0 * m * m;
      mm = std::max(mm, inv[1][i].m);
    }
    cudaEvent_t ev = F->prof.start();
    cuda_check(launch_invert_resident(d_res + b, inv[1].data() + b, e - b, F->status, st), "invert launch");
    F->prof.stop(LRS_PROF_INVERT, ev, fl, by, mm, 3, e - b);
  }
  for (auto& [d, t] : grid_tasks) {
    cudaEvent_t e = F->prof.start();
    cuda_check(launch_invert(d, 1, t.m, TeamKind::Grid, grid_team_size(t.m, false), F->status, st), "invert launch");
    F->prof.stop(LRS_PROF_INVERT, e, 2.0 * t.m * t.m * (double)t.m, 16.0 * t.m * t.m, t.m, 2, 1);
  }
  if (d_mirror_m) launch_copy(d_mirror_m, (int)mirror_m.size(), st);
}

// The deferred resident inverses alone (a batch without resident reductions),
// in waves on the main stream, then their mirror copies.
void Factorizer::launch_deferred_inverses() {
  if (!deferred_inv.empty()) {
    std::vector<int> ms, c0(deferred_inv.size()), cw(deferred_inv.size());
    for (const InvTask& t : deferred_inv) ms.push_back(t.m);
    auto waves = plan_resident_waves(ms.data(), (int)ms.size(), false, c0.data(), cw.data());
    if (waves.empty()) fail(LRS_ERR_STATE, "resident inverses no longer fit");
    for (size_t i = 0; i < deferred_inv.size(); ++i) { deferred_inv[i].cta0 = c0[i]; deferred_inv[i].cw = cw[i]; }
    const InvTask* d = F->stager.put(deferred_inv);
    for (auto [b, e] : waves) {
      double fl = 0.0, by = 0.0;
      int mm = 0;
      for (int i = b; i < e; ++i) {
        const double m = deferred_inv[i].m;
        fl += 2.0 * m * m * m;
        by += 16.0 * m * m;
        mm = std::max(mm, deferred_inv[i].m);
      }
      cudaEvent_t ev = F->prof.start();
      cuda_check(launch_invert_resident(d + b, deferred_inv.data() + b, e - b, F->status, st), "invert launch");
      F->prof.stop(LRS_PROF_INVERT, ev, fl, by, mm, 3, e - b);
    }
  }
  if (!deferred_mirror.empty()) launch_copy(F->stager.put(deferred_mirror), (int)deferred_mirror.size(), st);
  deferred_inv.clear();
  deferred_mirror.clear();
}

// Eliminate (Sec. 2.2) for a set of nodes with no edge between them: invert
// each pivot block in place, form A_pp^{-1} A_{p,k}, then
// A_{q,k} -= A_{q,p} (A_pp^{-1} A_{p,k}) over all neighbour pairs, summed per
// target block in the order of `nodes`.
void Factorizer::eliminate(const std::vector<int32_t>& nodes,
                           const std::vector<const std::vector<int32_t>*>& nbrs, bool pre_inverted,
                           const SchurGroups& groups) {
  const auto h0 = std::chrono::steady_clock::now();
  struct Acc {
    double& to;
    std::chrono::steady_clock::time_point t0;
    ~Acc() { to += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); }
  } acc{F->stats.host_elim_ms, h0};
  if (!pre_inverted) launch_inverses(nodes, st, false);
  // T_{p,k} = A_pp^{-1} A_{p,k}
  std::vector<std::vector<const double*>> T(nodes.size());
  for (size_t a = 0; a < nodes.size(); ++a) {
    const int32_t p = nodes[a];
    const int m = sz[p];
    for (int32_t k : *nbrs[a]) {
      const int mk = sz[k];
      double* t = (m && mk) ? F->persist.take((size_t)m * mk) : nullptr;
      T[a].push_back(t);
      if (t) add_gemm(t, m, nullptr, 0, m, mk, 0, GemmTerm{get(p, p).p, get(p, k).p, m, m, m, 0}, false, lowp);
    }
  }
  flush_gemm();
  // Schur updates, gathered per target block (groups: built from the same
  // neighbour lists before the batch's sync)
  const auto& pairs = groups.pairs;
  const auto& order = groups.order;
  const auto& first = groups.first;
  std::vector<std::vector<const double*>> Lp(nodes.size());   // A_{q,p} of each pivot's neighbours
  for (size_t a = 0; a < nodes.size(); ++a) {
    const auto& nb = *nbrs[a];
    const int32_t p = nodes[a];
    Lp[a].assign(nb.size(), nullptr);
    for (size_t u = 0; u < nb.size(); ++u)
      if (sz[p] && sz[nb[u]]) Lp[a][u] = get(nb[u], p).p;
  }
  // the product terms of target o
  std::vector<GemmTerm> lst;
  auto terms_of = [&](size_t o) -> const std::vector<GemmTerm>& {
    lst.clear();
    for (int e = first[o]; e < first[o + 1]; ++e) {
      const SchurGroups::Pair& pr = pairs[e];
      const int32_t p = nodes[pr.a];
      const int m = sz[p];
      const int32_t q = (*nbrs[pr.a])[pr.u], k = (*nbrs[pr.a])[pr.v];
      if (m && sz[q] && sz[k]) lst.push_back(GemmTerm{Lp[pr.a][pr.u], T[pr.a][pr.v], sz[q], m, m, 0});
    }
    return lst;
  };
  // symmetric path: A_kq = A_qk^T before and after, so only q <= k is formed
  // (a diagonal block on and below its tile diagonal, then mirrored) and the
  // block (k, q) is the transpose of (q, k); copies run after the products
  std::vector<CopyTask> after;
  std::vector<char> fresh(order.size());
  std::vector<Blk> tgts(order.size());              // one lookup per target
  for (size_t o = 0; o < order.size(); ++o) {        // every target exists before any is read
    auto [q, k] = order[o];
    bool inserted;
    Blk& b = blocks.find_or_insert(key(q, k), inserted);
    if (inserted) b = Blk{arena_for(q, k).take((size_t)sz[q] * sz[k]), sz[q], sz[k]};
    fresh[o] = inserted;
    tgts[o] = b;
  }
  for (size_t o = 0; o < order.size(); ++o) {
    auto [q, k] = order[o];
    const auto& lst = terms_of(o);
    const Blk tgt = tgts[o];
    if (tgt.rows == 0 || tgt.cols == 0) continue;
    if (sym && q > k) {
      if (fresh[o] && lst.empty()) ct.push_back(CopyTask{nullptr, tgt.p, 0, tgt.rows, tgt.rows, tgt.cols, 2, 0.0});
      else if (!lst.empty()) after.push_back(CopyTask{get(k, q).p, tgt.p, sz[k], tgt.rows, tgt.rows, tgt.cols, 1, 0.0});
      continue;
    }
    const bool diag = sym && q == k;
    if (!fresh[o]) {
      if (!lst.empty()) add_gemm(tgt.p, tgt.rows, nullptr, 0, tgt.rows, tgt.cols, kAccumulate | kSubtract, lst, diag, lowp);
    } else if (lst.empty()) {
      ct.push_back(CopyTask{nullptr, tgt.p, 0, tgt.rows, tgt.rows, tgt.cols, 2, 0.0});
    } else {
      add_gemm(tgt.p, tgt.rows, nullptr, 0, tgt.rows, tgt.cols, kSubtract, lst, diag, lowp);
    }
    if (diag && !lst.empty()) after.push_back(CopyTask{tgt.p, tgt.p, tgt.rows, tgt.rows, tgt.rows, tgt.cols, 3, 0.0});
  }
  flush_gemm();
  ct.insert(ct.end(), after.begin(), after.end());
  flush_copy();
  // keep the factor for the solve; remove the nodes from the graph
  for (size_t a = 0; a < nodes.size(); ++a) {
    const int32_t p = nodes[a];
    ElimRecord rec;
    rec.level = level;
    rec.node = p;
    rec.m = sz[p];
    rec.inv = sz[p] ? get(p, p).p : nullptr;
    for (size_t v = 0; v < nbrs[a]->size(); ++v) {
      const int32_t q = (*nbrs[a])[v];
      rec.nbr.push_back(q);
      rec.nbr_m.push_back(sz[q]);
      rec.L.push_back((sz[p] && sz[q]) ? get(q, p).p : nullptr);
      rec.T.push_back(T[a][v]);
      blocks.erase(key(q, p));
      blocks.erase(key(p, q));
    }
    blocks.erase(key(p, p));
    F->recs.push_back(std::move(rec));
  }
}

// Adds the wall time of its scope to a host-time counter (ms).
struct HostTimer {
  double& to;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  explicit HostTimer(double& t) : to(t) {}
  ~HostTimer() { to += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); }
};

void Factorizer::batch(const LevelPlan& lp, const std::vector<int32_t>& js) {
  double compress_ms = 0.0;
  std::unique_ptr<HostTimer> tc(new HostTimer(compress_ms));
  // --- C: Gram matrix and spectrum of every stacked well-separated block
  std::vector<EigTask> eig;
  std::vector<int32_t> eig_j;
  F->scratch.reset();
  const size_t nb = js.size();
  {
    // the super-nodes' pivot blocks are final now: invert them on the side
    // stream while the compression runs on the main stream
    std::vector<int32_t> snodes;
    for (int32_t j : js) snodes.push_back(local_node(j, kSlotS));
    launch_inverses(snodes, F->side, true, /*defer=*/true);
  }
  int* d_rank = reinterpret_cast<int*>(F->scratch.take(nb));
  std::vector<int64_t> sig_at(nb, -1);
  int64_t sig_total = 0;
  std::vector<double*> Vs(nb, nullptr);
  // spectra on a team of CTAs: every block of at least kEigClusterMin, and
  // all of them when the batch has fewer than half as many as there are SMs
  // (one CTA each would leave most SMs idle)
  int n_spec = 0;
  for (size_t a = 0; a < nb; ++a) {
    const int32_t j = js[a];
    if (!lp.ws[j].empty() && sz[local_node(j, kSlotS)] > 0) ++n_spec;
  }
  const int team_min = n_spec < kFewSpectra ? 1 : kEigClusterMin;
  int n_large = 0;
  bool large_resident = true;          // every large spectrum reduced in shared memory, then sub-teams
  for (size_t a = 0; a < nb; ++a) {
    const int32_t j = js[a];
    const int m = sz[local_node(j, kSlotS)];
    if (!lp.ws[j].empty() && m >= team_min) {
      ++n_large;
      large_resident = large_resident && resident_fits(m, true);
    }
  }
  const bool large_on_grid = n_large <= kGridTeamMaxTasks;
  // without the resident reduction the one-CTA form keeps every m < kEigClusterMin
  const int eig_large_min = large_resident ? team_min : kEigClusterMin;
  for (size_t a = 0; a < nb; ++a) {
    const int32_t j = js[a], s = local_node(j, kSlotS);
    const int m = sz[s];
    const auto& ws = lp.ws[j];
    if (ws.empty() || m == 0) continue;
    int rho = 0;
    std::vector<GemmTerm> terms;
    for (int32_t p : ws) {
      const int mp = sz[p];
      rho += 2 * mp;
      if (mp == 0) continue;
      const double* Ak = get(p, s).p;
      terms.push_back(GemmTerm{Ak, Ak, mp, mp, mp, 1});                   // A_k^T A_k
      if (!sym) {
        const double* Bk = get(s, p).p;
        terms.push_back(GemmTerm{Bk, Bk, m, m, mp, 2});                   // B_k^T B_k
      }
    }
    if (rho == 0) continue;
    if (m > kEigMaxM) fail(LRS_ERR_INVALID_ARG, "a compression block exceeds the largest the spectrum kernels take");
    double* G = F->scratch.take((size_t)m * m);
    int warps = 8;
    if (m >= eig_large_min)
      warps = large_resident ? 8 * kMaxTeam : large_on_grid ? 8 * grid_team_size(m, true) : 8 * kDenseCluster;
    double* W = F->scratch.take(eig_workspace(m, warps));
    double* V = F->scratch.take((size_t)m * m);
    sig_at[a] = sig_total;
    sig_total += m;
    Vs[a] = V;
    add_gemm(G, m, nullptr, 0, m, m, 0, terms, /*lower_only=*/true, lowp_gram);   // G is symmetric
    // symmetric: B_k = A_k^T, so M^T M = 2 sum A_k^T A_k (Sec. 4.3)
    eig.push_back(EigTask{G, W, V, nullptr, d_rank + a, m, rho, F->eps, sym ? 2.0 : 1.0});
    eig.back().trunc_rule = F->trunc_rule;
    eig.back().below_sq = &F->status->below_sq;
    eig_j.push_back((int32_t)a);
  }
  double* d_sig = F->scratch.take((size_t)std::max<int64_t>(sig_total, 1));
  for (size_t e = 0; e < eig.size(); ++e) eig[e].sigma = d_sig + sig_at[eig_j[e]];
  flush_gemm();
  {
    // spectra: small Gram matrices one CTA each (in shared memory); large ones
    // on a cluster each, or, when the batch has only a few, on the whole GPU
    std::vector<EigTask> small, large;
    int smax = 0, lmax = 0;
    double sbytes = 0.0, lbytes = 0.0;
    for (const EigTask& t : eig) {
      const double b = 8.0 * ((double)t.m * t.m * 2 + t.m);
      if (t.m >= eig_large_min) { large.push_back(t); lmax = std::max(lmax, t.m); lbytes += b; }
      else { small.push_back(t); smax = std::max(smax, t.m); sbytes += b; }
    }
    if (!small.empty()) {
      const EigTask* d = F->stager.put(small);
      cudaEvent_t e = F->prof.start();
      cuda_check(launch_eig(d, (int)small.size(), smax, TeamKind::Cta, 1, F->status, st), "spectrum launch");
      F->prof.stop(LRS_PROF_SPECTRUM, e, 0.0, sbytes, smax, 0, (int)small.size());   // flops: device counter
    }
    // large ones: the Householder reduction resident in shared memory (waves
    // on teams of CTAs), then the rest of each spectrum on a cluster per
    // block, or on the whole GPU when the batch has only a few
    std::vector<std::pair<int, int>> waves;
    if (!large.empty()) {
      std::vector<int> ms, c0(large.size()), cw(large.size());
      for (const EigTask& t : large) ms.push_back(t.m);
      waves = plan_resident_waves(ms.data(), (int)ms.size(), true, c0.data(), cw.data());
      if (!waves.empty())
        for (size_t i = 0; i < large.size(); ++i) {
          large[i].cta0 = c0[i];
          large[i].cw = cw[i];
          large[i].H = F->scratch.take(tridiag_resident_workspace(large[i].m));
        }
    }
    // the super-nodes' large inverses (deferred at the batch's start; they do
    // not depend on the compression) share the reductions' waves: one
    // cooperative launch per wave, inverses first, each team on its own CTAs.
    // Such a launch is timed as spectrum (kind 5), with the inverses' flops.
    std::vector<std::pair<int, int>> mixed;
    const int ni = (int)deferred_inv.size();
    if (!waves.empty() && ni > 0) {
      const int nt = ni + (int)large.size();
      std::vector<int> ms, c0(nt), cw(nt);
      std::vector<char> kinds;
      for (const InvTask& t : deferred_inv) { ms.push_back(t.m); kinds.push_back(0); }
      for (const EigTask& t : large) { ms.push_back(t.m); kinds.push_back(1); }
      mixed = plan_mixed_waves(ms.data(), kinds.data(), nt, c0.data(), cw.data());
      for (auto [b, e] : mixed) {
        // CTAs of the wave's inverses come first; the reductions count from their end
        int inv_ctas = 0;
        for (int i = b; i < std::min(e, ni); ++i) inv_ctas = std::max(inv_ctas, c0[i] + (ms[i] + cw[i] - 1) / cw[i]);
        for (int i = b; i < e; ++i) {
          if (i < ni) {
            deferred_inv[i].cta0 = c0[i];
            deferred_inv[i].cw = cw[i];
          } else {
            large[i - ni].cta0 = c0[i] - inv_ctas;
            large[i - ni].cw = cw[i];
          }
        }
      }
    }
    const EigTask* d_large = large.empty() ? nullptr : F->stager.put(large);
    if (!mixed.empty()) {
      const InvTask* d_inv = F->stager.put(deferred_inv);
      for (auto [b, e] : mixed) {
        const int ib = b, ie = std::min(e, ni), eb = std::max(b, ni) - ni, ee = e - ni;
        int mm = 0;
        double by = 0.0, fl = 0.0;                      // flops: the inverses' (the spectra's come from the device)
        for (int i = ib; i < ie; ++i) {
          const double mi = deferred_inv[i].m;
          by += 16.0 * mi * mi;
          fl += 2.0 * mi * mi * mi;
        }
        for (int i = eb; i < ee; ++i) {
          mm = std::max(mm, large[i].m);
          by += 8.0 * (double)large[i].m * large[i].m;
        }
        cudaEvent_t ev = F->prof.start();
        cuda_check(launch_resident_mix(d_inv + ib, deferred_inv.data() + ib, std::max(0, ie - ib), d_large + eb,
                                       large.data() + eb, std::max(0, ee - eb), F->status, st),
                   "inverse and reduction launch");
        F->prof.stop(LRS_PROF_SPECTRUM, ev, fl, by, mm, 5, e - b);
      }
      if (!deferred_mirror.empty()) launch_copy(F->stager.put(deferred_mirror), (int)deferred_mirror.size(), st);
      deferred_inv.clear();
      deferred_mirror.clear();
    } else {
      launch_deferred_inverses();
      for (auto [b, e] : waves) {
        int mm = 0;
        double by = 0.0;
        for (int i = b; i < e; ++i) {
          mm = std::max(mm, large[i].m);
          by += 8.0 * (double)large[i].m * large[i].m;
        }
        cudaEvent_t ev = F->prof.start();
        cuda_check(launch_tridiag_resident(d_large + b, large.data() + b, e - b, F->status, st), "reduction launch");
        F->prof.stop(LRS_PROF_SPECTRUM, ev, 0.0, by, mm, 3, e - b);
      }
    }
    if (!large.empty() && !waves.empty()) {
      // every block of the batch on its own sub-team of CTAs, in one launch
      // per wave (the latency-bound phases of different blocks overlap)
      std::vector<int> ms, t0(large.size()), tsz(large.size());
      for (const EigTask& t : large) ms.push_back(t.m);
      const int cap = sub_team_capacity(lmax);
      auto sw = plan_sub_teams(ms.data(), (int)ms.size(), cap, t0.data(), tsz.data());
      unsigned long long* bars =
          reinterpret_cast<unsigned long long*>(F->scratch.take(4 * large.size()));
      cuda_check(cudaMemsetAsync(bars, 0, 4 * large.size() * sizeof(unsigned long long), st), "barriers");
      for (size_t i = 0; i < large.size(); ++i) {
        large[i].team0 = t0[i];
        large[i].team_size = tsz[i];
        large[i].bar = bars + 4 * i;
      }
      const EigTask* d_sub = F->stager.put(large);
      for (auto [b, e] : sw) {
        int mm = 0, ctas = 0;
        double by = 0.0;
        for (int i = b; i < e; ++i) {
          mm = std::max(mm, large[i].m);
          ctas = std::max(ctas, large[i].team0 + large[i].team_size);
          by += 8.0 * ((double)large[i].m * large[i].m * 2 + large[i].m);
        }
        cudaEvent_t ev = F->prof.start();
        cuda_check(launch_eig(d_sub + b, e - b, mm, TeamKind::Sub, ctas, F->status, st), "spectrum launch");
        F->prof.stop(LRS_PROF_SPECTRUM, ev, 0.0, by, mm, 4, e - b);
      }
    } else if (!large.empty() && !large_on_grid) {
      cudaEvent_t e = F->prof.start();
      cuda_check(launch_eig(d_large, (int)large.size(), lmax, TeamKind::Cluster, kDenseCluster, F->status, st),
                 "spectrum launch");
      F->prof.stop(LRS_PROF_SPECTRUM, e, 0.0, lbytes, lmax, 1, (int)large.size());
    } else {
      for (size_t i = 0; i < large.size(); ++i) {
        const EigTask& t = large[i];
        cudaEvent_t e = F->prof.start();
        cuda_check(launch_eig(d_large + i, 1, t.m, TeamKind::Grid, grid_team_size(t.m, true), F->status, st),
                   "spectrum launch");
        F->prof.stop(LRS_PROF_SPECTRUM, e, 0.0, 8.0 * ((double)t.m * t.m * 2 + t.m), t.m, 2, 1);
      }
    }
  }
  launch_deferred_inverses();                       // when no resident reduction took them
  // the eliminations' Schur structure depends on the neighbour lists alone:
  // build it now, while the device computes the spectra
  SchurGroups groups_s, groups_b;
  {
    std::vector<const std::vector<int32_t>*> ns, nbb;
    for (int32_t j : js) {
      ns.push_back(&lp.nbs[j]);
      nbb.push_back(&lp.nbb[j]);
    }
    groups_s.build(ns);
    groups_b.build(nbb);
  }
  std::vector<int> rank(nb, 0);
  std::vector<double> sig(sig_total);
  tc.reset();
  {
    // the one sync of the batch (the copies into pageable memory wait for the
    // stream, and so does the flush)
    const auto w0 = std::chrono::steady_clock::now();
    if (!eig.empty()) {
      cuda_check(cudaMemcpyAsync(rank.data(), d_rank, nb * sizeof(int), cudaMemcpyDeviceToHost, st), "ranks");
      if (sig_total)
        cuda_check(cudaMemcpyAsync(sig.data(), d_sig, sig_total * sizeof(double), cudaMemcpyDeviceToHost, st),
                   "sigma");
    }
    F->stager.flush();
    F->stats.host_wait_ms +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  }
  tc.reset(new HostTimer(compress_ms));
  for (size_t a = 0; a < nb; ++a) if (sig_at[a] < 0) rank[a] = 0;
  // --- A: new nodes b, P(b) and the edges of the Sec. 4.3 edge rules
  for (size_t a = 0; a < nb; ++a) {
    const int32_t j = js[a], s = local_node(j, kSlotS), b = local_node(j, kSlotB), Pn = local_node(j, kSlotP);
    const int m = sz[s], r = rank[a];
    sz[b] = sz[Pn] = r;
    F->ranks.push_back(r);
    F->sigma_off.push_back((int64_t)F->sigma_all.size());
    if (sig_at[a] >= 0) {
      int rho = 0;
      for (int32_t p : lp.ws[j]) rho += 2 * sz[p];
      const int nsv = std::min(rho, m);
      F->sigma_all.insert(F->sigma_all.end(), sig.begin() + sig_at[a], sig.begin() + sig_at[a] + nsv);
    }
    F->stats.max_rank = std::max(F->stats.max_rank, r);
    for (int32_t p : lp.ws[j]) {
      if (r > 0 && sz[p] > 0) {
        const Blk Apk = get(p, s), Bpk = get(s, p);
        Blk R = make(p, Pn), QT = make(Pn, p);
        add_gemm(R.p, R.rows, nullptr, 0, sz[p], r, 0, GemmTerm{Apk.p, Vs[a], sz[p], m, m, 0}, false, lowp);
        if (sym) ct.push_back(CopyTask{R.p, QT.p, sz[p], r, r, sz[p], 1, 0.0});   // Q_k^T = R_k^T
        else add_gemm(QT.p, QT.rows, nullptr, 0, r, sz[p], 0, GemmTerm{Vs[a], Bpk.p, m, m, m, 1}, false, lowp);
      } else {
        make(p, Pn);
        make(Pn, p);
      }
    }
    Blk bs = make(b, s), sb = make(s, b), bP = make(b, Pn), Pb = make(Pn, b);
    if (r > 0 && m > 0) {
      ct.push_back(CopyTask{Vs[a], bs.p, m, r, r, m, 1, 0.0});   // s -> b carries V^T
      ct.push_back(CopyTask{Vs[a], sb.p, m, m, m, r, 0, 0.0});   // b -> s carries V
    }
    if (r > 0) {
      ct.push_back(CopyTask{nullptr, bP.p, 0, r, r, r, 2, -1.0});  // b <-> P(b) carry -I
      ct.push_back(CopyTask{nullptr, Pb.p, 0, r, r, r, 2, -1.0});
    }
  }
  flush_gemm();
  flush_copy();
  for (size_t a = 0; a < nb; ++a) {
    const int32_t j = js[a], s = local_node(j, kSlotS);
    for (int32_t p : lp.ws[j]) {
      blocks.erase(key(s, p));
      blocks.erase(key(p, s));
    }
  }
  F->stats.n_compress += (int64_t)nb;
  tc.reset();
  F->stats.host_compress_ms += compress_ms;
  // --- S and B: eliminate the super-nodes, then their black-nodes
  std::vector<int32_t> nodes;
  std::vector<const std::vector<int32_t>*> nbrs;
  for (int32_t j : js) { nodes.push_back(local_node(j, kSlotS)); nbrs.push_back(&lp.nbs[j]); }
  const int r0 = (int)F->recs.size();
  cuda_check(cudaStreamWaitEvent(st, F->ev_join, 0), "join wait");
  eliminate(nodes, nbrs, true, groups_s);
  F->phases.emplace_back(r0, (int)F->recs.size() - r0);
  nodes.clear();
  nbrs.clear();
  for (int32_t j : js) { nodes.push_back(local_node(j, kSlotB)); nbrs.push_back(&lp.nbb[j]); }
  const int r1 = (int)F->recs.size();
  eliminate(nodes, nbrs, false, groups_b);
  F->phases.emplace_back(r1, (int)F->recs.size() - r1);
  for (int32_t j : js) {             // pivot sizes in Algorithm 1's order: s_j, then b_j
    F->pivots.push_back(sz[local_node(j, kSlotS)]);
    F->pivots.push_back(sz[local_node(j, kSlotB)]);
  }
}

void Factorizer::run(const double* d_val) {
  const int L = P.depth;
  // the symmetric path: asserted, or detected from the values (pattern and
  // values exactly symmetric)
  sym = F->symmetry == LRS_SYM_SYMMETRIC;
  if (F->symmetry == LRS_SYM_DETECT && !P.tpos.empty() && P.nnz > 0) {
    int64_t* d_tpos = reinterpret_cast<int64_t*>(F->scratch.take((size_t)P.nnz));
    cuda_check(cudaMemcpyAsync(d_tpos, P.tpos.data(), P.nnz * sizeof(int64_t), cudaMemcpyHostToDevice, st), "tpos");
    launch_asymmetry(d_val, d_tpos, P.nnz, F->status, st);
    int asym = 1;
    cuda_check(cudaMemcpyAsync(&asym, &F->status->asymmetric, sizeof(int), cudaMemcpyDeviceToHost, st), "symmetry");
    cuda_check(cudaStreamSynchronize(st), "symmetry test");
    sym = asym == 0;
    F->scratch.reset();
  }
  F->stats.symmetric = sym ? 1 : 0;
  lowp = F->precision == LRS_PREC_FP32;
  lowp_gram = lowp && F->eps >= LRS_PREC_FP32_GRAM_EPS;
  F->stats.precision = F->precision;
  F->off_red.assign(L + 1, {});
  F->off_black.assign(L + 1, {});
  std::vector<int> redsz(size_t(1) << L);
  for (int32_t c = 0; c < (int32_t(1) << L); ++c) redsz[c] = P.leaf_off[c + 1] - P.leaf_off[c];
  F->off_red[L].assign(P.leaf_off.begin(), P.leaf_off.end() - 1);
  int64_t ext = P.n;
  BlockMap old;
  for (const LevelPlan& lp : P.levels) {
    level = lp.level;
    const int32_t ns = lp.nsuper;
    sz.assign(3 * (size_t)ns, 0);
    for (int32_t j = 0; j < ns; ++j) sz[local_node(j, kSlotS)] = redsz[2 * j] + redsz[2 * j + 1];
    blocks.reset(96 * (size_t)ns, 3 * (size_t)ns);   // the level's blocks with their fill-in, without rehashing
    {
      HostTimer tm(F->stats.host_merge_ms);
      if (level == L) assemble_leaf(d_val);
      else merge(old, redsz);
    }
    if (F->trunc_rule == LRS_TRUNC_CUROFF6) add_level_norm();
    F->trans[level & 1].reset();        // red-red blocks of the level below were consumed by the merge
    for (const auto& b : lp.batches) {
      batch(lp, b);
      ++F->stats.n_batches;
    }
    for (int32_t j = 0; j < ns; ++j) F->stats.max_pivot = std::max(F->stats.max_pivot, sz[local_node(j, kSlotS)]);
    // place black-nodes of level i and red-nodes of level i-1 in x_e
    F->off_black[level].resize(ns);
    for (int32_t j = 0; j < ns; ++j) { F->off_black[level][j] = ext; ext += sz[local_node(j, kSlotB)]; }
    F->off_red[level - 1].resize(ns);
    redsz.assign(ns, 0);
    for (int32_t j = 0; j < ns; ++j) {
      F->off_red[level - 1][j] = ext;
      redsz[j] = sz[local_node(j, kSlotP)];
      ext += redsz[j];
    }
    old.swap(blocks);
  }
  F->ext_n = ext;
  F->stats.flops_factor = flops;
  F->stats.flops_factor_f32 = flops32;
}

}  // namespace

void run_factor(lrs_factor_t* F, const double* val, int val_on_device) {
  const lrs_plan& P = *F->plan;
  Factorizer fz(F);
  const double* d_val = val;
  double* owned = nullptr;
  if (!val_on_device) {
    owned = static_cast<double*>(F->al.get(std::max<size_t>(P.nnz, 1) * sizeof(double)));
    cuda_check(cudaMemcpyAsync(owned, val, P.nnz * sizeof(double), cudaMemcpyHostToDevice, F->stream), "values");
    d_val = owned;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, F->stream);
  try {
    const auto h0 = std::chrono::steady_clock::now();
    F->stats.host_wait_ms = 0.0;
    F->stats.host_elim_ms = 0.0;
    F->stats.host_merge_ms = 0.0;
    F->stats.host_compress_ms = 0.0;
    fz.run(d_val);
    F->stats.host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0).count();
  } catch (...) {
    cudaStreamSynchronize(F->stream);
    if (owned) F->al.put(owned, P.nnz * sizeof(double));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventRecord(e1, F->stream);
  cuda_check(cudaStreamSynchronize(F->stream), "factor");
  F->emu_ws.release();                              // digit slices: needed only while factoring
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  F->stats.factor_ms = ms;
  // keep the values of A for the GMRES products
  if (owned) F->d_val = owned;
  else {
    F->d_val = static_cast<double*>(F->al.get(std::max<size_t>(P.nnz, 1) * sizeof(double)));
    cuda_check(cudaMemcpyAsync(F->d_val, val, P.nnz * sizeof(double), cudaMemcpyDeviceToDevice, F->stream), "values");
  }
  DeviceStatus hs{};
  cuda_check(cudaMemcpy(&hs, F->status, sizeof(hs), cudaMemcpyDeviceToHost), "status");
  F->prof.collect();
  if (F->prof.on) F->prof.acc[LRS_PROF_SPECTRUM].flops += (double)hs.eig_flops;
  F->stats.eig_flops = (double)hs.eig_flops;
  for (int k = 0; k < 5; ++k) {
    F->stats.eig_cycles[k] = (double)hs.eig_cycles[k];
    F->stats.eig_lead_ms[k] = (double)hs.eig_lead_ns[k] * 1e-6;
  }
  if (hs.singular) fail(LRS_ERR_SINGULAR_PIVOT, "singular pivot block");
  if (hs.numeric) fail(LRS_ERR_NUMERIC, "NaN or Inf in the factorization");
  if (hs.wait_timeout) fail(LRS_ERR_TIMEOUT, "a wait between the CTAs of a dense kernel expired");
  F->stats.depth = P.depth;
  F->stats.n = P.n;
  F->stats.ext_n = F->ext_n;
  F->stats.factor_bytes = (int64_t)(F->persist.held());
}

void move_factor_to_f32(lrs_factor_t* F) {
  // one region, each block starting on a 32-float (128-byte) boundary
  auto pad = [](int64_t c) { return (c + 31) & ~int64_t(31); };
  int64_t total = 0;
  for (const ElimRecord& r : F->recs) {
    total += pad((int64_t)r.m * r.m);
    for (size_t v = 0; v < r.nbr.size(); ++v) total += 2 * pad((int64_t)r.m * r.nbr_m[v]);
  }
  float* base = reinterpret_cast<float*>(F->store32.take((size_t)std::max<int64_t>((total + 1) / 2, 1)));
  std::vector<ConvTask> tasks;
  int64_t at = 0;
  auto move = [&](const double* src, int64_t count) -> const float* {
    if (!src || count <= 0) return nullptr;
    float* dst = base + at;
    at += pad(count);
    tasks.push_back(ConvTask{src, dst, count});
    return dst;
  };
  for (ElimRecord& r : F->recs) {
    r.inv32 = move(r.inv, (int64_t)r.m * r.m);
    r.L32.assign(r.nbr.size(), nullptr);
    r.T32.assign(r.nbr.size(), nullptr);
    for (size_t v = 0; v < r.nbr.size(); ++v) {
      r.L32[v] = move(r.L[v], (int64_t)r.nbr_m[v] * r.m);
      r.T32[v] = move(r.T[v], (int64_t)r.m * r.nbr_m[v]);
    }
  }
  if (!tasks.empty()) {
    const ConvTask* d = F->stager.put(tasks);
    launch_to_f32(d, (int)tasks.size(), F->stream);
    cuda_check(cudaGetLastError(), "factor to FP32");
  }
  cuda_check(cudaStreamSynchronize(F->stream), "factor to FP32");
  F->stager.flush();
  for (ElimRecord& r : F->recs) {                 // the FP64 blocks go away
    r.inv = nullptr;
    std::fill(r.L.begin(), r.L.end(), nullptr);
    std::fill(r.T.begin(), r.T.end(), nullptr);
  }
  F->persist.release();
  F->apply32 = true;
  F->prog.nrhs = 0;
  F->stats.factor_bytes = (int64_t)F->store32.held();
}


}  // namespace lrs

int64_t lrs_factor::node_offset(int level, int32_t v) const {
  const int32_t j = lrs::local_cluster(v);
  switch (lrs::local_slot(v)) {
    case lrs::kSlotS: return off_red[level][2 * j];
    case lrs::kSlotB: return off_black[level][j];
    default: return off_red[level - 1][j];
  }
}
