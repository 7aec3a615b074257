// lrs_oracle.cpp -- plain FP64 CPU oracle of the hierarchical sparse solver of
// Pouransari, Coulier & Darve, "Fast hierarchical solvers for sparse matrices
// using extended sparsification and low-rank approximation" (arXiv 1510.07363).
//
// TEST INFRASTRUCTURE.  This library exists to check the CUDA library against
// the paper.  Only the test suite, the package smoke check and the CPU
// baseline of the benchmark load it; the product path never does.  It shares
// no code, header or table with the CUDA library: the only common ground is
// the seeded input generators, which hold none of the method's arithmetic.
//
// Style: sequential, unblocked, std containers, one routine per step of the
// paper, each citing the passage it follows.  Speed is not a goal.
//
// Readings of the paper that this file fixes (the paper is silent on them):
//  * nested partitioning (Sec. 3, nested partitionings): recursive coordinate
//    bisection.  Split a cluster along the axis of largest coordinate extent
//    (ties: lowest axis), stable-sorted by (coordinate, index); child 0 gets
//    the first floor(|S|/2) indices.  Depth l = ceil(log2(n / leaf)).
//  * edges are kept for both directions of every adjacent pair (Def. adj is
//    symmetric); a direction with no stored entries is a zero block.
//  * in-level elimination order (Sec. 6 item 6 allows any order): greedy
//    batches of super-nodes with no edge between them, scanned by ascending
//    cluster index, each batch processed in ascending cluster index.
//  * truncation (eq. cutOff1): r = #{k < min(rho, m) : sigma_k >= eps*sigma_0},
//    r = 0 when there is no well-separated neighbour or sigma_0 = 0.  At
//    eps = 0 every singular value is kept and the factorization is exact.
//    The rule is applied as printed, with no absolute floor: a stacked block
//    that is zero in exact arithmetic but carries rounding-level fill keeps
//    the ranks its computed singular values give.
//  * zero-rank compressions still create the (empty) black node, its red
//    parent and their edges, so the block pattern does not depend on ranks.
//  * pivot blocks are factored by LU with partial pivoting inside the block;
//    an exactly zero pivot is reported as a singular pivot.
//  * GMRES (Saad & Schultz 1986, cited in Sec. 5.2): restarted, modified
//    Gram-Schmidt Arnoldi, Givens rotations, x0 = 0, preconditioner applied
//    on the right (A M y = b, x = M y) so that the GMRES residual is the true
//    residual of eq. accres; convergence is confirmed on the true residual.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <set>
#include <utility>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Dense column-major blocks and the textbook kernels the method calls.
// ---------------------------------------------------------------------------

struct Block {
  int r = 0, c = 0;
  std::vector<double> a;
  Block() {}
  Block(int rows, int cols) : r(rows), c(cols), a((size_t)rows * cols, 0.0) {}
  double& at(int i, int j) { return a[(size_t)j * r + i]; }
  double at(int i, int j) const { return a[(size_t)j * r + i]; }
};

// C -= A * B
void gemm_sub(const Block& A, const Block& B, Block& C) {
  for (int j = 0; j < C.c; ++j)
    for (int k = 0; k < A.c; ++k) {
      double b = B.at(k, j);
      if (b == 0.0) continue;
      for (int i = 0; i < C.r; ++i) C.at(i, j) -= A.at(i, k) * b;
    }
}

// A * B
Block gemm(const Block& A, const Block& B) {
  Block C(A.r, B.c);
  for (int j = 0; j < C.c; ++j)
    for (int k = 0; k < A.c; ++k) {
      double b = B.at(k, j);
      for (int i = 0; i < C.r; ++i) C.at(i, j) += A.at(i, k) * b;
    }
  return C;
}

Block transpose(const Block& A) {
  Block T(A.c, A.r);
  for (int j = 0; j < A.c; ++j)
    for (int i = 0; i < A.r; ++i) T.at(j, i) = A.at(i, j);
  return T;
}

// LU with partial pivoting, in place (Doolittle; unit lower L below the
// diagonal, U on and above).  piv[k] is the row swapped with row k at step k.
// The first row of largest magnitude wins a tie.  Returns false on an exactly
// zero pivot.
bool lu_factor(Block& A, std::vector<int>& piv) {
  const int m = A.r;
  piv.assign(m, 0);
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = std::fabs(A.at(k, k));
    for (int i = k + 1; i < m; ++i)
      if (std::fabs(A.at(i, k)) > best) { best = std::fabs(A.at(i, k)); p = i; }
    piv[k] = p;
    if (best == 0.0) return false;
    if (p != k)
      for (int j = 0; j < m; ++j) std::swap(A.at(k, j), A.at(p, j));
    const double d = A.at(k, k);
    for (int i = k + 1; i < m; ++i) A.at(i, k) /= d;
    for (int j = k + 1; j < m; ++j) {
      const double u = A.at(k, j);
      if (u == 0.0) continue;
      for (int i = k + 1; i < m; ++i) A.at(i, j) -= A.at(i, k) * u;
    }
  }
  return true;
}

// Overwrite B (m x c) with A^{-1} B using the factors from lu_factor.
void lu_solve(const Block& LU, const std::vector<int>& piv, double* B, int m, int c, int ldb) {
  for (int j = 0; j < c; ++j) {
    double* b = B + (size_t)j * ldb;
    for (int k = 0; k < m; ++k)
      if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    for (int k = 0; k < m; ++k)
      for (int i = k + 1; i < m; ++i) b[i] -= LU.at(i, k) * b[k];
    for (int k = m - 1; k >= 0; --k) {
      b[k] /= LU.at(k, k);
      for (int i = 0; i < k; ++i) b[i] -= LU.at(i, k) * b[k];
    }
  }
}

Block lu_solve_block(const Block& LU, const std::vector<int>& piv, const Block& B) {
  Block X = B;
  lu_solve(LU, piv, X.a.data(), X.r, X.c, X.r);
  return X;
}

// R factor of a Householder QR of the tall matrix Y (rows >= cols); only the
// upper-triangular cols x cols factor is returned (the orthogonal factor is
// not needed: the right singular vectors of Y and R coincide).
Block householder_r(Block Y) {
  const int rows = Y.r, cols = Y.c;
  for (int k = 0; k < cols; ++k) {
    double norm2 = 0.0;
    for (int i = k; i < rows; ++i) norm2 += Y.at(i, k) * Y.at(i, k);
    const double norm = std::sqrt(norm2);
    if (norm == 0.0) continue;
    const double alpha = Y.at(k, k) >= 0.0 ? -norm : norm;   // new diagonal
    std::vector<double> v(rows - k);
    for (int i = k; i < rows; ++i) v[i - k] = Y.at(i, k);
    v[0] -= alpha;
    double vv = 0.0;
    for (double x : v) vv += x * x;
    if (vv == 0.0) continue;
    for (int j = k; j < cols; ++j) {
      double dot = 0.0;
      for (int i = k; i < rows; ++i) dot += v[i - k] * Y.at(i, j);
      const double f = 2.0 * dot / vv;
      for (int i = k; i < rows; ++i) Y.at(i, j) -= f * v[i - k];
    }
  }
  Block R(cols, cols);
  for (int j = 0; j < cols; ++j)
    for (int i = 0; i <= j; ++i) R.at(i, j) = Y.at(i, j);
  return R;
}

// Singular values and right singular vectors of M (rho x m), largest first,
// by one-sided Jacobi (Hestenes 1958) on M itself (rho <= m) or on the R
// factor of its QR decomposition (rho > m).  sigma has min(rho, m) entries;
// W is m x m orthogonal with W(:,k) the k-th right singular vector.
void svd_right(const Block& M, std::vector<double>& sigma, Block& W) {
  const int m = M.c;
  Block Y = (M.r > m) ? householder_r(M) : M;
  const int k = Y.r;
  W = Block(m, m);
  for (int i = 0; i < m; ++i) W.at(i, i) = 1.0;
  const double tol = 1e-15;
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = 0; i < k; ++i) {
          alpha += Y.at(i, p) * Y.at(i, p);
          beta += Y.at(i, q) * Y.at(i, q);
          gamma += Y.at(i, p) * Y.at(i, q);
        }
        if (gamma == 0.0 || std::fabs(gamma) <= tol * std::sqrt(alpha * beta)) continue;
        rotated = true;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t);
        const double s = c * t;
        for (int i = 0; i < k; ++i) {
          const double yp = Y.at(i, p), yq = Y.at(i, q);
          Y.at(i, p) = c * yp - s * yq;
          Y.at(i, q) = s * yp + c * yq;
        }
        for (int i = 0; i < m; ++i) {
          const double wp = W.at(i, p), wq = W.at(i, q);
          W.at(i, p) = c * wp - s * wq;
          W.at(i, q) = s * wp + c * wq;
        }
      }
    if (!rotated) break;
  }
  std::vector<double> norms(m);
  for (int j = 0; j < m; ++j) {
    double s2 = 0.0;
    for (int i = 0; i < k; ++i) s2 += Y.at(i, j) * Y.at(i, j);
    norms[j] = std::sqrt(s2);
  }
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return norms[a] > norms[b]; });
  Block Ws(m, m);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) Ws.at(i, j) = W.at(i, order[j]);
  W = Ws;
  const int nsv = std::min(M.r, m);
  sigma.resize(nsv);
  for (int j = 0; j < nsv; ++j) sigma[j] = norms[order[j]];
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// H-tree nodes (Def. Htree).  Every node belongs to one cluster of the nested
// partitioning; a cluster is named by its heap index h = 2^level + j (j the
// 0-based index within its level).  Node ids are 4*h + kind:
//   red(i, j)   : cluster j of P_i,               kind 0
//   super(i, j) : pair red(i,2j), red(i,2j+1);    cluster j of P_{i-1}, kind 1
//   black(i, j) : parent of super(i, j);          cluster j of P_{i-1}, kind 2
// and the parent of black(i, j) is red(i-1, j), the same cluster.
// ---------------------------------------------------------------------------

enum { RED = 0, SUPER = 1, BLACK = 2 };

inline int red_id(int i, int j) { return (((1 << i) + j) << 2) | RED; }
inline int super_id(int i, int j) { return (((1 << (i - 1)) + j) << 2) | SUPER; }
inline int black_id(int i, int j) { return (((1 << (i - 1)) + j) << 2) | BLACK; }
inline int cluster_of(int id) { return id >> 2; }
inline int kind_of(int id) { return id & 3; }
inline int level_of_heap(int h) { int l = 0; while (h > 1) { h >>= 1; ++l; } return l; }

struct ElimRecord {          // one eliminated node, kept for the solve (Alg. 2-4)
  int node = 0;
  Block lu;                  // LU factors of Mat(e_{p->p})
  std::vector<int> piv;
  std::vector<int> nbr;      // neighbours at elimination time (all eliminated later)
  std::vector<Block> Lq;     // Mat(e_{p->q}) = A_{q,p}
  std::vector<Block> Uq;     // Mat(e_{q->p}) = A_{p,q}
};

struct CompressRecord {      // one Compress(s) (Sec. 4.3)
  int snode = 0;
  std::vector<int> ws;       // well-separated neighbours p_1..p_t
  int rho = 0, m = 0, r = 0;
  std::vector<double> sigma;
  double below = 0.0;        // eq. curOff6: ||all levels below||_F at this compression
  Block M;                   // the stacked matrix of eq. lra, kept on request
  Block V;                   // its kept right singular vectors, kept on request
};

struct Oracle {
  // input
  int64_t n = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colind;
  std::vector<double> val;
  int dim = 0;
  std::vector<double> coords;
  int L = 0;                                  // depth of the H-tree
  // nested partitioning
  std::vector<int32_t> perm;                  // perm[k] = original index at position k
  std::vector<int32_t> leaf_off;              // 2^L + 1 offsets into perm
  std::vector<int32_t> leaf_of;               // leaf cluster of each original index
  std::vector<std::vector<std::set<int>>> adj;  // adj[i][j]: clusters adjacent to j in P_i
  // factorization state
  std::map<int, int> size;                    // node id -> number of variables
  std::map<std::pair<int, int>, Block> blk;   // (row node, col node) -> A_{row,col}
  std::map<int, std::set<int>> nbr;           // interaction edges among live nodes
  std::vector<ElimRecord> elim;
  std::vector<CompressRecord> comp;
  std::vector<std::vector<std::vector<int>>> batches;  // per level (L..1): batches of super ids
  std::map<int, int64_t> off;                 // offset of each red / black node in x_e
  int64_t ext_size = 0;                       // length of the extended vector x_e
  bool factored = false;
  bool capture_m = false;
  double eps = 0.0;
  int min_dist = 2;                           // well-separated: cluster distance >= this
  bool natural_order = false;                 // one super-node per batch, ascending index
  int trunc_rule = 0;                         // 0: eq. cutOff1, 1: eq. curOff6
  double below_sq = 0.0;                      // eq. curOff6: running sum of squared block norms
};

// ---------------------------------------------------------------------------
// Nested partitionings P_0..P_l (Sec. 3) by recursive coordinate bisection.
// ---------------------------------------------------------------------------

void bisect(const Oracle& o, std::vector<int32_t>& idx) {
  double lo[8], hi[8];
  for (int d = 0; d < o.dim; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
  for (int32_t v : idx)
    for (int d = 0; d < o.dim; ++d) {
      double x = o.coords[(size_t)v * o.dim + d];
      lo[d] = std::min(lo[d], x);
      hi[d] = std::max(hi[d], x);
    }
  int axis = 0;
  double ext = idx.empty() ? 0.0 : hi[0] - lo[0];
  for (int d = 1; d < o.dim; ++d)
    if (!idx.empty() && hi[d] - lo[d] > ext) { ext = hi[d] - lo[d]; axis = d; }
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
    double xa = o.coords[(size_t)a * o.dim + axis], xb = o.coords[(size_t)b * o.dim + axis];
    if (xa != xb) return xa < xb;
    return a < b;
  });
}

void build_partition(Oracle& o) {
  std::vector<std::vector<int32_t>> cur(1);
  cur[0].resize(o.n);
  std::iota(cur[0].begin(), cur[0].end(), 0);
  for (int lev = 0; lev < o.L; ++lev) {
    std::vector<std::vector<int32_t>> next(cur.size() * 2);
    for (size_t j = 0; j < cur.size(); ++j) {
      std::vector<int32_t> s = cur[j];
      bisect(o, s);
      size_t h = s.size() / 2;
      next[2 * j].assign(s.begin(), s.begin() + h);
      next[2 * j + 1].assign(s.begin() + h, s.end());
    }
    cur.swap(next);
  }
  o.perm.clear();
  o.leaf_off.assign(cur.size() + 1, 0);
  o.leaf_of.assign(o.n, 0);
  for (size_t j = 0; j < cur.size(); ++j) {
    o.leaf_off[j] = (int32_t)o.perm.size();
    for (int32_t v : cur[j]) { o.perm.push_back(v); o.leaf_of[v] = (int32_t)j; }
  }
  o.leaf_off[cur.size()] = (int32_t)o.perm.size();
}

// Adjacent clusters (Def. adj): leaf clusters are adjacent when a stored entry
// couples them in either direction; clusters of a coarser level are adjacent
// when some pair of their leaf descendants is.
void build_adjacency(Oracle& o) {
  o.adj.assign(o.L + 1, {});
  for (int i = 0; i <= o.L; ++i) o.adj[i].assign(1u << i, {});
  for (int64_t row = 0; row < o.n; ++row)
    for (int64_t e = o.rowptr[row]; e < o.rowptr[row + 1]; ++e) {
      int a = o.leaf_of[row], b = o.leaf_of[o.colind[e]];
      if (a == b) continue;
      for (int i = o.L; i >= 0; --i) {
        int ca = a >> (o.L - i), cb = b >> (o.L - i);
        if (ca == cb) break;
        o.adj[i][ca].insert(cb);
        o.adj[i][cb].insert(ca);
      }
    }
}

bool adjacent(const Oracle& o, int level, int ca, int cb) {
  return ca == cb || o.adj[level][ca].count(cb) > 0;
}

// Well-separated clusters (Def. wellSep with Def. distance): distance in the
// cluster graph of the level at least o.min_dist.  2 is the paper's rule (not
// adjacent); 3 is the stronger variant its conclusion (Sec. 7) suggests: not
// adjacent and no cluster adjacent to both.
bool well_separated(const Oracle& o, int level, int ca, int cb) {
  if (adjacent(o, level, ca, cb)) return false;
  if (o.min_dist <= 2) return true;
  for (int c : o.adj[level][ca])
    if (o.adj[level][cb].count(c)) return false;
  return true;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Algorithm 1 (factorization) and its sub-steps.
// ---------------------------------------------------------------------------

enum { OK = 0, ERR_INVALID = 1, ERR_SINGULAR = 3, ERR_NOT_CONVERGED = 4 };

Block& block_at(Oracle& o, int row, int col) {
  auto key = std::make_pair(row, col);
  auto it = o.blk.find(key);
  if (it == o.blk.end()) it = o.blk.emplace(key, Block(o.size[row], o.size[col])).first;
  return it->second;
}

void link(Oracle& o, int a, int b) {
  if (a == b) return;
  o.nbr[a].insert(b);
  o.nbr[b].insert(a);
}

// Initialize(l) (Sec. 4.1): leaf red-nodes carry the equations of A under P_l;
// an interaction edge joins adjacent leaf clusters.
void initialize(Oracle& o) {
  const int L = o.L;
  for (int j = 0; j < (1 << L); ++j) {
    int id = red_id(L, j);
    o.size[id] = o.leaf_off[j + 1] - o.leaf_off[j];
    o.nbr[id];
    o.off[id] = o.leaf_off[j];
  }
  o.ext_size = o.n;
  std::vector<int32_t> pos(o.n);
  for (int64_t k = 0; k < o.n; ++k) pos[o.perm[k]] = (int32_t)k;
  for (int j = 0; j < (1 << L); ++j) {
    block_at(o, red_id(L, j), red_id(L, j));
    for (int q : o.adj[L][j]) {
      block_at(o, red_id(L, j), red_id(L, q));
      link(o, red_id(L, j), red_id(L, q));
    }
  }
  for (int64_t row = 0; row < o.n; ++row)
    for (int64_t e = o.rowptr[row]; e < o.rowptr[row + 1]; ++e) {
      int64_t col = o.colind[e];
      int a = o.leaf_of[row], b = o.leaf_of[col];
      Block& B = block_at(o, red_id(L, a), red_id(L, b));
      B.at(pos[row] - o.leaf_off[a], pos[col] - o.leaf_off[b]) += o.val[e];
    }
}

// MergeRedNodes (Sec. 4.2): every sibling pair of red-nodes at level i becomes
// the super-node s_j^[i]; the block between two super-nodes is the 2 x 2
// concatenation of the blocks between their red-nodes, and Var/RHS are the
// concatenations (eqs. concatX, concatRHS).
void merge_level(Oracle& o, int i) {
  const int ns = 1 << (i - 1);
  for (int j = 0; j < ns; ++j) {
    int s = super_id(i, j);
    o.size[s] = o.size[red_id(i, 2 * j)] + o.size[red_id(i, 2 * j + 1)];
    o.off[s] = o.off[red_id(i, 2 * j)];
    o.nbr[s];
  }
  std::map<std::pair<int, int>, Block> merged;
  std::vector<std::pair<int, int>> dead;
  for (auto& kv : o.blk) {
    int ra = kv.first.first, rb = kv.first.second;
    if (kind_of(ra) != RED || kind_of(rb) != RED) continue;
    int ha = cluster_of(ra), hb = cluster_of(rb);
    if (level_of_heap(ha) != i || level_of_heap(hb) != i) continue;
    int ja = ha - (1 << i), jb = hb - (1 << i);
    int sa = super_id(i, ja / 2), sb = super_id(i, jb / 2);
    int roff = (ja & 1) ? o.size[red_id(i, ja - 1)] : 0;
    int coff = (jb & 1) ? o.size[red_id(i, jb - 1)] : 0;
    auto key = std::make_pair(sa, sb);
    auto it = merged.find(key);
    if (it == merged.end()) it = merged.emplace(key, Block(o.size[sa], o.size[sb])).first;
    const Block& src = kv.second;
    for (int c = 0; c < src.c; ++c)
      for (int r = 0; r < src.r; ++r) it->second.at(roff + r, coff + c) = src.at(r, c);
    dead.push_back(kv.first);
  }
  for (auto& k : dead) o.blk.erase(k);
  for (int j = 0; j < ns; ++j) {     // every super-node has its pivot block
    int s = super_id(i, j);
    if (!merged.count({s, s})) merged.emplace(std::make_pair(s, s), Block(o.size[s], o.size[s]));
  }
  for (auto& kv : merged) {
    o.blk.emplace(kv.first, std::move(kv.second));
    link(o, kv.first.first, kv.first.second);
  }
  for (int j = 0; j < (1 << i); ++j) o.nbr.erase(red_id(i, j));
}

// Compress(s) (Sec. 4.3): stack the blocks of the well-separated edges of s
// (eq. lra), truncate the SVD by eq. cutOff1, and replace those edges by the
// low-rank chain through b = black(i, j) and P(b) = red(i-1, j).
void compress(Oracle& o, int i, int j) {
  const int s = super_id(i, j);
  const int hs = cluster_of(s);
  const int lev = i - 1;                       // clusters of level-i nodes live in P_{i-1}
  CompressRecord rec;
  rec.snode = s;
  for (int p : o.nbr[s]) {
    int hp = cluster_of(p);
    if (well_separated(o, lev, hs - (1 << lev), hp - (1 << lev))) rec.ws.push_back(p);
  }
  const int m = o.size[s];
  int rho = 0;
  for (int p : rec.ws) rho += 2 * o.size[p];
  Block M(rho, m);
  int row = 0;
  for (int p : rec.ws) {                       // A_k = Mat(e_{s -> p_k}) = A_{p_k, s}
    const Block& A = o.blk.at({p, s});
    for (int c = 0; c < m; ++c)
      for (int r = 0; r < A.r; ++r) M.at(row + r, c) = A.at(r, c);
    row += A.r;
  }
  for (int p : rec.ws) {                       // B_k with B_k^T = Mat(e_{p_k -> s}) = A_{s, p_k}
    const Block& Bt = o.blk.at({s, p});
    for (int c = 0; c < m; ++c)
      for (int r = 0; r < Bt.c; ++r) M.at(row + r, c) = Bt.at(c, r);
    row += Bt.c;
  }
  std::vector<double> sigma;
  Block W;
  int r = 0;
  rec.below = std::sqrt(o.below_sq);
  if (rho > 0 && m > 0) {
    svd_right(M, sigma, W);
    if (o.trunc_rule == 0) {
      if (!sigma.empty() && sigma[0] > 0.0)    // eq. cutOff1: sigma_k / sigma_0 >= eps
        for (double sv : sigma)
          if (sv >= o.eps * sigma[0]) ++r;
    } else {
      // eq. curOff6: the smallest k with ||M - U_k S_k V_k^T||_F < eps ||all
      // levels below||_F, where ||M - U_k S_k V_k^T||_F^2 = sum_{j >= k} sigma_j^2
      const int nsv = (int)sigma.size();
      const double bound = o.eps * rec.below;
      r = nsv;
      for (int k = 0; k <= nsv; ++k) {
        double tail = 0.0;
        for (int j = nsv - 1; j >= k; --j) tail += sigma[j] * sigma[j];
        if (std::sqrt(tail) < bound) { r = k; break; }
      }
    }
  }
  Block V(m, r);
  for (int c = 0; c < r; ++c)
    for (int q = 0; q < m; ++q) V.at(q, c) = W.at(q, c);
  Block RQ = (rho > 0) ? gemm(M, V) : Block(0, r);   // [R_1..R_t; Q_1..Q_t]

  const int b = black_id(i, j), P = red_id(i - 1, j);
  o.size[b] = r;
  o.size[P] = r;
  o.nbr[b];
  o.nbr[P];
  // rows of RQ: A-part then B-part, in the order of rec.ws
  int arow = 0, brow = rho / 2;
  for (int p : rec.ws) {
    const int mp = o.size[p];
    Block R(mp, r), QT(r, mp);
    for (int c = 0; c < r; ++c)
      for (int q = 0; q < mp; ++q) {
        R.at(q, c) = RQ.at(arow + q, c);
        QT.at(c, q) = RQ.at(brow + q, c);
      }
    arow += mp;
    brow += mp;
    o.blk.erase({p, s});                       // remove the well-separated edges
    o.blk.erase({s, p});
    o.nbr[s].erase(p);
    o.nbr[p].erase(s);
    o.blk[{p, P}] = R;                         // P(b) -> p_k carries R_k
    o.blk[{P, p}] = QT;                        // p_k -> P(b) carries Q_k^T
    link(o, P, p);
  }
  Block VT = transpose(V), mI(r, r);
  for (int q = 0; q < r; ++q) mI.at(q, q) = -1.0;
  o.blk[{b, s}] = VT;                          // s -> b carries V^T
  o.blk[{s, b}] = V;                           // b -> s carries V
  o.blk[{b, P}] = mI;                          // b <-> P(b) carry -I
  o.blk[{P, b}] = mI;
  o.blk[{b, b}] = Block(r, r);
  o.blk[{P, P}] = Block(r, r);
  link(o, s, b);
  link(o, b, P);
  rec.rho = rho;
  rec.m = m;
  rec.r = r;
  rec.sigma = sigma;
  if (o.capture_m) { rec.M = std::move(M); rec.V = V; }
  o.comp.push_back(std::move(rec));
}

// Eliminate(p) (Sec. 2.2 and 4.4): block Gauss elimination of one node.  For
// every out-edge p -> q and in-edge k -> p, A_{q,k} -= A_{q,p} A_{p,p}^{-1} A_{p,k}
// (the edge is created when absent); then p leaves the graph and its edges
// are kept as the factor for the solve.
int eliminate(Oracle& o, int p) {
  ElimRecord rec;
  rec.node = p;
  rec.lu = o.blk.at({p, p});
  if (!lu_factor(rec.lu, rec.piv)) return ERR_SINGULAR;
  rec.nbr.assign(o.nbr[p].begin(), o.nbr[p].end());
  std::vector<Block> T;                        // A_{p,p}^{-1} A_{p,k}
  for (int k : rec.nbr) T.push_back(lu_solve_block(rec.lu, rec.piv, o.blk.at({p, k})));
  for (size_t a = 0; a < rec.nbr.size(); ++a) {
    const int q = rec.nbr[a];
    const Block& Aqp = o.blk.at({q, p});
    for (size_t c = 0; c < rec.nbr.size(); ++c) {
      const int k = rec.nbr[c];
      gemm_sub(Aqp, T[c], block_at(o, q, k));
      link(o, q, k);
    }
  }
  for (int q : rec.nbr) {
    rec.Lq.push_back(o.blk.at({q, p}));
    rec.Uq.push_back(o.blk.at({p, q}));
    o.blk.erase({q, p});
    o.blk.erase({p, q});
    o.nbr[q].erase(p);
  }
  o.blk.erase({p, p});
  o.nbr.erase(p);
  o.elim.push_back(std::move(rec));
  return OK;
}

// Algorithm 1: levels from leaf to root; at each level merge, then compress,
// eliminate the super-node and eliminate its black-node, batch by batch.
int factor(Oracle& o, double eps, int max_batches) {
  o.eps = eps;
  o.size.clear(); o.blk.clear(); o.nbr.clear(); o.elim.clear(); o.comp.clear();
  o.batches.clear(); o.off.clear();
  initialize(o);
  int batch_count = 0;
  o.below_sq = 0.0;
  for (int i = o.L; i >= 1; --i) {
    merge_level(o, i);
    // eq. curOff6: ||all levels below||_F^2 adds the squared Frobenius norms of
    // every block of this level (its system as the level starts, after merging)
    for (const auto& kv : o.blk)
      for (double v : kv.second.a) o.below_sq += v * v;
    std::vector<int> remaining((size_t)1 << (i - 1));
    std::iota(remaining.begin(), remaining.end(), 0);
    std::vector<std::vector<int>> level_batches;
    while (!remaining.empty()) {
      if (max_batches > 0 && batch_count >= max_batches) {   // partial run: sampled records only
        o.batches.push_back(level_batches);
        return OK;
      }
      ++batch_count;
      std::vector<int> batch, rest;
      for (int j : remaining) {
        int s = super_id(i, j);
        bool free = !(o.natural_order && !batch.empty());
        for (int t : batch)
          if (o.nbr[s].count(super_id(i, t))) { free = false; break; }
        (free ? batch : rest).push_back(j);
      }
      for (int j : batch) {
        compress(o, i, j);
        int st = eliminate(o, super_id(i, j));
        if (st != OK) return st;
        st = eliminate(o, black_id(i, j));
        if (st != OK) return st;
      }
      std::vector<int> ids;
      for (int j : batch) ids.push_back(super_id(i, j));
      level_batches.push_back(ids);
      remaining.swap(rest);
    }
    o.batches.push_back(level_batches);
    // place the new black and red nodes in the extended vector; siblings of
    // level i-1 are adjacent so that a super-node is one contiguous range
    for (int j = 0; j < (1 << (i - 1)); ++j) {
      o.off[black_id(i, j)] = o.ext_size;
      o.ext_size += o.size[black_id(i, j)];
    }
    for (int j = 0; j < (1 << (i - 1)); ++j) {
      o.off[red_id(i - 1, j)] = o.ext_size;
      o.ext_size += o.size[red_id(i - 1, j)];
    }
  }
  o.factored = true;
  return OK;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Algorithms 2-4 (solve) and GMRES.
// ---------------------------------------------------------------------------

// Algorithm 2: SetRHS, forward traversal in elimination order with SolveL
// (Alg. 3), backward traversal in reverse order with SolveU (Alg. 4).  A
// super-node's Var/RHS is the contiguous range of its two red-nodes in x_e,
// so concatenation (eq. concatRHS) and SplitVar are implicit.
void apply_one(const Oracle& o, const double* b, double* x) {
  std::vector<double> xe(o.ext_size, 0.0);
  for (int64_t k = 0; k < o.n; ++k) xe[k] = b[o.perm[k]];     // SetRHS
  for (const ElimRecord& rec : o.elim) {                      // SolveL
    const int64_t op = o.off.at(rec.node);
    const int mp = rec.lu.r;
    std::vector<double> f(xe.begin() + op, xe.begin() + op + mp);
    lu_solve(rec.lu, rec.piv, f.data(), mp, 1, mp);
    for (size_t a = 0; a < rec.nbr.size(); ++a) {
      const Block& Aqp = rec.Lq[a];
      double* yq = xe.data() + o.off.at(rec.nbr[a]);
      for (int c = 0; c < Aqp.c; ++c)
        for (int r = 0; r < Aqp.r; ++r) yq[r] -= Aqp.at(r, c) * f[c];
    }
  }
  for (auto it = o.elim.rbegin(); it != o.elim.rend(); ++it) { // SolveU
    const ElimRecord& rec = *it;
    const int64_t op = o.off.at(rec.node);
    const int mp = rec.lu.r;
    std::vector<double> v(xe.begin() + op, xe.begin() + op + mp);
    for (size_t a = 0; a < rec.nbr.size(); ++a) {
      const Block& Apq = rec.Uq[a];
      const double* xq = xe.data() + o.off.at(rec.nbr[a]);
      for (int c = 0; c < Apq.c; ++c)
        for (int r = 0; r < Apq.r; ++r) v[r] -= Apq.at(r, c) * xq[c];
    }
    lu_solve(rec.lu, rec.piv, v.data(), mp, 1, mp);
    std::copy(v.begin(), v.end(), xe.begin() + op);
  }
  for (int64_t k = 0; k < o.n; ++k) x[o.perm[k]] = xe[k];
}

void spmv(const Oracle& o, const double* x, double* y) {
  for (int64_t row = 0; row < o.n; ++row) {
    double s = 0.0;
    for (int64_t e = o.rowptr[row]; e < o.rowptr[row + 1]; ++e) s += o.val[e] * x[o.colind[e]];
    y[row] = s;
  }
}

double norm2(const std::vector<double>& v) {
  double s = 0.0;
  for (double x : v) s += x * x;
  return std::sqrt(s);
}

// Restarted GMRES(restart), x0 = 0, modified Gram-Schmidt Arnoldi and Givens
// rotations.  precond 0: none; 1: right preconditioning by the factorization
// (A M y = b, x = M y; the stopping residual is the true one of eq. accres);
// 2: left preconditioning, the paper's form (M A x = M b; it stops on the
// preconditioned residual ||M (b - A x)|| / ||M b|| of eq. GMRES_residual).
// Returns the Arnoldi steps taken, the final true relative residual and
// (precond 2) the final preconditioned one.
int gmres_one(const Oracle& o, const double* b, double* x, int restart, int maxit, double tol,
              int precond, int* iters_out, double* relres_out, double* prec_out = nullptr) {
  if (precond == 2) {
    const int64_t n = o.n;
    std::vector<double> bb(b, b + n), mb(n), xv(n, 0.0), r(n), w(n), z(n);
    apply_one(o, bb.data(), mb.data());
    const double bnorm = norm2(bb), mbnorm = norm2(mb);
    int iters = 0;
    double prec = 0.0;
    if (mbnorm > 0.0) {
      r = mb;                                  // M (b - A x0), x0 = 0
      double beta = mbnorm;
      prec = 1.0;
      while (iters < maxit) {
        std::vector<std::vector<double>> V(1, std::vector<double>(n));
        for (int64_t k = 0; k < n; ++k) V[0][k] = r[k] / beta;
        std::vector<std::vector<double>> H;
        std::vector<double> cs, sn, g(1, beta);
        int k = 0;
        for (; k < restart && iters < maxit; ++k) {
          spmv(o, V[k].data(), z.data());     // w = M (A v)
          apply_one(o, z.data(), w.data());
          std::vector<double> h(k + 2, 0.0);
          for (int j = 0; j <= k; ++j) {
            double d = 0.0;
            for (int64_t t = 0; t < n; ++t) d += w[t] * V[j][t];
            h[j] = d;
            for (int64_t t = 0; t < n; ++t) w[t] -= d * V[j][t];
          }
          h[k + 1] = norm2(w);
          V.emplace_back(n, 0.0);
          if (h[k + 1] != 0.0)
            for (int64_t t = 0; t < n; ++t) V[k + 1][t] = w[t] / h[k + 1];
          for (int j = 0; j < k; ++j) {
            double t0 = cs[j] * h[j] + sn[j] * h[j + 1];
            h[j + 1] = -sn[j] * h[j] + cs[j] * h[j + 1];
            h[j] = t0;
          }
          double den = std::hypot(h[k], h[k + 1]);
          double c = den == 0.0 ? 1.0 : h[k] / den, s = den == 0.0 ? 0.0 : h[k + 1] / den;
          cs.push_back(c);
          sn.push_back(s);
          h[k] = c * h[k] + s * h[k + 1];
          h[k + 1] = 0.0;
          g.push_back(-s * g[k]);
          g[k] = c * g[k];
          H.push_back(h);
          ++iters;
          if (std::fabs(g[k + 1]) / mbnorm <= tol || den == 0.0) { ++k; break; }
        }
        std::vector<double> y(k, 0.0);        // x += V y, y = H \ g
        for (int i = k - 1; i >= 0; --i) {
          double s = g[i];
          for (int j = i + 1; j < k; ++j) s -= H[j][i] * y[j];
          y[i] = H[i][i] != 0.0 ? s / H[i][i] : 0.0;
        }
        for (int j = 0; j < k; ++j)
          for (int64_t t = 0; t < n; ++t) xv[t] += y[j] * V[j][t];
        spmv(o, xv.data(), w.data());
        for (int64_t t = 0; t < n; ++t) z[t] = bb[t] - w[t];
        apply_one(o, z.data(), r.data());
        beta = norm2(r);
        prec = beta / mbnorm;
        if (prec <= tol || beta == 0.0) break;
      }
    }
    spmv(o, xv.data(), w.data());
    double rr = 0.0;
    for (int64_t t = 0; t < n; ++t) rr += (bb[t] - w[t]) * (bb[t] - w[t]);
    std::copy(xv.begin(), xv.end(), x);
    *iters_out = iters;
    *relres_out = bnorm > 0.0 ? std::sqrt(rr) / bnorm : 0.0;
    if (prec_out) *prec_out = prec;
    return prec <= tol ? OK : ERR_NOT_CONVERGED;
  }
  const int64_t n = o.n;
  std::vector<double> bb(b, b + n), xv(n, 0.0), r(n), w(n), z(n);
  const double bnorm = norm2(bb);
  int iters = 0;
  if (bnorm == 0.0) {
    std::fill(x, x + n, 0.0);
    *iters_out = 0;
    *relres_out = 0.0;
    return OK;
  }
  auto precond_apply = [&](const std::vector<double>& in, std::vector<double>& out) {
    if (precond) apply_one(o, in.data(), out.data());
    else out = in;
  };
  r = bb;                                   // x0 = 0
  double beta = bnorm;
  double relres = 1.0;
  bool converged = false;
  while (!converged && iters < maxit) {
    std::vector<std::vector<double>> V(1, std::vector<double>(n));
    for (int64_t k = 0; k < n; ++k) V[0][k] = r[k] / beta;
    std::vector<std::vector<double>> H;     // H[j] = column j, length j+2
    std::vector<double> cs, sn, g(1, beta);
    int k = 0;
    bool inner_done = false;
    for (; k < restart && iters < maxit; ++k) {
      precond_apply(V[k], z);
      spmv(o, z.data(), w.data());
      std::vector<double> h(k + 2, 0.0);
      for (int j = 0; j <= k; ++j) {        // modified Gram-Schmidt
        double d = 0.0;
        for (int64_t t = 0; t < n; ++t) d += w[t] * V[j][t];
        h[j] = d;
        for (int64_t t = 0; t < n; ++t) w[t] -= d * V[j][t];
      }
      h[k + 1] = norm2(w);
      V.emplace_back(n, 0.0);
      if (h[k + 1] != 0.0)
        for (int64_t t = 0; t < n; ++t) V[k + 1][t] = w[t] / h[k + 1];
      for (int j = 0; j < k; ++j) {         // previous Givens rotations
        double t0 = cs[j] * h[j] + sn[j] * h[j + 1];
        h[j + 1] = -sn[j] * h[j] + cs[j] * h[j + 1];
        h[j] = t0;
      }
      double den = std::hypot(h[k], h[k + 1]);
      double c = den == 0.0 ? 1.0 : h[k] / den, s = den == 0.0 ? 0.0 : h[k + 1] / den;
      cs.push_back(c);
      sn.push_back(s);
      h[k] = c * h[k] + s * h[k + 1];
      h[k + 1] = 0.0;
      g.push_back(-s * g[k]);
      g[k] = c * g[k];
      H.push_back(h);
      ++iters;
      relres = std::fabs(g[k + 1]) / bnorm;
      if (relres <= tol || den == 0.0) { ++k; inner_done = true; break; }
    }
    (void)inner_done;
    // y = H(1:k,1:k) \ g(1:k), then x += M (V y)
    std::vector<double> y(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int j = i + 1; j < k; ++j) s -= H[j][i] * y[j];
      y[i] = H[i][i] != 0.0 ? s / H[i][i] : 0.0;
    }
    std::vector<double> u(n, 0.0);
    for (int j = 0; j < k; ++j)
      for (int64_t t = 0; t < n; ++t) u[t] += y[j] * V[j][t];
    precond_apply(u, z);
    for (int64_t t = 0; t < n; ++t) xv[t] += z[t];
    spmv(o, xv.data(), w.data());
    for (int64_t t = 0; t < n; ++t) r[t] = bb[t] - w[t];
    beta = norm2(r);
    relres = beta / bnorm;
    if (relres <= tol) converged = true;
    if (beta == 0.0) break;
  }
  std::copy(xv.begin(), xv.end(), x);
  *iters_out = iters;
  *relres_out = relres;
  return converged ? OK : ERR_NOT_CONVERGED;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI (host pointers; column-major n x nrhs for multi-vector arguments).
// ---------------------------------------------------------------------------

extern "C" {

int lrso_create(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                int dim, const double* coords, int leaf_size, int depth, void** out) {
  if (!out || n <= 0 || !rowptr || !colind || !val || !coords || dim < 1 || dim > 8) return ERR_INVALID;
  Oracle* o = new Oracle();
  o->n = n;
  o->rowptr.assign(rowptr, rowptr + n + 1);
  o->colind.assign(colind, colind + rowptr[n]);
  o->val.assign(val, val + rowptr[n]);
  o->dim = dim;
  o->coords.assign(coords, coords + n * dim);
  if (depth <= 0) {
    if (leaf_size <= 0) { delete o; return ERR_INVALID; }
    int l = 0;
    while ((int64_t)leaf_size << l < n) ++l;   // l = ceil(log2(n / leaf))
    depth = std::max(l, 1);
  }
  if (depth > 24) { delete o; return ERR_INVALID; }
  o->L = depth;
  build_partition(*o);
  build_adjacency(*o);
  *out = o;
  return OK;
}

void lrso_destroy(void* h) { delete static_cast<Oracle*>(h); }

int lrso_depth(void* h) { return static_cast<Oracle*>(h)->L; }

// Minimum cluster distance of a well-separated pair: 2 (the paper's
// Def. wellSep, default) or 3 (the variant of Sec. 7); applies to the next
// factorization.
int lrso_set_separation(void* h, int min_dist) {
  if (min_dist != 2 && min_dist != 3) return ERR_INVALID;
  static_cast<Oracle*>(h)->min_dist = min_dist;
  return OK;
}

int lrso_set_values(void* h, const double* val) {
  Oracle* o = static_cast<Oracle*>(h);
  o->val.assign(val, val + o->rowptr[o->n]);
  o->factored = false;
  return OK;
}

int lrso_factor(void* h, double eps, int capture_m) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!(eps >= 0.0)) return ERR_INVALID;
  o->capture_m = capture_m != 0;
  return factor(*o, eps, 0);
}

// The first max_batches batches of Algorithm 1 only (records of a sample of
// a large problem); the factorization is left incomplete.
int lrso_factor_partial(void* h, double eps, int max_batches) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!(eps >= 0.0) || max_batches < 1) return ERR_INVALID;
  o->capture_m = false;
  const int st = factor(*o, eps, max_batches);
  o->factored = false;
  return st;
}

int64_t lrso_ext_size(void* h) { return static_cast<Oracle*>(h)->ext_size; }

int lrso_apply(void* h, const double* b, double* x, int nrhs) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->factored) return ERR_INVALID;
  for (int c = 0; c < nrhs; ++c) apply_one(*o, b + (size_t)c * o->n, x + (size_t)c * o->n);
  return OK;
}

// GMRES with the paper's left preconditioning (precond 2 of gmres_one): per
// column its iterations, true relative residual and preconditioned residual.
int lrso_gmres_left(void* h, const double* b, double* x, int nrhs, int restart, int maxit, double tol,
                    int* iters, double* relres, double* prec) {
  Oracle* o = static_cast<Oracle*>(h);
  if (!o->factored || restart < 1 || maxit < 1) return ERR_INVALID;
  int status = OK;
  for (int c = 0; c < nrhs; ++c) {
    int st = gmres_one(*o, b + (size_t)c * o->n, x + (size_t)c * o->n, restart, maxit, tol, 2, iters + c,
                       relres + c, prec + c);
    if (st != OK) status = st;
  }
  return status;
}

// In-level order: 0 the greedy batches (default), 1 natural -- one super-node
// at a time by ascending index (Alg. 1 as printed); applies to the next
// factorization.
int lrso_set_order(void* h, int natural) {
  static_cast<Oracle*>(h)->natural_order = natural != 0;
  return OK;
}

int lrso_spmv(void* h, const double* x, double* y, int nrhs) {
  Oracle* o = static_cast<Oracle*>(h);
  for (int c = 0; c < nrhs; ++c) spmv(*o, x + (size_t)c * o->n, y + (size_t)c * o->n);
  return OK;
}

int lrso_gmres(void* h, const double* b, double* x, int nrhs, int restart, int maxit, double tol,
               int precond, int* iters, double* relres) {
  Oracle* o = static_cast<Oracle*>(h);
  if (precond && !o->factored) return ERR_INVALID;
  if (restart < 1 || maxit < 1) return ERR_INVALID;
  int status = OK;
  for (int c = 0; c < nrhs; ++c) {
    int st = gmres_one(*o, b + (size_t)c * o->n, x + (size_t)c * o->n, restart, maxit, tol,
                       precond, iters + c, relres + c);
    if (st != OK) status = st;
  }
  return status;
}

// Symbolic and per-step records, flattened to int32 arrays:
//  0 perm (n)            1 leaf offsets (2^l + 1)
//  2 batches: per level l..1: [level, nbatch, (count, super ids...)...]
//  3 compressions in order: [super id, t, well-separated ids...]
//  4 eliminations in order: [node id, degree, neighbour ids...]
//  5 ranks in compression order          6 pivot sizes in elimination order
static void export_all(const Oracle& o, int what, std::vector<int32_t>& v) {
  v.clear();
  switch (what) {
    case 0: v.assign(o.perm.begin(), o.perm.end()); break;
    case 1: v.assign(o.leaf_off.begin(), o.leaf_off.end()); break;
    case 2:
      for (size_t li = 0; li < o.batches.size(); ++li) {
        v.push_back(o.L - (int)li);
        v.push_back((int32_t)o.batches[li].size());
        for (auto& b : o.batches[li]) {
          v.push_back((int32_t)b.size());
          for (int s : b) v.push_back(s);
        }
      }
      break;
    case 3:
      for (auto& c : o.comp) {
        v.push_back(c.snode);
        v.push_back((int32_t)c.ws.size());
        for (int p : c.ws) v.push_back(p);
      }
      break;
    case 4:
      for (auto& e : o.elim) {
        v.push_back(e.node);
        v.push_back((int32_t)e.nbr.size());
        for (int q : e.nbr) v.push_back(q);
      }
      break;
    case 5: for (auto& c : o.comp) v.push_back(c.r); break;
    case 6: for (auto& e : o.elim) v.push_back(e.lu.r); break;
    default: break;
  }
}

int64_t lrso_export_size(void* h, int what) {
  std::vector<int32_t> v;
  export_all(*static_cast<Oracle*>(h), what, v);
  return (int64_t)v.size();
}

int lrso_export(void* h, int what, int32_t* out) {
  std::vector<int32_t> v;
  export_all(*static_cast<Oracle*>(h), what, v);
  std::copy(v.begin(), v.end(), out);
  return OK;
}

int lrso_compress_count(void* h) { return (int)static_cast<Oracle*>(h)->comp.size(); }

// eq. curOff6's ||all levels below||_F at compression k (recorded for either rule).
double lrso_compress_below(void* h, int k) { return static_cast<Oracle*>(h)->comp.at(k).below; }

// Truncation rule of the next factorization: 0 eq. cutOff1 (default), 1 eq. curOff6.
int lrso_set_trunc_rule(void* h, int rule) {
  if (rule != 0 && rule != 1) return ERR_INVALID;
  static_cast<Oracle*>(h)->trunc_rule = rule;
  return OK;
}

int lrso_compress_info(void* h, int k, int32_t* info4) {
  const CompressRecord& c = static_cast<Oracle*>(h)->comp.at(k);
  info4[0] = c.snode; info4[1] = c.rho; info4[2] = c.m; info4[3] = c.r;
  return OK;
}

int lrso_compress_sigma(void* h, int k, double* out) {
  const CompressRecord& c = static_cast<Oracle*>(h)->comp.at(k);
  std::copy(c.sigma.begin(), c.sigma.end(), out);
  return (int)c.sigma.size();
}

int lrso_compress_matrix(void* h, int k, double* out) {
  const CompressRecord& c = static_cast<Oracle*>(h)->comp.at(k);
  if (c.M.r != c.rho || c.M.c != c.m) return ERR_INVALID;
  std::copy(c.M.a.begin(), c.M.a.end(), out);
  return OK;
}

int lrso_compress_v(void* h, int k, double* out) {
  const CompressRecord& c = static_cast<Oracle*>(h)->comp.at(k);
  if (c.V.r != c.m || c.V.c != c.r) return ERR_INVALID;
  std::copy(c.V.a.begin(), c.V.a.end(), out);
  return OK;
}

}  // extern "C"
