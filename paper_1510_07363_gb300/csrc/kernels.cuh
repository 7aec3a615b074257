// kernels.cuh -- device task descriptors and launchers of liblrs.  Every
// kernel works on column-major FP64 blocks described by plain pointers and
// leading dimensions; the host builds arrays of descriptors (one per output
// tile, matrix or copy) and launches one grid over them.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

namespace lrs {

constexpr int kTile = 64;        // output tile edge of the gather GEMM
constexpr int kTileK = 16;       // contraction chunk staged in shared memory
constexpr int kTrvChunks = 4;    // traversal kernels: chunks whose loads are in flight together

// One contribution to a gather-GEMM output block: op(A) (rows x k) times
// op(B) (k x cols).  op(X) = X, or X^T when the matching trans bit is set.
// V: the element type (double; float for the precision form's traversal).
template <class V>
struct GemmTermT {
  const V* A;
  const V* B;
  int lda, ldb, k;
  int trans;                     // bit 0: transpose A, bit 1: transpose B
};

// One output tile (ti, tj) of the block C (rows x cols), 64 x 64 for the
// FP64 gather GEMM (64 x 16 for the narrow traversal kernels):
//   C = init + sign * sum_terms op(A) op(B)
// init = D (when D != nullptr), else C (mode & kAccumulate), else 0.
template <class V>
struct GemmTaskT {
  V* C;
  const V* D;
  int ldc, ldd;
  int rows, cols;
  int ti, tj;
  int term0, nterm;
  int mode;
};
using GemmTerm = GemmTermT<double>;
using GemmTask = GemmTaskT<double>;
using GemmTerm32 = GemmTermT<float>;
using GemmTask32 = GemmTaskT<float>;
enum : int { kAccumulate = 1, kSubtract = 2 };

// In-place inverse of an m x m block by Gauss-Jordan with partial pivoting.
// W: m x m workspace (used by the cluster form for the final column order).
struct InvTask {
  double* A;
  double* W;
  int m, lda;
  int cta0 = 0, cw = 0;          // resident form: first CTA of the block's team, columns per CTA
};

// Symmetric eigen-decomposition of the Gram matrix G (m x m, overwritten; only
// its lower triangle is read -- the upper one is filled by symmetry) by
// Householder tridiagonalisation, bisection and inverse iteration.  Writes
// the singular values sigma_k = sqrt(lambda_k) largest first (m of them; the
// first min(rho, m) are M's), the first `rank` eigenvectors into V (m x m,
// leading dimension m) and the rank by the rule
// sigma_k >= eps * sigma_0 (eq. cutOff1), applied as printed (no absolute
// floor; a zero spectrum has rank 0), or by eq. curOff6 (trunc_rule below).
struct EigTask {
  double* G;
  double* W;                     // workspace of eig_workspace(m, team warps) doubles
  double* V;                     // m x m output (first rank columns used)
  double* sigma;                 // m outputs
  int* rank;                     // one int
  int m, rho;
  double eps;
  // G's eigenvalues times gram_scale are sigma^2 (2 when G holds one of two
  // equal halves of M^T M, the symmetric case)
  double gram_scale = 1.0;
  // Householder slots of a reduction already done by the resident kernel
  // (nullptr: the spectrum kernel reduces G itself).  Slot k (m + 4 doubles):
  // reflector k in rows k+1..m-1, then d_k, e_k, beta_k.
  double* H = nullptr;
  int cta0 = 0, cw = 0;          // resident reduction: first CTA of the block's team, columns per CTA
  // sub-team launch (TeamKind::Sub): the block's CTAs [team0, team0 + team_size)
  // and its barrier words (arrival count, generation, abort; zeroed before the launch)
  int team0 = 0, team_size = 0;
  unsigned long long* bar = nullptr;
  // truncation rule: 0 eq. cutOff1 (sigma_k >= eps sigma_0); 1 eq. curOff6 (the
  // smallest k with sum_{j >= k} sigma_j^2 < (eps ||all levels below||_F)^2,
  // *below_sq holding ||all levels below||_F^2)
  int trunc_rule = 0;
  const double* below_sq = nullptr;
};

// Rectangular copy: dst(i, j) = src(i, j) (mode 0), src(j, i) (mode 1),
// alpha * delta_ij (mode 2); mode 3: dst(i, j) = dst(j, i) for i < j (a square
// block's lower triangle mirrored onto its upper one in place; src = dst);
// mode 4: alpha * delta_{i, j + lds} (a column piece of alpha * I starting at
// column lds).
struct CopyTask {
  const double* src;
  double* dst;
  int lds, ldd, rows, cols;
  int mode;
  double alpha;
};

// Dense kernels on one block run on a "team": one CTA (small blocks, shared
// memory), a thread-block cluster of kDenseCluster CTAs, the whole grid of a
// cooperative launch, or a sub-team of CTAs of a cooperative launch that
// serves several blocks (see dense.cu; the resident forms are declared below).
enum class TeamKind { Cta, Cluster, Grid, Sub };
constexpr int kDenseCluster = 8;
constexpr int kMaxTeam = 256;          // CTAs a grid team may have (norm-partial slots)
constexpr int kInvClusterMin = 129;    // invert blocks with m >= this on a team of CTAs
// Largest blocks the dense kernels take: a spectrum keeps 8 vectors of m
// doubles in shared memory (64 m + 64 bytes), an inverse 2 doubles and 2 ints
// per row (24 m + 64 bytes), within the 227 KB a CTA may have.
constexpr int kEigMaxM = (227 * 1024 - 64) / 64;   // 3631
constexpr int kInvMaxM = (227 * 1024 - 64) / 24;   // 9682
constexpr int kEigClusterMin = 161;    // spectra with m >= this on a team of CTAs
constexpr int kFewSpectra = 76;        // a batch with fewer spectra puts every one on a team
constexpr int kGridTeamMaxTasks = 4;   // at most this many large blocks: one grid launch each
// Spectrum workspace for a team with `warps` warps: p, the Gram-Schmidt
// coefficients of one block of kGsBlock vectors and its Gram matrix, and 6m
// doubles of inverse-iteration scratch per thread that may hold an
// eigenvector (the first min(m, threads) of the team's threads).
constexpr int kGsBlock = 16;
inline size_t eig_workspace(int m, int warps) {
  const size_t th = (size_t)warps * 32;
  const size_t w = th < (size_t)m ? th : (size_t)m;
  return (size_t)m + (size_t)kGsBlock * (m + kGsBlock) + (size_t)6 * m * (w > 0 ? w : 1) + 64;
}

struct DeviceStatus {            // written by kernels, read by the host
  int singular;                  // a pivot block had an exactly zero pivot
  int numeric;                   // NaN or Inf met
  int eig_unconverged;           // Jacobi reached its sweep limit
  int wait_timeout;              // a bounded wait between CTAs of a team expired
  int asymmetric;                // some a_ij != a_ji (the symmetry test)
  int pad;
  unsigned long long amax_bits;  // bit pattern of max |a_ij| (>= 0, so ordered as integers)
  unsigned long long eig_flops;  // algorithmic flops of the spectra
  // SM cycles spent in the spectrum phases (summed over CTAs): tridiagonal
  // reduction, bisection, inverse iteration, Gram-Schmidt, back-transformation
  unsigned long long eig_cycles[5];
  // wall time (ns) of the same phases on the first CTA of each multi-CTA block, summed
  unsigned long long eig_lead_ns[5];
  double below_sq;               // eq. curOff6: sum of squared norms of every level's blocks so far
};

void launch_gemm(const GemmTask* tasks, int ntask, const GemmTerm* terms, cudaStream_t st);
// The precision form's products on the tensor cores (tc_gemm.cu): tasks are
// kTcTile x kTcTile output tiles (ti, tj in those units); operands are split
// into TF32 head + FP32 tail and multiplied as three TF32 products with FP32
// accumulation in tensor memory, the sum added to the FP64 init in FP64.  A
// bounded wait that expires sets status->wait_timeout.
constexpr int kTcTile = 128;
size_t gemm_tc_smem_bytes();
cudaError_t launch_gemm_tc(const GemmTask* tasks, int ntask, const GemmTerm* terms, DeviceStatus* status,
                           cudaStream_t st);
// The FP64 form's products with FP64 emulated on the tensor cores
// (emu_gemm.cu): tasks are kEmuTileM x kEmuTileN output tiles (ti, tj in those
// units).  Every distinct operand of a launch is first split once (one
// exponent per row of op(A) / column of op(B) per group of kEmuGroup K chunks
// of kEmuChunk, eight 7-bit digit slices stored as BF16 in the layout the
// tensor core reads); the product kernel then copies digit slices into shared
// memory with bulk copies, sums the digit products exactly on the tensor cores
// and recombines them in 64-bit integers; accuracy at or below an FP64
// product's rounding.  A task may hold at most kEmuMaxChunks chunks (its
// integer sums stay in range).  A bounded wait that expires sets
// status->wait_timeout.
constexpr int kEmuTileM = 128, kEmuTileN = 64, kEmuChunk = 64, kEmuGroup = 8, kEmuMaxChunks = 512;
constexpr int kEmuSplitRows = 8;      // rows of an operand one split CTA takes (with all 512 k of a group)
constexpr double kEmuMinWork = 64.0 * 64.0 * 64.0;   // multiply-adds below which FP64 FMAs are used
int gemm_emu_chunks(const GemmTerm* terms, int nterm);
// One distinct operand, split once: op(X)(r, k) = kcontig ? P[k + r ld] :
// P[r + k ld], rows x k, rows padded to rows_pad (a multiple of tile).
// Outputs: dig (digit slices), ex (exponent per (group, row), [g rows_pad + r]),
// bad (1 where a row holds a non-finite entry; zeroed before the split).
struct EmuSplitTask {
  const double* P;
  int ld, kcontig, rows, k, tile, rows_pad, cta0;
  uint8_t* dig;
  int* ex;
  int* bad;
};
// The split operands of one term of the launch (parallel to its terms).
struct EmuTerm {
  const uint8_t* a_dig;
  const int* a_ex;
  const int* a_bad;
  const uint8_t* b_dig;
  const int* b_ex;
  const int* b_bad;
  int a_tiles, a_rows_pad, b_tiles, b_rows_pad, k;
};
// Host plan of one launch: the distinct operands and, per term, where their
// splits live, as byte offsets into one workspace of `bytes` bytes until
// bind(workspace) turns them into device pointers.  The bad flags occupy
// [bad_off, bad_off + bad_bytes) of the workspace and must be zeroed first.
struct EmuPlan {
  std::vector<EmuSplitTask> split;
  std::vector<EmuTerm> eterms;
  size_t bytes = 0, bad_off = 0, bad_bytes = 0;
  int split_ctas = 0;
  void bind(uint8_t* base);
};
EmuPlan plan_gemm_emu(const GemmTask* tasks, int ntask, const GemmTerm* terms, int nterms);
// The split launch then the product launch (d_split, d_eterms: device copies
// of the bound plan's arrays; the bad flags already zeroed).
cudaError_t launch_gemm_emu(const EmuPlan& plan, const EmuSplitTask* d_split, const GemmTask* d_tasks, int ntask,
                            const EmuTerm* d_eterms, DeviceStatus* status, cudaStream_t st);
// The same for blocks of at most 16 columns (solves with <= 16 right-hand
// sides): 64 x 16 tiles, every thread owning four outputs.  split > 1 splits
// each task's contraction over `split` CTAs (partials in `part`, split * ntask
// * 1024 doubles, added in a fixed order by a second launch).
// pdl: programmatic dependent launch (the traversal graph): the kernel may start
// while the previous launch of the stream drains, and waits for it in its prologue.
void launch_gemm_narrow(const GemmTask* tasks, int ntask, const GemmTerm* terms, cudaStream_t st, int split = 1,
                        double* part = nullptr, bool pdl = false);
constexpr int kSplitTarget = 4 * 152;   // CTAs a split narrow launch aims for
// The same traversal kernels in FP32 (the precision form's factor is stored in
// FP32 and its traversal runs in FP32 arithmetic): tiles of 64 rows x 16
// columns at column 16 tj, any number of right-hand sides; part holds
// split * ntask * 1024 floats (narrow) or split * ntask * 64 (one column).
void launch_gemm_narrow32(const GemmTask32* tasks, int ntask, const GemmTerm32* terms, cudaStream_t st,
                          int split = 1, float* part = nullptr, bool pdl = false);
void launch_gemv32(const GemmTask32* tasks, int ntask, const GemmTerm32* terms, cudaStream_t st, int split = 1,
                   float* part = nullptr, bool pdl = false);
// dst[i] = (float) src[i] for the blocks of a factor moved to FP32 storage
struct ConvTask {
  const double* src;
  float* dst;
  int64_t count;
};
void launch_to_f32(const ConvTask* tasks, int ntask, cudaStream_t st);
// One right-hand side (cols == 1, operands not transposed): a matrix-vector
// product per 64-row tile, bound by HBM; split as launch_gemm_narrow (part:
// split * ntask * 64 doubles).
void launch_gemv(const GemmTask* tasks, int ntask, const GemmTerm* terms, cudaStream_t st, int split = 1,
                 double* part = nullptr, bool pdl = false);
// kind Cta / Cluster: one team per task; kind Grid: ntask == 1, `team` CTAs.
cudaError_t launch_invert(const InvTask* tasks, int ntask, int max_m, TeamKind kind, int team,
                          DeviceStatus* status, cudaStream_t st);
// Cta keeps G in shared memory (every m < kEigClusterMin); Cluster and Grid
// work on G in global memory (Grid: ntask == 1 on `team` CTAs); Sub: every
// task on its own sub-team (team0, team_size set, tasks ordered by team0,
// `team` = total CTAs), reduced already (H set).  Grid and Sub are
// cooperative launches: main stream only.
cudaError_t launch_eig(const EigTask* tasks, int ntask, int max_m, TeamKind kind, int team, DeviceStatus* status,
                       cudaStream_t st);
// CTAs a grid team may use for one block of size m (<= what is co-resident).
int grid_team_size(int m, bool eig);
// Sub-team launches of spectra: CTAs one launch may hold (blocks up to max_m),
// and the plan -- waves [begin, end) of at most `capacity` blocks, each block
// given CTAs in proportion to m^3 (at least one, at most kMaxTeam).
int sub_team_capacity(int max_m);
std::vector<std::pair<int, int>> plan_sub_teams(const int* m, int n, int capacity, int* team0, int* size);
// Resident forms of the pivot inverse and of the Householder reduction of a
// spectrum: each block is worked on by a team of CTAs that keep their share
// of its columns (cw each) in shared memory for the whole run, one CTA per SM,
// exchanging only one column (inverse) or a reflector and a p vector
// (reduction) per step through the block's workspace.  Blocks are launched in
// waves (cooperative launches of at most one CTA per SM); a wave gives each of
// its blocks a team in proportion to its work.
//   plan_resident_waves: fills cta0 and cw of tasks [0, n) of sizes m[i]
//     (kept in order) and returns the waves as index ranges [begin, end);
//     empty when some block does not fit.  sms: SMs to plan for (0: this GPU's).
//   launch_invert_resident: one wave; W of each task inv_resident_workspace(m).
//   launch_tridiag_resident: one wave; H of each task tridiag_resident_workspace(m);
//     afterwards launch_eig (kind Grid or Cluster) with H set finishes the spectra.
// h_tasks: the host copy of the wave's d_tasks.  Main stream only.
constexpr size_t kResidentSmemMax = 220 * 1024;
std::vector<std::pair<int, int>> plan_resident_waves(const int* m, int n, bool eig, int* cta0, int* cw, int sms = 0);
// The same over blocks of both kinds (eigs[i] != 0: a reduction, else an
// inverse); a wave may then hold both.
std::vector<std::pair<int, int>> plan_mixed_waves(const int* m, const char* eigs, int n, int* cta0, int* cw,
                                                  int sms = 0);
size_t inv_resident_workspace(int m);
size_t tridiag_resident_workspace(int m);
bool resident_fits(int m, bool eig);
cudaError_t launch_invert_resident(const InvTask* d_tasks, const InvTask* h_tasks, int n, DeviceStatus* status,
                                   cudaStream_t st);
cudaError_t launch_tridiag_resident(const EigTask* d_tasks, const EigTask* h_tasks, int n, DeviceStatus* status,
                                    cudaStream_t st);
// One wave of both kinds in one cooperative launch: ninv inverses (cta0 from 0)
// and neig reductions (cta0 from 0 among the reductions' CTAs), each team on
// its own CTAs.
cudaError_t launch_resident_mix(const InvTask* d_inv, const InvTask* h_inv, int ninv, const EigTask* d_eig,
                                const EigTask* h_eig, int neig, DeviceStatus* status, cudaStream_t st);
void launch_copy(const CopyTask* tasks, int ntask, cudaStream_t st);
// Sum of squares of blocks (eq. curOff6's ||all levels below||_F^2): task i's
// rows x cols entries (column-major, leading dimension ld) summed into
// partial[i] by one CTA, then *acc += sum_i partial[i] in index order by one
// CTA (deterministic).
struct SumSqTask {
  const double* p;
  int rows, cols, ld;
};
void launch_sumsq(const SumSqTask* tasks, int ntask, double* partial, double* acc, cudaStream_t st);
// One CTA waits on words[0] (never set) with words[1] as its abort word and
// stores what the bounded wait returned in words[2] (words zeroed by the caller).
cudaError_t launch_bounded_wait_selftest(unsigned long long* words, DeviceStatus* status, cudaStream_t st);
void launch_scatter(const double* val, const int64_t* dst_off, int64_t nnz, double* base, cudaStream_t st);
// status->amax_bits = max(status->amax_bits, bits of max_e |val[e]|); NaN sets status->numeric.
void launch_amax(const double* val, int64_t nnz, DeviceStatus* status, cudaStream_t st);
// status->asymmetric = 1 when val[e] != val[tpos[e]] for some e.
void launch_asymmetry(const double* val, const int64_t* tpos, int64_t nnz, DeviceStatus* status, cudaStream_t st);

// Vector kernels of the solve.  Multi-vectors are column-major with leading
// dimension ld; `ncol` columns.
void launch_permute_in(const double* b, int64_t n, int ncol, const int32_t* perm, double* ye,
                       int64_t ld_e, cudaStream_t st);
void launch_permute_out(const double* xe, int64_t ld_e, int64_t n, int ncol, const int32_t* perm,
                        double* x, cudaStream_t st);
// The same into / out of an FP32 extended vector (the precision form's traversal).
void launch_permute_in32(const double* b, int64_t n, int ncol, const int32_t* perm, float* ye, int64_t ld_e,
                         cudaStream_t st);
void launch_permute_out32(const float* xe, int64_t ld_e, int64_t n, int ncol, const int32_t* perm, double* x,
                          cudaStream_t st);
void launch_spmv(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                 const double* x, double* y, int ncol, cudaStream_t st);
// Segmented multi-vectors (GMRES on a batched plan): the n rows split into
// nseg segments, rows [seg_off[s], seg_off[s+1]) of every column; entry
// (i, c) belongs to group g = c * nseg + seg[i].  nseg = 1 with seg_off and
// seg NULL is the plain case, group g = c.
struct Segments {
  int nseg = 1;
  const int64_t* seg_off = nullptr;   // device, nseg + 1
  const int32_t* seg = nullptr;       // device, n: segment of each row
};
// out[g] = sum over the rows of group g of x(i, c) * y(i, c), deterministic
// two-pass reduction through `partial` (ncol * dot_partials(nseg) doubles).
constexpr int kDotBlocks = 152;
inline int dot_parts(int nseg) { return nseg >= kDotBlocks ? 1 : kDotBlocks / nseg; }
inline size_t dot_partials(int nseg) { return (size_t)nseg * dot_parts(nseg); }
void launch_dot(const double* x, const double* y, int64_t n, int ncol, const Segments& sg, double* partial,
                double* out, cudaStream_t st);
// y(i, c) += sign * coef[g] * x(i, c)
void launch_axpy_col(const double* coef, double sign, const double* x, double* y, int64_t n,
                     int ncol, const Segments& sg, cudaStream_t st);
// y(i, c) = x(i, c) / sqrt(nrm2[g]) (0 where nrm2[g] == 0 or mask[g] == 0)
void launch_scale_col(const double* nrm2, const int* mask, const double* x, double* y, int64_t n,
                      int ncol, const Segments& sg, cudaStream_t st);
// u(i, c) = sum_j coef[j * G + g] * V_j(i, c), V_j at V + j * stride, G = ncol * nseg
void launch_combine(const double* coef, int nvec, const double* V, int64_t stride, double* u,
                    int64_t n, int ncol, const Segments& sg, cudaStream_t st);
// r = b - r (in place on r)
void launch_residual(const double* b, double* r, int64_t count, cudaStream_t st);

}  // namespace lrs
