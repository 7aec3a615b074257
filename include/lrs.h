/* lrs.h -- C ABI of a GB300 (sm_103a) implementation of the hierarchical
 * sparse solver of Pouransari, Coulier & Darve, "Fast hierarchical solvers for
 * sparse matrices using extended sparsification and low-rank approximation"
 * (arXiv 1510.07363).
 *
 * The problem (Sec. 1, eq. linsys): solve A x = b for a sparse n x n matrix A
 * with an accuracy eps fixed a priori; factor once, then solve for many
 * right-hand sides, stand-alone or as the preconditioner of GMRES (Sec. 5.2).
 *
 *   lrs_analyze  host only: nested partitioning, H-tree, block pattern and
 *                elimination order (Sec. 3, Alg. 1 without numbers)
 *   lrs_factor   GPU: Algorithm 1 -- merge, compress (eq. lra, eq. cutOff1),
 *                eliminate super-node and black-node, level by level
 *   lrs_apply    GPU: Algorithms 2-4, one forward + backward traversal
 *   lrs_solve    GPU: restarted GMRES preconditioned by lrs_apply
 *
 * Conventions shared by every call:
 *  - Status: every function returning int returns LRS_OK (0) or an LRS_ERR_*
 *    code; lrs_status_string() names it.  No C++ exception crosses this ABI
 *    and no call exits the process.  Out-parameters are written only on
 *    LRS_OK, except lrs_solve_info, which is always filled.
 *  - Ownership: the caller owns every array it passes; the library copies
 *    what it keeps.  lrs_plan and lrs_factor are opaque and owned by the
 *    library until the matching *_destroy call.
 *  - Dense multi-vectors are column-major n x nrhs with leading dimension n.
 *  - Floating point is IEEE binary64 throughout this interface.
 *  - GPU calls run on the stream given in lrs_factor_opts (NULL: the legacy
 *    default stream) of the device current at lrs_factor time, and return
 *    after that stream has finished the call's work.
 */
#ifndef LRS_H
#define LRS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LRS_API __attribute__((visibility("default")))
#else
#define LRS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define LRS_OK 0
#define LRS_ERR_INVALID_ARG 1    /* bad pointer, size, option or pattern */
#define LRS_ERR_OOM 2            /* device or host allocation failed */
#define LRS_ERR_SINGULAR_PIVOT 3 /* a pivot block had an exactly zero pivot */
#define LRS_ERR_NOT_CONVERGED 4  /* GMRES stopped at maxit above tol */
#define LRS_ERR_TIMEOUT 5        /* a bounded device wait expired */
#define LRS_ERR_CUDA 6           /* a CUDA runtime call failed */
#define LRS_ERR_NUMERIC 7        /* NaN or Inf met in the factorization */
#define LRS_ERR_STATE 8          /* call out of order (e.g. solve before factor) */

typedef struct lrs_plan lrs_plan;
typedef struct lrs_factor lrs_factor_t;

/* Device allocator hooks.  alloc returns a device pointer of at least `bytes`
 * bytes aligned to 256, usable on `stream`, or NULL on failure; free releases
 * it.  Both NULL: the library uses cudaMalloc / cudaFree. */
typedef void* (*lrs_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*lrs_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

/* A sparse matrix in CSR form (host memory) with one point per unknown for the
 * coordinate bisection that builds the nested partitioning (Sec. 3).
 * Column indices of a row must be distinct; they need not be sorted.  The
 * pattern's block structure is symmetrised: a block is kept for both
 * directions of every adjacent cluster pair (Def. adj). */
typedef struct {
  int64_t n;               /* rows = columns, >= 1 */
  const int64_t* rowptr;   /* n + 1 entries, rowptr[0] = 0 */
  const int32_t* colind;   /* rowptr[n] entries in [0, n) */
  const double* val;       /* rowptr[n] values; lrs_analyze ignores them */
  int dim;                 /* coordinate dimension, 1..8 */
  const double* coords;    /* n * dim, row-major (point k at coords[k*dim]) */
} lrs_csr;

typedef struct {
  int leaf_size;           /* target unknowns per leaf cluster (depth = 0) */
  int depth;               /* tree depth l >= 1; 0: ceil(log2(n / leaf_size)) */
  int separation;          /* smallest cluster distance (Def. distance) of a
                              well-separated pair: 0 or 2 the paper's Def. wellSep
                              (not adjacent); 3 the stronger variant of Sec. 7
                              (not adjacent and no cluster adjacent to both), which
                              compresses fewer interactions and keeps more fill */
} lrs_analyze_opts;

typedef struct {
  double eps;              /* truncation sigma_k / sigma_0 >= eps (eq. cutOff1), >= 0,
                              on the whole stacked block of eq. lra; eps = 0 keeps every
                              singular value (an exact factorization) */
  void* stream;            /* cudaStream_t for every GPU call on this factor */
  lrs_alloc_fn alloc;      /* optional device allocator (see above) */
  lrs_free_fn free;
  void* alloc_ctx;
  int profile;             /* nonzero: time every kernel launch with CUDA events */
  int symmetry;            /* LRS_SYM_DETECT (0), LRS_SYM_GENERAL or LRS_SYM_SYMMETRIC */
  int precision;           /* LRS_PREC_FP64 (0) or LRS_PREC_TF32 (= LRS_PREC_FP32, the precision form) */
  int trunc_rule;          /* LRS_TRUNC_CUTOFF1 (0) or LRS_TRUNC_CUROFF6 (see below) */
  int gemm;                /* engine of the FP64 block products: LRS_GEMM_AUTO (0), _FP64 or _EMU */
} lrs_factor_opts;

/* Engines of the FP64 block products -- the Schur updates A_qk -= A_qp
 * (A_pp^{-1} A_pk) and the products A_pp^{-1} A_pk (Sec. 2.2), the
 * projections and the Gram matrices of the compression (Sec. 4.3).
 * LRS_GEMM_EMU forms the FP64 products on the tensor cores by Ozaki's
 * splitting: per group of 512 values of k each row of op(A) and each column
 * of op(B) is scaled by its largest power of two and cut into eight 7-bit
 * digits (exact BF16 numbers); the 36 digit products that matter are summed
 * exactly in FP32 on the tensor cores and combined in 64-bit integers.  Its
 * error per group is below 2^-41 max_k |a_ik| max_k |b_kj| (an FP64 dot
 * product of length 512 may err by 2^-35 of the same), plus, when a row of
 * op(A) and a column of op(B) peak in different groups, at most 2^(cut - 58)
 * per group of the product of their maxima over the whole contraction (cut =
 * 5 + ceil(log2(chunks of 64 values of k))): an output's running sum is kept at
 * the largest row and column scales seen; results are deterministic.  LRS_GEMM_FP64
 * uses FP64 FMAs on the CUDA cores.  LRS_GEMM_AUTO is LRS_GEMM_EMU.  The
 * precision form's products are TF32 (LRS_PREC_TF32) whatever the engine;
 * its FP64 Gram matrices (eps < LRS_PREC_FP32_GRAM_EPS) use the engine.
 * LRS_GEMM_TF32 names the precision form's split for lrs_block_gemm. */
#define LRS_GEMM_AUTO 0
#define LRS_GEMM_FP64 1
#define LRS_GEMM_EMU 2
#define LRS_GEMM_TF32 3

/* Truncation rules of the compression (Sec. 6).  LRS_TRUNC_CUTOFF1, eq.
 * cutOff1: keep sigma_k >= eps sigma_0 of the stacked block of eq. lra.
 * LRS_TRUNC_CUROFF6, eq. curOff6 (Sec. 6.3): keep the smallest k with
 * ||M - U_k S_k V_k^T||_F = (sum_{j >= k} sigma_j^2)^(1/2) < eps N, where
 * N^2 sums the squared Frobenius norms of every block of the current level
 * and of the levels below, each level's blocks taken as the level starts
 * (after MergeRedNodes); at the leaf level N = ||A||_F.  On a plan of
 * lrs_analyze_batch N covers every instance's blocks. */
#define LRS_TRUNC_CUTOFF1 0
#define LRS_TRUNC_CUROFF6 1

/* The precision form: the factorization's block products -- the Schur
 * updates A_qk -= A_qp (A_pp^{-1} A_pk), the products A_pp^{-1} A_pk, the
 * projections R_k, Q_k^T and, for eps >= LRS_PREC_FP32_GRAM_EPS, the
 * compression Gram matrices -- run on the tensor cores: operands rounded from
 * the FP64 blocks to FP32 and split into a TF32 head and tail, three TF32
 * products per pair with FP32 accumulation (relative error about 1e-6), the
 * results added to FP64 blocks.  Pivot-block inverses, the spectra and rank
 * decisions, the traversals and GMRES stay FP64, so GMRES refines the
 * solution to the requested tolerance.  Below LRS_PREC_FP32_GRAM_EPS the Gram
 * matrices stay FP64: a Gram matrix with product error u resolves
 * sigma_k / sigma_0 near eps only to about u / (2 eps).  Once factored, the
 * stored blocks (A_pp^{-1}, A_qp, A_pp^{-1} A_pq) move to FP32 storage (half
 * the bytes; lrs_stats.factor_bytes) and the traversals run in FP32
 * arithmetic on FP32 copies of the vectors (relative rounding about 1e-7,
 * far below the truncation); right-preconditioned GMRES is flexible, so it
 * still reaches the requested tolerance in FP64. */
#define LRS_PREC_FP64 0
#define LRS_PREC_TF32 1        /* the precision form: TF32 tensor-core products, FP32 storage */
#define LRS_PREC_FP32 LRS_PREC_TF32   /* the same form under its storage type's name */
#define LRS_PREC_FP32_GRAM_EPS 1e-2

/* Symmetric matrices (A = A^T, Sec. 4.3: A_k = B_k) need only half of the
 * compression work, and every Schur update A_qk -= A_qp A_pp^{-1} A_pk is the
 * transpose of the one for (k, q): the factorization then computes one of
 * each pair (and the lower half of each diagonal block) and transposes.
 * LRS_SYM_DETECT uses that path when the stored values are exactly symmetric
 * (pattern and values; tested on the device), LRS_SYM_SYMMETRIC when the
 * caller asserts it, LRS_SYM_GENERAL never. */
#define LRS_SYM_DETECT 0
#define LRS_SYM_GENERAL 1
#define LRS_SYM_SYMMETRIC 2

/* Per-kernel-class launch profile (see lrs_factor_profile).  flops and bytes
 * are the algorithmic counts of the launched work, computed on the host from
 * the block sizes (not hardware counters). */
#define LRS_PROF_FACTOR_GEMM 0   /* Gram, projections, A_pp^{-1} A_pk, Schur (FP64 FMAs) */
#define LRS_PROF_INVERT 1        /* pivot-block inverses */
#define LRS_PROF_SPECTRUM 2      /* spectra of the Gram matrices */
#define LRS_PROF_COPY 3          /* merge, V, V^T, -I placement */
#define LRS_PROF_ASSEMBLE 4      /* leaf assembly, max |a_ij| */
#define LRS_PROF_APPLY_GEMM 5    /* forward / backward traversal products */
#define LRS_PROF_SPMV 6          /* A x in GMRES */
#define LRS_PROF_VECTOR 7        /* dots, axpys, scaling, permutations */
#define LRS_PROF_FACTOR_GEMM_F32 8   /* the same products on the tensor cores (precision form) */
#define LRS_PROF_FACTOR_GEMM_EMU 9   /* the FP64 products emulated on the tensor cores (LRS_GEMM_EMU) */
#define LRS_PROF_CLASSES 10
typedef struct {
  int64_t launches;
  double ms;               /* summed device time of the launches */
  double flops;
  double bytes;
} lrs_prof_entry;

/* GMRES sides (Sec. 5.2).  Right (default): GMRES on A M y = b, x = M y,
 * stopping on the true residual ||b - A x|| / ||b|| <= tol (eq. accres).
 * Left, the paper's form: GMRES on M A x = M b, stopping on the
 * preconditioned residual ||M (b - A x)|| / ||M b|| <= tol (eq.
 * GMRES_residual). */
#define LRS_GMRES_RIGHT 0
#define LRS_GMRES_LEFT 1

typedef struct {
  int restart;             /* Krylov dimension before restart, >= 1 (30) */
  int maxit;               /* total Arnoldi steps per right-hand side, >= 1 */
  double tol;              /* stopping tolerance of the chosen side (see above) */
  int side;                /* LRS_GMRES_RIGHT (0) or LRS_GMRES_LEFT */
  int precond_residual;    /* right side: nonzero also reports the preconditioned
                              residual (two more applications of M); the left
                              side always reports both */
} lrs_solve_opts;

typedef struct {
  int iters;               /* largest iteration count over the right-hand sides
                              (and instances of a batched plan) */
  int status;              /* LRS_OK or LRS_ERR_NOT_CONVERGED (on the side's criterion) */
  double rel_res;          /* largest true relative residual ||b - A x|| / ||b|| (eq. accres) */
  double rel_res_precond;  /* largest ||M (b - A x)|| / ||M b|| (eq. GMRES_residual);
                              -1 when not computed (right side, precond_residual = 0) */
} lrs_solve_info;

typedef struct {
  int depth;               /* l */
  int64_t n;               /* original unknowns */
  int64_t ext_n;           /* unknowns of the extended system (Sec. 4.5) */
  int64_t n_compress;      /* compressions performed */
  int64_t n_batches;       /* independent batches over all levels */
  double factor_ms;        /* device time of the last lrs_factor */
  double flops_factor;     /* algorithmic flops of the factorization's products and
                              inverses (Gram, projections, A_pp^{-1} A_pk, Schur) */
  double eig_flops;        /* algorithmic flops of the compression spectra */
  double eig_cycles[5];    /* SM cycles of the spectra per phase: tridiagonal reduction,
                              bisection, inverse iteration, Gram-Schmidt, back-transformation */
  int64_t factor_bytes;    /* device bytes held by the factor */
  int64_t apply_bytes;     /* bytes one lrs_apply reads from the stored factor */
  int max_rank;            /* largest rank r of any compression */
  int max_pivot;           /* largest pivot block */
  int symmetric;           /* 1 when the symmetric path was taken */
  int precision;           /* LRS_PREC_* of the factorization */
  double flops_factor_f32; /* the part of flops_factor formed in FP32 */
  double host_ms;          /* host wall time of the last lrs_factor's planning and launches */
  double host_wait_ms;     /* ... of which spent waiting for the device (once per batch) */
  double host_elim_ms;     /* ... of which spent planning and launching eliminations */
  double host_merge_ms;    /* ... of which spent in leaf assembly and MergeRedNodes */
  double host_compress_ms; /* ... of which spent planning compressions before and after the
                              batch's sync (Gram, spectra, new nodes and edges) */
  double eig_lead_ms[5];   /* wall time of the same spectrum phases on the first CTA of each
                              block spread over several CTAs, summed over those blocks */
} lrs_stats;

/* lrs_analyze (Sec. 3 and the symbolic part of Alg. 1): builds the nested
 * partitioning P_0..P_l by recursive coordinate bisection (split along the
 * axis of largest extent, ties to the lowest axis; order by (coordinate,
 * index); the first floor(|S|/2) indices form child 0), the cluster
 * adjacency of every level (Def. adj), and the elimination order: at each
 * level, greedy batches of super-nodes with no edge between them, scanned by
 * ascending cluster index (Sec. 6 item 6 allows any order).  Host only; A->val
 * may be NULL.  Errors: LRS_ERR_INVALID_ARG for a NULL pointer, n < 1, dim
 * outside 1..8, a column index outside [0, n), a repeated column in a row,
 * a coordinate that is not finite, depth outside 1..24, leaf_size < 1 with
 * depth 0, or separation other than 0, 2 or 3. */
LRS_API int lrs_analyze(const lrs_csr* A, const lrs_analyze_opts* opts, lrs_plan** out);

/* lrs_analyze_batch: the batched form -- `count` independent matrices A[0..
 * count-1] (an array of lrs_csr, host memory) analysed into one plan, so that
 * lrs_factor eliminates them together, every level's clusters of all
 * instances in the same batches and launches, and lrs_solve runs one GMRES
 * per instance and right-hand side.  The paper treats one matrix at a time;
 * the union is the block-diagonal matrix diag(A[0], ..., A[count-1]), rows of
 * instance k following those of instance k-1 (lrs_plan_export what = 5 gives
 * the offsets).  Instance k is partitioned exactly as lrs_analyze(A[k], opts)
 * would (depth d_k from opts), and its subtree becomes one cluster of the
 * union's tree: instances are placed by descending d_k (ascending k on ties)
 * at leaf offsets that are multiples of 2^(d_k); l = ceil(log2 sum 2^(d_k));
 * clusters holding no instance are empty.  No cluster then mixes instances,
 * so the factorization and the preconditioner of each instance are those of
 * the instance alone.  Values for lrs_factor are the instances' CSR values
 * concatenated in order.  Errors: those of lrs_analyze for any instance;
 * LRS_ERR_INVALID_ARG for count < 1, more than 2^31 - 1 unknowns in all or
 * l > 24. */
LRS_API int lrs_analyze_batch(int count, const lrs_csr* A, const lrs_analyze_opts* opts, lrs_plan** out);

/* Symbolic records of the plan as int32 arrays, the same layout the test
 * oracle exports (node id = 4 * h + kind, h the heap index 2^level + j of the
 * node's cluster; kind 0 red-node, 1 super-node, 2 black-node, Def. Htree):
 *   0 perm: original index at each position            (n)
 *   1 leaf cluster offsets into perm                     (2^l + 1)
 *   2 batches: per level l..1 [level, nbatch, (count, super ids...)...]
 *   3 compressions in order: [super id, t, well-separated neighbour ids...]
 *   4 eliminations in order: [node id, degree, neighbour ids...]
 *   5 instances: per instance [first row, rows, first leaf, depth]  (4 per
 *     instance; one instance [0, n, 0, l] for lrs_analyze)
 * With out == NULL only *count is written.  LRS_ERR_INVALID_ARG for an
 * unknown `what`; *count is the number of int32 values. */
LRS_API int lrs_plan_export(const lrs_plan* plan, int what, int32_t* out, int64_t* count);
LRS_API void lrs_plan_destroy(lrs_plan* plan);

/* lrs_factor (Alg. 1): values `val` in the CSR order of the analysed pattern
 * (host pointer when val_on_device == 0, device pointer otherwise).  Returns
 * LRS_ERR_SINGULAR_PIVOT if a pivot block is exactly singular, LRS_ERR_NUMERIC
 * on NaN/Inf, LRS_ERR_OOM when the allocator fails, LRS_ERR_CUDA on a CUDA
 * error, LRS_ERR_INVALID_ARG (before any launch of that block) when a
 * super-node with a compression exceeds 3631 unknowns or a pivot block 9682:
 * the dense kernels keep per-row vectors in shared memory.  Such blocks come
 * with eps = 0 (no truncation) on large problems.  The factor holds a
 * reference to the plan: lrs_plan_destroy may come before lrs_factor_destroy
 * (the plan is freed with its last factor).  At most one lrs_factor may run on a device at a time (calls from
 * several threads must be serialised): the dense kernels of large blocks are
 * cooperative launches whose CTAs wait on one another. */
LRS_API int lrs_factor(const lrs_plan* plan, const double* val, int val_on_device,
               const lrs_factor_opts* opts, lrs_factor_t** out);

/* lrs_apply (Alg. 2-4): x = M b for nrhs columns, M the approximate inverse
 * held by the factor.  b and x are device pointers when on_device != 0,
 * host pointers otherwise; they may not alias. */
LRS_API int lrs_apply(lrs_factor_t* f, const double* b, double* x, int nrhs, int on_device);

/* lrs_solve: restarted GMRES on A x = b preconditioned by the factor, x0 = 0,
 * each right-hand side to its own tolerance: right preconditioning (A M y = b,
 * x = M y) to the true relative residual tol, or the paper's left
 * preconditioning (M A x = M b) to the preconditioned residual tol
 * (opts->side).  On a plan of lrs_analyze_batch every instance
 * and right-hand side is a GMRES of its own (its rows of the column; inner
 * products over those rows only), all advancing in lock step through shared
 * traversal and SpMV launches.  Pointers as for lrs_apply.  Returns
 * LRS_ERR_NOT_CONVERGED (x still written) when some column stops at maxit. */
LRS_API int lrs_solve(lrs_factor_t* f, const double* b, double* x, int nrhs, int on_device,
              const lrs_solve_opts* opts, lrs_solve_info* info);

/* lrs_apply_static: the same x = M b as lrs_apply, but it allocates no device
 * memory.  It is for callers that cannot call cudaMalloc when they apply the
 * preconditioner -- code running inside another framework's fixed memory
 * pool or under a hard memory budget, or on a path where an allocation could
 * fail or stall.  The paper has no counterpart; this is an interface choice.
 *  - b and x are device pointers (column-major n x nrhs); the caller owns them.
 *  - Its scratch (three extended vectors and the traversal's task tables) is a
 *    file-scope device array of 2^21 doubles (16 MiB) that every GPU loading
 *    this library holds until the process exits.  A request that does not fit
 *    (about ext_n * nrhs > 699050 for small factors) returns
 *    LRS_ERR_INVALID_ARG before any GPU work.
 *  - The device current at the call must be the factor's (the one current at
 *    lrs_factor); otherwise LRS_ERR_INVALID_ARG before any GPU work.
 *  - A factor of the precision form (FP32 storage) is refused with
 *    LRS_ERR_INVALID_ARG; lrs_apply serves it.
 *  - The call cannot be captured into a CUDA graph: it synchronises the
 *    factor's stream (below).  Its first call on a device also looks up the
 *    array's device address (with that device current); make that first call
 *    while no stream of the device is capturing.
 *  - Every call reuses the same array: calls that overlap on the GPU (other
 *    streams, other threads, other factors) race and must be serialised by the
 *    caller.  The call synchronises the factor's stream before it returns. */
LRS_API int lrs_apply_static(lrs_factor_t* f, const double* b, double* x, int nrhs);

/* Per-compression ranks in compression order (what = 5), pivot sizes in
 * elimination order (what = 6), and GMRES iteration counts of the last
 * lrs_solve (what = 7): one per column, or on a batched plan one per (column
 * c, instance k) at index c * count + k.  Same calling convention as
 * lrs_plan_export. */
LRS_API int lrs_factor_export(const lrs_factor_t* f, int what, int32_t* out, int64_t* count);
/* Singular values of compression k (largest first, min(rho, m) of them); with
 * out == NULL only *count is written. */
LRS_API int lrs_factor_sigma(const lrs_factor_t* f, int64_t k, double* out, int64_t* count);
LRS_API int lrs_factor_stats(const lrs_factor_t* f, lrs_stats* out);
/* Accumulated launch profile of every GPU call on f since it was created or
 * since the last call with reset != 0 (which zeroes it after copying).
 * out has LRS_PROF_CLASSES entries.  All zero unless opts.profile was set. */
LRS_API int lrs_factor_profile(lrs_factor_t* f, lrs_prof_entry* out, int reset);

/* lrs_selftest_bounded_wait: checks on the current device the bounded wait
 * that the CTAs of the resident dense kernels use between one another.  One
 * CTA waits on a flag that nothing sets; the wait must give up after its time
 * limit (2 s), set the kernel status's timeout word and the team's abort word.
 * Returns LRS_ERR_TIMEOUT when it did exactly that (the expected outcome; the
 * context stays usable), LRS_ERR_STATE when the wait ended otherwise,
 * LRS_ERR_OOM / LRS_ERR_CUDA on allocation or launch failure.  *waited_ms
 * receives the kernel's duration.  The paper has no counterpart: the
 * resident kernels are this implementation's. */
LRS_API int lrs_selftest_bounded_wait(double* waited_ms);
/* lrs_block_gemm: one block product on the current device with the engine
 * given (LRS_GEMM_FP64, LRS_GEMM_EMU or LRS_GEMM_TF32):
 *   C = init + sign op(A) op(B),  op(A) rows x k, op(B) k x cols,
 * init = C when accumulate != 0 (else 0), sign = -1 when subtract != 0 (else
 * +1); every matrix column-major in device memory with the leading dimension
 * given, op(X) = X^T when transX != 0.  It is the product that each Schur
 * update of Eliminate performs (Sec. 2.2), exposed so that the engines can be
 * checked and timed on their own.  Synchronous; *ms (optional) receives the
 * kernel's duration.  Errors: LRS_ERR_INVALID_ARG (sizes, null pointers, an
 * unknown engine, k > 32768 for LRS_GEMM_EMU), LRS_ERR_TIMEOUT (a tensor-core
 * wait expired), LRS_ERR_OOM, LRS_ERR_CUDA. */
LRS_API int lrs_block_gemm(int engine, int rows, int cols, int k, const double* A, int lda, int transa,
                           const double* B, int ldb, int transb, double* C, int ldc, int accumulate,
                           int subtract, double* ms);
LRS_API void lrs_factor_destroy(lrs_factor_t* f);

/* ---- The serving form ---------------------------------------------------
 * A request loop around resident factorizations.  The paper factors once and
 * solves many right-hand sides (Sec. 1); the serving form keeps many factors
 * resident and serves a stream of requests against them.  It has no
 * counterpart in the paper; it is built from lrs_factor and lrs_solve.
 *  - lrs_server_factor queues a factorization.  It is admitted when a worker
 *    is free and its reservation (reserve_bytes; 0: 65536 bytes per unknown)
 *    fits in hbm_budget next to the resident factors and the other admitted
 *    factorizations; once built the factor stays resident (its reservation
 *    replaced by the bytes it holds) until lrs_server_evict.  A reservation
 *    above the whole budget is refused: lrs_server_factor returns LRS_ERR_OOM.
 *  - lrs_server_solve queues a GMRES solve (lrs_solve semantics) against a
 *    factor ticket, resident or still queued.  Solves go before factorizations.
 *    A worker takes the oldest solve whose factor is built and idle, with the
 *    later queued solves against the same factor and the same lrs_solve_opts
 *    while their right-hand sides total at most max_batch_rhs (continuous
 *    batching): one multi-column GMRES, every column its own Krylov process,
 *    the columns scattered back to their requests.
 *  - `workers` requests run at once.  With the library's executor every
 *    factor has its own CUDA stream and stream-ordered allocations, so solves
 *    on different factors overlap on the device (one factor runs one solve at
 *    a time); factorizations run one at a time, as lrs_factor requires.
 *  - lrs_server_wait blocks until the request has finished, fills *info and
 *    forgets the ticket (a factor ticket stays valid for solves and evict);
 *    a second wait on the same ticket returns LRS_ERR_INVALID_ARG.
 *  - Factorizations are admitted in submission order; one that does not fit
 *    waits (ahead of later ones) until evictions free enough of the budget.
 *  - Host pointers only.  val, b and x belong to the caller and must stay
 *    valid until the request's lrs_server_wait returns.
 *  - Executor hooks: factor_fn / solve_fn / release_fn replace the library's
 *    GPU executor (all three or none); they run on the server's worker
 *    threads, concurrently for different factors.
 * Errors: LRS_ERR_INVALID_ARG for bad options, an unknown ticket or a solve
 * against a ticket that is not a factor; LRS_ERR_STATE for a solve against an
 * evicted factor or requests cancelled by lrs_server_destroy; a failed
 * factorization's status is also the status of the solves queued against it. */
typedef struct lrs_server lrs_server;
typedef int (*lrs_exec_factor_fn)(void* ctx, const lrs_plan* plan, const double* val, double eps, int precision,
                                  void** factor, size_t* bytes);
typedef int (*lrs_exec_solve_fn)(void* ctx, void* factor, const double* b, double* x, int nrhs,
                                 const lrs_solve_opts* opts, lrs_solve_info* info);
typedef void (*lrs_exec_release_fn)(void* ctx, void* factor);

typedef struct {
  size_t hbm_budget;       /* bytes that resident and admitted factors may hold, > 0 */
  int workers;             /* requests executed at once, >= 1 */
  int max_batch_rhs;       /* right-hand sides merged into one solve, >= 1 */
  lrs_exec_factor_fn factor_fn;   /* executor hooks (see above); NULL: the GPU executor */
  lrs_exec_solve_fn solve_fn;
  lrs_exec_release_fn release_fn;
  void* exec_ctx;
} lrs_server_opts;

typedef struct {
  int status;              /* LRS_OK or the request's LRS_ERR_* code */
  int iters;               /* solves: largest iteration count of the GMRES it ran in */
  double rel_res;          /* solves: largest true relative residual of that GMRES */
  int batch_rhs;           /* solves: right-hand sides of that GMRES */
  size_t bytes;            /* factorizations: bytes the factor holds */
  double queue_ms;         /* submission to start */
  double run_ms;           /* start to end */
} lrs_request_info;

LRS_API int lrs_server_create(const lrs_server_opts* opts, lrs_server** out);
LRS_API int lrs_server_factor(lrs_server* s, const lrs_plan* plan, const double* val, double eps, int precision,
                              size_t reserve_bytes, int64_t* ticket);
LRS_API int lrs_server_solve(lrs_server* s, int64_t factor_ticket, const double* b, double* x, int nrhs,
                             const lrs_solve_opts* opts, int64_t* ticket);
LRS_API int lrs_server_wait(lrs_server* s, int64_t ticket, lrs_request_info* info);
/* Releases a factor once its queued and running solves are done; later solves
 * against it fail with LRS_ERR_STATE. */
LRS_API int lrs_server_evict(lrs_server* s, int64_t factor_ticket);
/* Bytes held by resident factors plus admitted reservations, resident
 * factors, and queued requests. */
LRS_API int lrs_server_stats(lrs_server* s, size_t* held_bytes, int* resident, int* queued);
/* Lets the running requests finish, drops the queued ones, releases every
 * factor and frees the server; its tickets are invalid afterwards (no
 * lrs_server_wait may be pending or follow). */
LRS_API void lrs_server_destroy(lrs_server* s);

/* Static description of a status code; never NULL. */
LRS_API const char* lrs_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LRS_H */
