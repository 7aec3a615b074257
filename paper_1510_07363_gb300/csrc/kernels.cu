// kernels.cu -- FP64 device kernels of liblrs (sm_103a).
//
// GB300 has ~2 FP64 FMA per clock per SM (1.19 TFLOP/s measured over 152
// SMs) against ~60x that in FP32, so every FP64 kernel here is bounded by the
// FP64 pipe, not by HBM: the designs keep that pipe fed (independent FMAs per
// thread, shared-memory staging so loads never stall it) and avoid spending
// FP64 issue slots on padding (warps whose part of a tile is empty skip the
// inner loop).
#include <algorithm>
#include <cstdio>

#include "kernels.cuh"

namespace lrs {

// ---------------------------------------------------------------------------
// Gather GEMM: one CTA per 64 x 64 output tile; the tile sums all its terms
// in a fixed order (deterministic, no atomics), then writes
// C = init + sign * sum.  Used for the Gram matrices of Compress (eq. lra),
// the projections R_k = A_k V and Q_k^T = V^T B_k^T, the products
// A_pp^{-1} A_{p,k}, the Schur updates of Eliminate (Sec. 2.2) and the
// block products of the solve (Alg. 3, 4).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gemm_kernel(const GemmTask* __restrict__ tasks,
                                                   const GemmTerm* __restrict__ terms) {
  __shared__ double As[kTileK][kTile + 1];
  __shared__ double Bs[kTileK][kTile + 1];
  const GemmTask t = tasks[blockIdx.x];
  const int row0 = t.ti * kTile, col0 = t.tj * kTile;
  const int m = min(kTile, t.rows - row0), n = min(kTile, t.cols - col0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wr = warp >> 1, wc = warp & 1;
  const int r0 = wr * 16 + (lane >> 3) * 4, c0 = wc * 32 + (lane & 7) * 4;
  const bool active = (wr * 16 < m) && (wc * 32 < n);
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  for (int it = 0; it < t.nterm; ++it) {
    const GemmTerm g = terms[t.term0 + it];
    const bool ta = g.trans & 1, tb = (g.trans >> 1) & 1;
    const double* __restrict__ A = ta ? g.A + (size_t)row0 * g.lda : g.A + row0;
    const double* __restrict__ B = tb ? g.B + col0 : g.B + (size_t)col0 * g.ldb;
    for (int k0 = 0; k0 < g.k; k0 += kTileK) {
      const int kc = min(kTileK, g.k - k0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int i, kk;
        if (!ta) { i = tid & 63; kk = (tid >> 6) + 4 * q; }
        else { kk = tid & 15; i = (tid >> 4) + 16 * q; }
        double v = 0.0;
        if (i < m && kk < kc)
          v = ta ? A[(k0 + kk) + (size_t)i * g.lda] : A[i + (size_t)(k0 + kk) * g.lda];
        As[kk][i] = v;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int j, kk;
        if (!tb) { kk = tid & 15; j = (tid >> 4) + 16 * q; }
        else { j = tid & 63; kk = (tid >> 6) + 4 * q; }
        double v = 0.0;
        if (j < n && kk < kc)
          v = tb ? B[j + (size_t)(k0 + kk) * g.ldb] : B[(k0 + kk) + (size_t)j * g.ldb];
        Bs[kk][j] = v;
      }
      __syncthreads();
      if (active) {
        for (int kk = 0; kk < kc; ++kk) {
          double av[4], bv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = As[kk][r0 + a];
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][c0 + b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
      }
      __syncthreads();
    }
  }
  if (!active) return;
  const double sign = (t.mode & kSubtract) ? -1.0 : 1.0;
  double* C = t.C + row0 + (size_t)col0 * t.ldc;
  const double* D = t.D ? t.D + row0 + (size_t)col0 * t.ldd : nullptr;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = c0 + b;
    if (j >= n) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = r0 + a;
      if (i >= m) continue;
      double init = 0.0;
      if (D) init = D[i + (size_t)j * t.ldd];
      else if (t.mode & kAccumulate) init = C[i + (size_t)j * t.ldc];
      C[i + (size_t)j * t.ldc] = fma(sign, acc[a][b], init);
    }
  }
}

void launch_gemm(const GemmTask* tasks, int ntask, const GemmTerm* terms, cudaStream_t st) {
  if (ntask > 0) gemm_kernel<<<ntask, 256, 0, st>>>(tasks, terms);
}

// ---------------------------------------------------------------------------
// Pivot-block inverse (the paper inverts pivot blocks, Sec. 5.1): in-place
// Gauss-Jordan with partial pivoting, one CTA per block, working in global
// memory (L1/L2 resident for the block sizes met here).  Row k is swapped with
// the first row of largest |a_ik|; the column interchanges that undo the row
// pivoting are applied at the end in reverse order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) invert_kernel(const InvTask* __restrict__ tasks,
                                                     DeviceStatus* status) {
  extern __shared__ double sm[];
  const InvTask t = tasks[blockIdx.x];
  const int m = t.m, lda = t.lda;
  double* A = t.A;
  double* f = sm;              // column k before the step
  double* rowk = sm + m;       // scaled row k
  int* ipiv = reinterpret_cast<int*>(sm + 2 * m);
  __shared__ double wbest[8];
  __shared__ int widx[8];
  __shared__ int s_p, s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) s_bad = 0;
  for (int k = 0; k < m; ++k) {
    double best = -1.0;
    int bi = m;
    for (int i = k + tid; i < m; i += 256) {
      const double v = fabs(A[i + (size_t)k * lda]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { wbest[warp] = best; widx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = wbest[0];
      int p = widx[0];
      for (int w = 1; w < 8; ++w)
        if (wbest[w] > b || (wbest[w] == b && widx[w] < p)) { b = wbest[w]; p = widx[w]; }
      s_p = p;
      ipiv[k] = p;
      if (!(b > 0.0) || p >= m) {
        s_bad = 1;
        if (b == 0.0) atomicExch(&status->singular, 1);
        else atomicExch(&status->numeric, 1);
      }
    }
    __syncthreads();
    if (s_bad) return;
    const int p = s_p;
    if (p != k)
      for (int j = tid; j < m; j += 256) {
        const double x = A[k + (size_t)j * lda];
        A[k + (size_t)j * lda] = A[p + (size_t)j * lda];
        A[p + (size_t)j * lda] = x;
      }
    __syncthreads();
    for (int i = tid; i < m; i += 256) f[i] = A[i + (size_t)k * lda];
    __syncthreads();
    const double inv = 1.0 / f[k];
    for (int j = tid; j < m; j += 256) {
      const double v = (j == k) ? inv : A[k + (size_t)j * lda] * inv;
      rowk[j] = v;
      A[k + (size_t)j * lda] = v;
    }
    __syncthreads();
    for (int j = warp; j < m; j += 8) {
      const double rj = rowk[j];
      double* col = A + (size_t)j * lda;
      for (int i = lane; i < m; i += 32) {
        if (i == k) continue;
        const double a = (j == k) ? 0.0 : col[i];
        col[i] = fma(-f[i], rj, a);
      }
    }
    __syncthreads();
  }
  for (int k = m - 1; k >= 0; --k) {
    const int p = ipiv[k];
    if (p != k)
      for (int i = tid; i < m; i += 256) {
        const double x = A[i + (size_t)k * lda];
        A[i + (size_t)k * lda] = A[i + (size_t)p * lda];
        A[i + (size_t)p * lda] = x;
      }
    __syncthreads();
  }
}

void launch_invert(const InvTask* tasks, int ntask, int max_m, DeviceStatus* status, cudaStream_t st) {
  if (ntask <= 0) return;
  const size_t smem = (size_t)max_m * (2 * sizeof(double) + sizeof(int)) + 16;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(invert_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  invert_kernel<<<ntask, 256, smem, st>>>(tasks, status);
}

// ---------------------------------------------------------------------------
// Compression spectrum (eq. lra, eq. cutOff1): the right singular vectors and
// singular values of the stacked matrix M are the eigenvectors and the square
// roots of the eigenvalues of its Gram matrix G = M^T M.  Parallel cyclic
// Jacobi on G, one CTA per matrix: each round rotates m/2 disjoint index
// pairs (round-robin schedule, pair 0 is (r, m'-1), pair t is
// ((r + t) mod (m'-1), (r - t) mod (m'-1)) for m' = m rounded up to even),
// first G <- G J and W <- W J column-wise, then G <- J^T G row-wise.  A pair is
// skipped when |g_pq| <= tol * sqrt(|g_pp g_qq|); a sweep without a rotation
// ends the iteration.  G lives in shared memory (odd leading dimension, so
// strided row access is conflict-free) when it fits, else in global memory.
// ---------------------------------------------------------------------------
constexpr int kEigSmemMax = 160;     // largest m kept in shared memory
constexpr int kEigMaxSweeps = 40;
constexpr double kEigTol = 1e-15;

__global__ void __launch_bounds__(256) eig_kernel(const EigTask* __restrict__ tasks,
                                                  DeviceStatus* status, int npair_max, int smem_m) {
  extern __shared__ double sm[];
  const EigTask t = tasks[blockIdx.x];
  const int m = t.m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (m == 0) {
    if (tid == 0) *t.rank = 0;
    return;
  }
  double* pc = sm;                                   // cosines of the round's pairs
  double* ps = pc + npair_max;                       // sines
  int* pp = reinterpret_cast<int*>(ps + npair_max);  // active pair list
  int* pq = pp + npair_max;
  int* order = pq + npair_max;                       // m' ints
  double* Gs = reinterpret_cast<double*>(order + 2 * npair_max + 2);
  const bool in_smem = m <= smem_m;          // smem holds a (smem_m | 1)^2 matrix
  const int ld = in_smem ? (m | 1) : m;
  double* G = in_smem ? Gs : t.G;
  double* W = t.W;
  __shared__ int s_nact, s_rank;
  if (in_smem)
    for (int j = warp; j < m; j += 8)
      for (int i = lane; i < m; i += 32) Gs[i + j * ld] = t.G[i + (size_t)j * m];
  for (int j = warp; j < m; j += 8)
    for (int i = lane; i < m; i += 32) W[i + (size_t)j * m] = (i == j) ? 1.0 : 0.0;
  __syncthreads();
  const int mp = m + (m & 1), npair = mp / 2, nr = mp - 1;
  int sweep = 0;
  for (; sweep < kEigMaxSweeps; ++sweep) {
    int rotations = 0;
    for (int r = 0; r < nr; ++r) {
      if (tid == 0) s_nact = 0;
      __syncthreads();
      for (int a = tid; a < npair; a += 256) {
        int p, q;
        if (a == 0) { p = r; q = mp - 1; }
        else { p = (r + a) % nr; q = (r - a + nr) % nr; }
        if (p > q) { int x = p; p = q; q = x; }
        if (q >= m) continue;
        const double gpq = G[p + (size_t)q * ld];
        const double gpp = G[p + (size_t)p * ld], gqq = G[q + (size_t)q * ld];
        if (gpq == 0.0 || fabs(gpq) <= kEigTol * sqrt(fabs(gpp) * fabs(gqq))) continue;
        const double tau = (gqq - gpp) / (2.0 * gpq);
        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + tt * tt);
        const int slot = atomicAdd(&s_nact, 1);
        pp[slot] = p;
        pq[slot] = q;
        pc[slot] = c;
        ps[slot] = tt * c;
      }
      __syncthreads();
      const int nact = s_nact;
      rotations += nact;
      if (nact == 0) continue;
      // per rotation: columns p, q of G and W and rows p, q of G, 6 flops per element pair
      if (tid == 0) atomicAdd(&status->eig_flops, 18ull * (unsigned long long)m * nact);
      // G <- G J, W <- W J: columns p, q of every active pair
      for (int a = warp; a < nact; a += 8) {
        const int p = pp[a], q = pq[a];
        const double c = pc[a], s = ps[a];
        double* gp = G + (size_t)p * ld;
        double* gq = G + (size_t)q * ld;
        for (int i = lane; i < m; i += 32) {
          const double x = gp[i], y = gq[i];
          gp[i] = fma(c, x, -s * y);
          gq[i] = fma(s, x, c * y);
        }
        double* wp = W + (size_t)p * m;
        double* wq = W + (size_t)q * m;
        for (int i = lane; i < m; i += 32) {
          const double x = wp[i], y = wq[i];
          wp[i] = fma(c, x, -s * y);
          wq[i] = fma(s, x, c * y);
        }
      }
      __syncthreads();
      // G <- J^T G: rows p, q of every active pair
      for (int a = warp; a < nact; a += 8) {
        const int p = pp[a], q = pq[a];
        const double c = pc[a], s = ps[a];
        for (int j = lane; j < m; j += 32) {
          const double x = G[p + (size_t)j * ld], y = G[q + (size_t)j * ld];
          G[p + (size_t)j * ld] = fma(c, x, -s * y);
          G[q + (size_t)j * ld] = fma(s, x, c * y);
        }
      }
      __syncthreads();
    }
    if (rotations == 0) break;
  }
  if (tid == 0 && sweep == kEigMaxSweeps) atomicExch(&status->eig_unconverged, 1);
  // sort eigenvalues descending (ties by index) by parallel ranking
  for (int k = tid; k < m; k += 256) {
    const double lk = G[k + (size_t)k * ld];
    if (lk != lk) atomicExch(&status->numeric, 1);
    int rk = 0;
    for (int j = 0; j < m; ++j) {
      const double lj = G[j + (size_t)j * ld];
      rk += (lj > lk) || (lj == lk && j < k);
    }
    order[rk] = k;
  }
  __syncthreads();
  for (int k = tid; k < m; k += 256) {
    const double l = G[order[k] + (size_t)order[k] * ld];
    t.sigma[k] = sqrt(fmax(l, 0.0));
  }
  __syncthreads();
  if (tid == 0) {
    const int nsv = min(t.rho, m);
    int r = 0;
    const double s0 = t.sigma[0];
    const double floor = t.eps > 0.0 ? t.floor_scale * __longlong_as_double((long long)*t.amax_bits) : 0.0;
    if (nsv > 0 && s0 > 0.0)
      for (int k = 0; k < nsv; ++k) r += (t.sigma[k] >= t.eps * s0) && (t.eps == 0.0 || t.sigma[k] > floor);
    s_rank = r;
    *t.rank = r;
  }
  __syncthreads();
  const int rank = s_rank;
  for (int c = warp; c < rank; c += 8) {
    const double* src = W + (size_t)order[c] * m;
    for (int i = lane; i < m; i += 32) t.V[i + (size_t)c * m] = src[i];
  }
}

void launch_eig(const EigTask* tasks, int ntask, int max_m, int max_small_m, DeviceStatus* status,
                cudaStream_t st) {
  if (ntask <= 0) return;
  const int npair_max = (max_m + 2) / 2 + 1;
  const size_t base = (size_t)npair_max * (2 * sizeof(double) + 4 * sizeof(int)) + 2 * sizeof(int) + 16;
  int smem_m = std::min(max_small_m, kEigSmemMax);
  size_t smem = base + (smem_m > 0 ? (size_t)(smem_m | 1) * (smem_m | 1) * sizeof(double) : 0);
  if (smem > 227 * 1024) {                 // pair tables of a very large block leave no room
    smem_m = 0;
    smem = base;
  }
  smem = (smem + 15) & ~size_t(15);
  cudaFuncSetAttribute(eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  eig_kernel<<<ntask, 256, smem, st>>>(tasks, status, npair_max, smem_m);
}

// ---------------------------------------------------------------------------
// Block copies (MergeRedNodes, placing V, V^T and -I of Compress).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) copy_kernel(const CopyTask* __restrict__ tasks) {
  const CopyTask t = tasks[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < t.cols; j += 8)
    for (int i = lane; i < t.rows; i += 32) {
      double v;
      if (t.mode == 0) v = t.src[i + (size_t)j * t.lds];
      else if (t.mode == 1) v = t.src[j + (size_t)i * t.lds];
      else v = (i == j) ? t.alpha : 0.0;
      t.dst[i + (size_t)j * t.ldd] = v;
    }
}

void launch_copy(const CopyTask* tasks, int ntask, cudaStream_t st) {
  if (ntask > 0) copy_kernel<<<ntask, 256, 0, st>>>(tasks);
}

__global__ void scatter_kernel(const double* __restrict__ val, const int64_t* __restrict__ off,
                               int64_t nnz, double* __restrict__ base) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    base[off[e]] = val[e];
}

void launch_scatter(const double* val, const int64_t* dst_off, int64_t nnz, double* base, cudaStream_t st) {
  if (nnz > 0) scatter_kernel<<<152 * 8, 256, 0, st>>>(val, dst_off, nnz, base);
}

__global__ void amax_kernel(const double* __restrict__ val, int64_t nnz, DeviceStatus* status) {
  double m = 0.0;
  bool nan = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const double a = fabs(val[e]);
    nan |= !(a <= 1.7976931348623157e308);
    m = fmax(m, a);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if (__any_sync(0xffffffffu, nan) && (threadIdx.x & 31) == 0) atomicExch(&status->numeric, 1);
  if ((threadIdx.x & 31) == 0) atomicMax(&status->amax_bits, (unsigned long long)__double_as_longlong(m));
}

void launch_amax(const double* val, int64_t nnz, DeviceStatus* status, cudaStream_t st) {
  if (nnz > 0) amax_kernel<<<152 * 2, 256, 0, st>>>(val, nnz, status);
}

// ---------------------------------------------------------------------------
// Vector kernels of the solve.
// ---------------------------------------------------------------------------
__global__ void permute_in_kernel(const double* __restrict__ b, int64_t n, int ncol,
                                  const int32_t* __restrict__ perm, double* __restrict__ ye, int64_t ld) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e % n, c = e / n;
    ye[k + c * ld] = b[perm[k] + c * n];
  }
}

__global__ void permute_out_kernel(const double* __restrict__ xe, int64_t ld, int64_t n, int ncol,
                                   const int32_t* __restrict__ perm, double* __restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e % n, c = e / n;
    x[perm[k] + c * n] = xe[k + c * ld];
  }
}

void launch_permute_in(const double* b, int64_t n, int ncol, const int32_t* perm, double* ye,
                       int64_t ld_e, cudaStream_t st) {
  permute_in_kernel<<<152 * 4, 256, 0, st>>>(b, n, ncol, perm, ye, ld_e);
}

void launch_permute_out(const double* xe, int64_t ld_e, int64_t n, int ncol, const int32_t* perm,
                        double* x, cudaStream_t st) {
  permute_out_kernel<<<152 * 4, 256, 0, st>>>(xe, ld_e, n, ncol, perm, x);
}

// y = A x for ncol columns: one warp per row, lanes stride the row's entries.
__global__ void __launch_bounds__(256) spmv_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ colind,
                                                   const double* __restrict__ val,
                                                   const double* __restrict__ x, double* __restrict__ y,
                                                   int ncol) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += warps) {
    const int64_t b = rowptr[row], e = rowptr[row + 1];
    for (int c = 0; c < ncol; ++c) {
      double s = 0.0;
      for (int64_t k = b + lane; k < e; k += 32) s = fma(val[k], x[colind[k] + c * n], s);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
      if (lane == 0) y[row + c * n] = s;
    }
  }
}

void launch_spmv(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                 const double* x, double* y, int ncol, cudaStream_t st) {
  spmv_kernel<<<152 * 16, 256, 0, st>>>(n, rowptr, colind, val, x, y, ncol);
}

__global__ void __launch_bounds__(256) dot_partial_kernel(const double* __restrict__ x,
                                                          const double* __restrict__ y, int64_t n,
                                                          double* __restrict__ partial) {
  const int c = blockIdx.y;
  const double* xc = x + (size_t)c * n;
  const double* yc = y + (size_t)c * n;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(xc[i], yc[i], s);
  __shared__ double red[8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partial[(size_t)c * kDotBlocks + blockIdx.x] = t;
  }
}

__global__ void dot_final_kernel(const double* __restrict__ partial, double* __restrict__ out) {
  const int c = blockIdx.x;
  __shared__ double red[kDotBlocks];
  for (int i = threadIdx.x; i < kDotBlocks; i += blockDim.x) red[i] = partial[(size_t)c * kDotBlocks + i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kDotBlocks; ++i) t += red[i];
    out[c] = t;
  }
}

void launch_dot(const double* x, const double* y, int64_t n, int ncol, double* partial, double* out,
                cudaStream_t st) {
  dot_partial_kernel<<<dim3(kDotBlocks, ncol), 256, 0, st>>>(x, y, n, partial);
  dot_final_kernel<<<ncol, 32, 0, st>>>(partial, out);
}

__global__ void axpy_col_kernel(const double* __restrict__ coef, double sign, const double* __restrict__ x,
                                double* __restrict__ y, int64_t n, int ncol) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ncol;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = fma(sign * coef[e / n], x[e], y[e]);
}

void launch_axpy_col(const double* coef, double sign, const double* x, double* y, int64_t n, int ncol,
                     cudaStream_t st) {
  axpy_col_kernel<<<152 * 8, 256, 0, st>>>(coef, sign, x, y, n, ncol);
}

__global__ void scale_col_kernel(const double* __restrict__ nrm2, const int* __restrict__ mask,
                                 const double* __restrict__ x, double* __restrict__ y, int64_t n, int ncol) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n;
    const double d = sqrt(nrm2[c]);
    y[e] = (d != 0.0 && mask[c]) ? x[e] / d : 0.0;
  }
}

void launch_scale_col(const double* nrm2, const int* mask, const double* x, double* y, int64_t n, int ncol,
                      cudaStream_t st) {
  scale_col_kernel<<<152 * 8, 256, 0, st>>>(nrm2, mask, x, y, n, ncol);
}

__global__ void combine_kernel(const double* __restrict__ coef, int nvec, const double* __restrict__ V,
                               int64_t stride, double* __restrict__ u, int64_t n, int ncol) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n;
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s = fma(coef[j * ncol + c], V[j * stride + e], s);
    u[e] = s;
  }
}

void launch_combine(const double* coef, int nvec, const double* V, int64_t stride, double* u, int64_t n,
                    int ncol, cudaStream_t st) {
  combine_kernel<<<152 * 8, 256, 0, st>>>(coef, nvec, V, stride, u, n, ncol);
}

__global__ void residual_kernel(const double* __restrict__ b, double* __restrict__ r, int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    r[e] = b[e] - r[e];
}

void launch_residual(const double* b, double* r, int64_t count, cudaStream_t st) {
  residual_kernel<<<152 * 8, 256, 0, st>>>(b, r, count);
}

}  // namespace lrs
