// kernels.cu -- device kernels of liblrs (sm_103a): the FP64 gather GEMM
// (the precision form's products are in tc_gemm.cu), the traversal GEMV / narrow
// GEMM, block copies, SpMV and the GMRES vector kernels (per column, or per
// (column, instance) segment on a batched plan).
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

// Programmatic dependent launch of the traversal kernels: a kernel lets the
// next launch of its stream start as soon as every CTA has begun, and waits for
// the previous grid to finish (its writes visible) before it touches the
// vectors -- the launch and CTA-scheduling latency of ~600 dependent launches
// per application then overlaps the previous phase.  Without the launch
// attribute both instructions do nothing.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <class... P, class... A>
void launch_maybe_pdl(void (*kernel)(P...), unsigned grid, unsigned block, cudaStream_t st, bool pdl, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---------------------------------------------------------------------------
// Gather GEMM: one CTA per 64 x 64 output tile; the tile sums all its terms
// in a fixed order (deterministic, no atomics), then writes
// C = init + sign * sum.  Used for the Gram matrices of Compress (eq. lra),
// the projections R_k = A_k V and Q_k^T = V^T B_k^T, the products
// A_pp^{-1} A_{p,k}, the Schur updates of Eliminate (Sec. 2.2) and the
// block products of the solve (Alg. 3, 4).
// ---------------------------------------------------------------------------
// The FP64 form (the precision form's products run on the tensor cores,
// tc_gemm.cu).
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

// Narrow gather GEMM: tiles of 64 rows x 16 columns (column 16 tj); thread
// (r, c) with r = tid / 16, c = tid % 16 owns rows 4r..4r+3 of column c.
// Split over the contraction: with S > 1, CTA (task, s) takes the K chunks
// g = s, s + S, ... of the task's terms (counted across terms in order) and
// writes its partial tile to part; gemm_narrow_reduce then adds the S partials
// of each output in order s = 0..S-1 (deterministic) and applies init and sign.
template <class V>
__global__ void __launch_bounds__(256) gemm_narrow_kernel(const GemmTaskT<V>* __restrict__ tasks,
                                                          const GemmTermT<V>* __restrict__ terms, int S,
                                                          V* __restrict__ part) {
  constexpr int TN = 16;
  __shared__ V As[kTrvChunks * kTileK][kTile + 1];
  __shared__ V Bs[kTrvChunks * kTileK][TN + 1];
  const GemmTaskT<V> t = tasks[blockIdx.x / S];
  pdl_enter();
  const int split = (int)blockIdx.x % S;
  const int row0 = t.ti * kTile, col0 = t.tj * TN;
  const int m = min(kTile, t.rows - row0), n = min(TN, t.cols - col0);
  const int tid = threadIdx.x;
  const int r0 = (tid >> 4) * 4, c = tid & 15;
  const bool active = r0 < m && c < n;
  V acc[4] = {V(0), V(0), V(0), V(0)};
  int g = 0;                                     // chunk counter across the terms
  for (int it = 0; it < t.nterm; ++it) {
    const GemmTermT<V> gt = terms[t.term0 + it];
    const bool ta = gt.trans & 1, tb = (gt.trans >> 1) & 1;
    const V* __restrict__ A = ta ? gt.A + (size_t)row0 * gt.lda : gt.A + row0;
    const V* __restrict__ B = tb ? gt.B + col0 : gt.B + (size_t)col0 * gt.ldb;
    const int nch = (gt.k + kTileK - 1) / kTileK;
    // this CTA's chunks of the term: ch = ch0, ch0 + S, ... (g + ch = split mod S);
    // kTrvChunks of them staged at once (their loads all in flight), then
    // summed chunk by chunk in order: the same order as one chunk at a time
    const int ch0 = ((split - g) % S + S) % S;
    for (int cb = ch0; cb < nch; cb += kTrvChunks * S) {
      int kcs[kTrvChunks];
#pragma unroll
      for (int cc = 0; cc < kTrvChunks; ++cc) {
        const int ch = cb + cc * S;
        kcs[cc] = ch < nch ? min(kTileK, gt.k - ch * kTileK) : 0;
      }
#pragma unroll
      for (int cc = 0; cc < kTrvChunks; ++cc) {
        const int k0 = (cb + cc * S) * kTileK, kc = kcs[cc];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int i, kk;
          if (!ta) { i = tid & 63; kk = (tid >> 6) + 4 * q; }
          else { kk = tid & 15; i = (tid >> 4) + 16 * q; }
          V v = V(0);
          if (i < m && kk < kc)
            v = ta ? A[(k0 + kk) + (size_t)i * gt.lda] : A[i + (size_t)(k0 + kk) * gt.lda];
          As[cc * kTileK + kk][i] = v;
        }
        const int kk = tid & 15, j = tid >> 4;
        V v = V(0);
        if (j < n && kk < kc)
          v = tb ? B[j + (size_t)(k0 + kk) * gt.ldb] : B[(k0 + kk) + (size_t)j * gt.ldb];
        Bs[cc * kTileK + kk][j] = v;
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int cc = 0; cc < kTrvChunks; ++cc)
          for (int kk = 0; kk < kcs[cc]; ++kk) {
            const V b = Bs[cc * kTileK + kk][c];
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a] = fma(As[cc * kTileK + kk][r0 + a], b, acc[a]);
          }
      }
      __syncthreads();
    }
    g += nch;
  }
  if (S > 1) {
    V* pt = part + (size_t)blockIdx.x * kTile * TN;
#pragma unroll
    for (int a = 0; a < 4; ++a) pt[(r0 + a) * TN + c] = acc[a];
    return;
  }
  if (!active) return;
  const V sign = (t.mode & kSubtract) ? V(-1) : V(1);
  V* C = t.C + row0 + (size_t)col0 * t.ldc;
  const V* D = t.D ? t.D + row0 + (size_t)col0 * t.ldd : nullptr;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = r0 + a;
    if (i >= m) continue;
    V init = V(0);
    if (D) init = D[i + (size_t)c * t.ldd];
    else if (t.mode & kAccumulate) init = C[i + (size_t)c * t.ldc];
    C[i + (size_t)c * t.ldc] = fma(sign, acc[a], init);
  }
}

template <class V>
__global__ void __launch_bounds__(256) gemm_narrow_reduce(const GemmTaskT<V>* __restrict__ tasks, int S,
                                                          const V* __restrict__ part) {
  constexpr int TN = 16;
  const GemmTaskT<V> t = tasks[blockIdx.x];
  pdl_enter();
  const int row0 = t.ti * kTile, col0 = t.tj * TN;
  const int m = min(kTile, t.rows - row0), n = min(TN, t.cols - col0);
  const int tid = threadIdx.x;
  const int r0 = (tid >> 4) * 4, c = tid & 15;
  if (r0 >= m || c >= n) return;
  V acc[4] = {V(0), V(0), V(0), V(0)};
  const V* pt = part + (size_t)blockIdx.x * S * kTile * TN;
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] += pt[(size_t)s * kTile * TN + (r0 + a) * TN + c];
  const V sign = (t.mode & kSubtract) ? V(-1) : V(1);
  V* C = t.C + row0 + (size_t)col0 * t.ldc;
  const V* D = t.D ? t.D + row0 + (size_t)col0 * t.ldd : nullptr;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = r0 + a;
    if (i >= m) continue;
    V init = V(0);
    if (D) init = D[i + (size_t)c * t.ldd];
    else if (t.mode & kAccumulate) init = C[i + (size_t)c * t.ldc];
    C[i + (size_t)c * t.ldc] = fma(sign, acc[a], init);
  }
}

template <class V>
void launch_narrow_t(const GemmTaskT<V>* tasks, int ntask, const GemmTermT<V>* terms, cudaStream_t st, int split,
                     V* part, bool pdl) {
  if (ntask <= 0) return;
  if (split <= 1 || part == nullptr) {
    launch_maybe_pdl(gemm_narrow_kernel<V>, ntask, 256, st, pdl, tasks, terms, 1, (V*)nullptr);
    return;
  }
  launch_maybe_pdl(gemm_narrow_kernel<V>, ntask * split, 256, st, pdl, tasks, terms, split, part);
  launch_maybe_pdl(gemm_narrow_reduce<V>, ntask, 256, st, pdl, tasks, split, (const V*)part);
}

void launch_gemm_narrow(const GemmTask* tasks, int ntask, const GemmTerm* terms, cudaStream_t st, int split,
                        double* part, bool pdl) {
  launch_narrow_t<double>(tasks, ntask, terms, st, split, part, pdl);
}

void launch_gemm_narrow32(const GemmTask32* tasks, int ntask, const GemmTerm32* terms, cudaStream_t st, int split,
                          float* part, bool pdl) {
  launch_narrow_t<float>(tasks, ntask, terms, st, split, part, pdl);
}

// Single right-hand side: y = init + sign * sum A b per 64-row tile, a
// matrix-vector product bound by HBM (every stored block read once).  Thread
// (r, q) with r = tid % 64, q = tid / 64 sums column chunks' columns
// q, q+4, .. of its row (coalesced 512-byte column segments); the four
// partial sums are added in order q = 0..3.  Split over the contraction as in
// gemm_narrow_kernel (S > 1: partial tiles, then gemv_reduce).
template <class V>
__global__ void __launch_bounds__(256) gemv_kernel(const GemmTaskT<V>* __restrict__ tasks,
                                                   const GemmTermT<V>* __restrict__ terms, int S,
                                                   V* __restrict__ part) {
  __shared__ V red[4][kTile];
  const GemmTaskT<V> t = tasks[blockIdx.x / S];
  pdl_enter();
  const int split = (int)blockIdx.x % S;
  const int row0 = t.ti * kTile;
  const int m = min(kTile, t.rows - row0);
  const int tid = threadIdx.x, r = tid & 63, q = tid >> 6;
  const bool on = r < m;
  V acc = V(0);
  int g = 0;
  for (int it = 0; it < t.nterm; ++it) {
    const GemmTermT<V> gt = terms[t.term0 + it];
    const V* __restrict__ A = gt.A + row0 + r;
    const V* __restrict__ B = gt.B;
    const int nch = (gt.k + kTileK - 1) / kTileK;
    // this CTA's chunks (as in gemm_narrow_kernel), kTrvChunks of them with
    // their loads in flight at once, summed in chunk order
    const int ch0 = ((split - g) % S + S) % S;
    for (int cb = ch0; cb < nch; cb += kTrvChunks * S) {
      V a[kTrvChunks][4], b[kTrvChunks][4];
#pragma unroll
      for (int cc = 0; cc < kTrvChunks; ++cc) {
        const int ch = cb + cc * S;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = ch * kTileK + q + 4 * u;
          const bool ok = ch < nch && on && k < gt.k;
          a[cc][u] = ok ? A[(size_t)k * gt.lda] : V(0);
          b[cc][u] = ok ? B[k] : V(0);
        }
      }
#pragma unroll
      for (int cc = 0; cc < kTrvChunks; ++cc)
        if (cb + cc * S < nch) {
#pragma unroll
          for (int u = 0; u < 4; ++u) acc = fma(a[cc][u], b[cc][u], acc);
        }
    }
    g += nch;
  }
  red[q][r] = acc;
  __syncthreads();
  if (q != 0) return;
  const V sum = ((red[0][r] + red[1][r]) + red[2][r]) + red[3][r];
  if (S > 1) {
    part[(size_t)blockIdx.x * kTile + r] = sum;
    return;
  }
  if (!on) return;
  const V sign = (t.mode & kSubtract) ? V(-1) : V(1);
  V init = V(0);
  if (t.D) init = t.D[row0 + r];
  else if (t.mode & kAccumulate) init = t.C[row0 + r];
  t.C[row0 + r] = fma(sign, sum, init);
}

template <class V>
__global__ void __launch_bounds__(64) gemv_reduce(const GemmTaskT<V>* __restrict__ tasks, int S,
                                                  const V* __restrict__ part) {
  const GemmTaskT<V> t = tasks[blockIdx.x];
  pdl_enter();
  const int row0 = t.ti * kTile;
  const int r = threadIdx.x;
  if (r >= min(kTile, t.rows - row0)) return;
  V sum = V(0);
  for (int s = 0; s < S; ++s) sum += part[((size_t)blockIdx.x * S + s) * kTile + r];
  const V sign = (t.mode & kSubtract) ? V(-1) : V(1);
  V init = V(0);
  if (t.D) init = t.D[row0 + r];
  else if (t.mode & kAccumulate) init = t.C[row0 + r];
  t.C[row0 + r] = fma(sign, sum, init);
}

template <class V>
void launch_gemv_t(const GemmTaskT<V>* tasks, int ntask, const GemmTermT<V>* terms, cudaStream_t st, int split,
                   V* part, bool pdl) {
  if (ntask <= 0) return;
  if (split <= 1 || part == nullptr) {
    launch_maybe_pdl(gemv_kernel<V>, ntask, 256, st, pdl, tasks, terms, 1, (V*)nullptr);
    return;
  }
  launch_maybe_pdl(gemv_kernel<V>, ntask * split, 256, st, pdl, tasks, terms, split, part);
  launch_maybe_pdl(gemv_reduce<V>, ntask, 64, st, pdl, tasks, split, (const V*)part);
}

void launch_gemv(const GemmTask* tasks, int ntask, const GemmTerm* terms, cudaStream_t st, int split,
                 double* part, bool pdl) {
  launch_gemv_t<double>(tasks, ntask, terms, st, split, part, pdl);
}

void launch_gemv32(const GemmTask32* tasks, int ntask, const GemmTerm32* terms, cudaStream_t st, int split,
                   float* part, bool pdl) {
  launch_gemv_t<float>(tasks, ntask, terms, st, split, part, pdl);
}

// The factor's blocks to FP32 storage (round to nearest), grid-stride over
// each task's entries; one CTA group per task.
__global__ void __launch_bounds__(256) to_f32_kernel(const ConvTask* __restrict__ tasks) {
  const ConvTask t = tasks[blockIdx.y];
  for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < t.count; i += (int64_t)gridDim.x * 256)
    t.dst[i] = __double2float_rn(t.src[i]);
}

void launch_to_f32(const ConvTask* tasks, int ntask, cudaStream_t st) {
  for (int t0 = 0; t0 < ntask; t0 += 65535) {
    const int n = ntask - t0 < 65535 ? ntask - t0 : 65535;
    to_f32_kernel<<<dim3(8, n), 256, 0, st>>>(tasks + t0);
  }
}

// ---------------------------------------------------------------------------
// Block copies (MergeRedNodes, placing V, V^T and -I of Compress).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) copy_kernel(const CopyTask* __restrict__ tasks) {
  const CopyTask t = tasks[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (t.mode == 1 || t.mode == 3) {
    // transposes through 32 x 32 tiles of shared memory (both sides coalesced);
    // mode 3 mirrors the lower triangle of a square block onto its upper one
    // in place: a tile is read completely before any of it is written, and
    // strictly upper tiles read only lower tiles, which are never written
    __shared__ double tile[32][33];
    for (int j0 = 0; j0 < t.cols; j0 += 32)
      for (int i0 = 0; i0 < t.rows; i0 += 32) {
        if (t.mode == 3 && i0 > j0) continue;
        for (int r = warp; r < 32; r += 8) {
          const int i = i0 + r, j = j0 + lane;
          if (i < t.rows && j < t.cols) tile[r][lane] = t.src[j + (size_t)i * t.lds];
        }
        __syncthreads();
        for (int c = warp; c < 32; c += 8) {
          const int i = i0 + lane, j = j0 + c;
          if (i < t.rows && j < t.cols && (t.mode == 1 || i < j)) t.dst[i + (size_t)j * t.ldd] = tile[lane][c];
        }
        __syncthreads();
      }
    return;
  }
  for (int j = warp; j < t.cols; j += 8)
    for (int i = lane; i < t.rows; i += 32) {
      double v;
      if (t.mode == 0) v = t.src[i + (size_t)j * t.lds];
      else if (t.mode == 2) v = (i == j) ? t.alpha : 0.0;
      else v = (i == j + t.lds) ? t.alpha : 0.0;         // mode 4: a column piece of alpha * I
      t.dst[i + (size_t)j * t.ldd] = v;
    }
}

// Block reduction of 256 values in a fixed order (deterministic).
__device__ double block_sum256(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  return red[0];
}

__global__ void __launch_bounds__(256) sumsq_kernel(const SumSqTask* __restrict__ tasks,
                                                    double* __restrict__ partial) {
  __shared__ double red[256];
  const SumSqTask t = tasks[blockIdx.x];
  double s = 0.0;
  for (int j = 0; j < t.cols; ++j)
    for (int i = threadIdx.x; i < t.rows; i += 256) {
      const double v = t.p[i + (size_t)j * t.ld];
      s = fma(v, v, s);
    }
  const double tot = block_sum256(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) sum_ordered_kernel(const double* __restrict__ partial, int n,
                                                          double* acc) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += partial[i];
  const double tot = block_sum256(s, red);
  if (threadIdx.x == 0) *acc += tot;
}

void launch_sumsq(const SumSqTask* tasks, int ntask, double* partial, double* acc, cudaStream_t st) {
  if (ntask <= 0) return;
  sumsq_kernel<<<ntask, 256, 0, st>>>(tasks, partial);
  sum_ordered_kernel<<<1, 256, 0, st>>>(partial, ntask, acc);
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

__global__ void asymmetry_kernel(const double* __restrict__ val, const int64_t* __restrict__ tpos, int64_t nnz,
                                 DeviceStatus* status) {
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    bad |= !(val[e] == val[tpos[e]]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(&status->asymmetric, 1);
}

void launch_asymmetry(const double* val, const int64_t* tpos, int64_t nnz, DeviceStatus* status, cudaStream_t st) {
  if (nnz > 0) asymmetry_kernel<<<152 * 2, 256, 0, st>>>(val, tpos, nnz, status);
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

__global__ void permute_in32_kernel(const double* __restrict__ b, int64_t n, int ncol,
                                    const int32_t* __restrict__ perm, float* __restrict__ ye, int64_t ld) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e % n, c = e / n;
    ye[k + c * ld] = (float)b[perm[k] + c * n];
  }
}

__global__ void permute_out32_kernel(const float* __restrict__ xe, int64_t ld, int64_t n, int ncol,
                                     const int32_t* __restrict__ perm, double* __restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e % n, c = e / n;
    x[perm[k] + c * n] = (double)xe[k + c * ld];
  }
}

void launch_permute_in32(const double* b, int64_t n, int ncol, const int32_t* perm, float* ye, int64_t ld_e,
                         cudaStream_t st) {
  permute_in32_kernel<<<152 * 4, 256, 0, st>>>(b, n, ncol, perm, ye, ld_e);
}

void launch_permute_out32(const float* xe, int64_t ld_e, int64_t n, int ncol, const int32_t* perm, double* x,
                          cudaStream_t st) {
  permute_out32_kernel<<<152 * 4, 256, 0, st>>>(xe, ld_e, n, ncol, perm, x);
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

// Block (s * parts + p, c) sums rows lo + p * 256 + t + k * parts * 256 of
// segment s; with one segment this is a plain grid-stride dot.
__global__ void __launch_bounds__(256) dot_partial_kernel(const double* __restrict__ x,
                                                          const double* __restrict__ y, int64_t n,
                                                          int nseg, int parts,
                                                          const int64_t* __restrict__ seg_off,
                                                          double* __restrict__ partial) {
  const int c = blockIdx.y;
  const int sgm = blockIdx.x / parts, part = blockIdx.x - sgm * parts;
  const int64_t lo = seg_off ? seg_off[sgm] : 0, hi = seg_off ? seg_off[sgm + 1] : n;
  const double* xc = x + (size_t)c * n;
  const double* yc = y + (size_t)c * n;
  double s = 0.0;
  for (int64_t i = lo + part * (int64_t)blockDim.x + threadIdx.x; i < hi; i += (int64_t)parts * blockDim.x)
    s = fma(xc[i], yc[i], s);
  __shared__ double red[8];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partial[((size_t)c * nseg + sgm) * parts + part] = t;
  }
}

__global__ void dot_final_kernel(const double* __restrict__ partial, int parts, double* __restrict__ out) {
  const size_t g = blockIdx.x;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < parts; ++i) t += partial[g * parts + i];
    out[g] = t;
  }
}

void launch_dot(const double* x, const double* y, int64_t n, int ncol, const Segments& sg, double* partial,
                double* out, cudaStream_t st) {
  const int parts = dot_parts(sg.nseg);
  dot_partial_kernel<<<dim3(sg.nseg * parts, ncol), 256, 0, st>>>(x, y, n, sg.nseg, parts, sg.seg_off, partial);
  dot_final_kernel<<<ncol * sg.nseg, 32, 0, st>>>(partial, parts, out);
}

__device__ __forceinline__ int64_t group_of(int64_t e, int64_t n, const int32_t* __restrict__ seg, int nseg) {
  const int64_t c = e / n;
  return seg ? c * nseg + seg[e - c * n] : c;
}

__global__ void axpy_col_kernel(const double* __restrict__ coef, double sign, const double* __restrict__ x,
                                double* __restrict__ y, int64_t n, int ncol, const int32_t* __restrict__ seg,
                                int nseg) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ncol;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = fma(sign * coef[group_of(e, n, seg, nseg)], x[e], y[e]);
}

void launch_axpy_col(const double* coef, double sign, const double* x, double* y, int64_t n, int ncol,
                     const Segments& sg, cudaStream_t st) {
  axpy_col_kernel<<<152 * 8, 256, 0, st>>>(coef, sign, x, y, n, ncol, sg.seg, sg.nseg);
}

__global__ void scale_col_kernel(const double* __restrict__ nrm2, const int* __restrict__ mask,
                                 const double* __restrict__ x, double* __restrict__ y, int64_t n, int ncol,
                                 const int32_t* __restrict__ seg, int nseg) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = group_of(e, n, seg, nseg);
    const double d = sqrt(nrm2[g]);
    y[e] = (d != 0.0 && mask[g]) ? x[e] / d : 0.0;
  }
}

void launch_scale_col(const double* nrm2, const int* mask, const double* x, double* y, int64_t n, int ncol,
                      const Segments& sg, cudaStream_t st) {
  scale_col_kernel<<<152 * 8, 256, 0, st>>>(nrm2, mask, x, y, n, ncol, sg.seg, sg.nseg);
}

__global__ void combine_kernel(const double* __restrict__ coef, int nvec, const double* __restrict__ V,
                               int64_t stride, double* __restrict__ u, int64_t n, int64_t ngroup,
                               const int32_t* __restrict__ seg, int nseg) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * (ngroup / nseg);
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = group_of(e, n, seg, nseg);
    double s = 0.0;
    for (int j = 0; j < nvec; ++j) s = fma(coef[j * ngroup + g], V[j * stride + e], s);
    u[e] = s;
  }
}

void launch_combine(const double* coef, int nvec, const double* V, int64_t stride, double* u, int64_t n,
                    int ncol, const Segments& sg, cudaStream_t st) {
  combine_kernel<<<152 * 8, 256, 0, st>>>(coef, nvec, V, stride, u, n, (int64_t)ncol * sg.nseg, sg.seg,
                                          sg.nseg);
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
