// dense.cu -- dense FP64 kernels on one block at a time: pivot-block inverses
// (Eliminate, Sec. 2.2) and the spectra of the compression Gram matrices
// (Compress, eq. lra / eq. cutOff1).
//
// A block is processed by a "team":
//  - one CTA (blocks that fit in shared memory, many per launch);
//  - resident teams (invert_resident_kernel, tridiag_resident_kernel): the
//    CTAs of a cooperative launch each hold a contiguous share of the block's
//    columns in shared memory for the whole run and exchange one column per
//    step through flags with bounded waits; blocks are packed into waves;
//  - sub-teams (eig_kernel<kSubTeam>): the rest of every large spectrum of a
//    batch in one cooperative launch, each block on its own CTAs with a
//    bounded flag barrier;
//  - a thread-block cluster or the whole grid, for blocks too large for the
//    resident forms.
// In the multi-CTA forms every scalar decision (pivot row, Householder
// reflector, norms, eigenvalue count) is made from the same data in the same
// order wherever it is needed, so all CTAs agree bit for bit.
#include <cooperative_groups.h>

#include <algorithm>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace lrs {
namespace {

// ---------------------------------------------------------------------------
// Bounded waits between the CTAs of one cooperative launch.  A flag word is 0
// until its producer publishes it (release); a waiter polls it (acquire) for
// at most kWaitNs of %globaltimer time, and also watches the team's abort
// word, so one failed wait ends every CTA's loop instead of leaving them
// spinning.  On expiry the waiter sets status->wait_timeout and the abort word.
// ---------------------------------------------------------------------------
constexpr unsigned long long kWaitNs = 2000000000ull;
constexpr unsigned long long kFlagBad = ~0ull;     // published instead of a pivot: stop

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Called by one thread.  Returns the flag's value, or 0 when the team aborted
// or the wait expired.
__device__ unsigned long long await_flag(const unsigned long long* flag, unsigned long long* abort_word,
                                         DeviceStatus* status) {
  unsigned long long v = ld_acquire(flag);
  if (v) return v;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    v = ld_acquire(flag);
    if (v) return v;
    if ((it & 15) == 15) {
      if (ld_acquire(abort_word)) return 0;
      if (global_ns() - t0 > kWaitNs) {
        atomicExch(&status->wait_timeout, 1);
        st_release(abort_word, 1);
        return 0;
      }
    }
    __nanosleep(32);
  }
}

// Barrier of a sub-team of CTAs inside one cooperative launch (bar: arrival
// count, generation, abort word).  Thread 0 reads the generation, arrives;
// the last to arrive resets the count and publishes the next generation, the
// others wait for it (bounded; an expired wait sets status->wait_timeout and
// the team's abort word, after which no member waits again, so the kernel
// runs to its end and the host reports the failure).
__device__ void sub_team_barrier(unsigned long long* bar, int size, DeviceStatus* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    if (size > 1 && !ld_acquire(&bar[2])) {
      const unsigned long long gen = ld_acquire(&bar[1]);
      __threadfence();
      const unsigned long long arrived = atomicAdd(&bar[0], 1ull) + 1;
      if (arrived == (unsigned long long)size) {
        atomicExch(&bar[0], 0ull);
        __threadfence();
        st_release(&bar[1], gen + 1);
      } else {
        const unsigned long long t0 = global_ns();
        for (unsigned it = 0; ld_acquire(&bar[1]) == gen; ++it) {
          if ((it & 15) == 15) {
            if (ld_acquire(&bar[2])) break;
            if (global_ns() - t0 > kWaitNs) {
              atomicExch(&status->wait_timeout, 1);
              st_release(&bar[2], 1);
              break;
            }
          }
          __nanosleep(32);
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Team kinds: one CTA (C = 1), a thread-block cluster (C = kDenseCluster),
// the whole grid of a cooperative launch working on a single block (C =
// kGridTeam, team size gridDim.x), or a sub-team of CTAs of a cooperative
// launch that works on several blocks at once (C = kSubTeam: CTAs [team0,
// team0 + team_size) of the launch, synchronised by sub_team_barrier).
// Columns are dealt out in chunks of CW columns.
constexpr int kGridTeam = 0;
constexpr int kSubTeam = -1;

template <int C>
struct Team {
  int rank = 0;
  int size = 1;
  unsigned long long* bar = nullptr;
  DeviceStatus* status = nullptr;
  __device__ Team() {
    if constexpr (C == kGridTeam) {
      rank = (int)blockIdx.x;
      size = (int)gridDim.x;
    } else if constexpr (C > 1) {
      rank = (int)cg::this_cluster().block_rank();
      size = C;
    }
  }
  __device__ Team(int r, int s, unsigned long long* b, DeviceStatus* st) : rank(r), size(s), bar(b), status(st) {}
  static constexpr int CW = (C == kGridTeam || C == kSubTeam) ? 16 : 32;
  __device__ void sync() const {
    if constexpr (C == kGridTeam) cg::this_grid().sync();
    else if constexpr (C == kSubTeam) sub_team_barrier(bar, size, status);
    else if constexpr (C > 1) cg::this_cluster().sync();
    else __syncthreads();
  }
  __device__ bool owns(int col) const { return ((col / CW) % size) == rank; }
  __device__ int gthread() const { return rank * 256 + (int)threadIdx.x; }
  __device__ int gwarp() const { return rank * 8 + ((int)threadIdx.x >> 5); }
  __device__ int nthreads() const { return size * 256; }
  __device__ int nwarps() const { return size * 8; }
};

// task index of this CTA
template <int C>
__device__ __forceinline__ int task_index() {
  if constexpr (C == kGridTeam) return 0;
  else return (int)blockIdx.x / C;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Sum over the CTA (same order in every CTA that calls it on the same data).
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += red[w];
  __syncthreads();
  return t;
}

// Maximum over the CTA (the same in every CTA that calls it on the same data).
__device__ __forceinline__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) t = fmax(t, red[w]);
  __syncthreads();
  return t;
}

// Householder reflector H = I - beta v v^T of entries k+1..m-1 of column k,
// with H x = alpha e_1: v_{k+1} = v0 and v_i = 2^sh col_i for i > k+1.  When
// the column's squared norm lies outside [2^-900, 2^900] -- fill at rounding
// level can leave a column whose squared norm is subnormal, and then 2 / v^T v
// overflows -- the column is first scaled by a power of two to unit size
// (exact); H does not depend on that scaling (v -> c v, beta -> beta / c^2).
// Inside the range sh = 0 and the arithmetic is the plain one.  Every thread
// of the CTA calls it and gets the same result.
struct Reflector {
  double v0, beta, alpha;
  int sh;
};
__device__ Reflector make_reflector(const double* col, int k, int m, double* red) {
  const int tid = threadIdx.x;
  double s2 = 0.0;
  for (int i = k + 1 + tid; i < m; i += 256) s2 = fma(col[i], col[i], s2);
  s2 = block_sum(s2, red);
  double x0 = col[k + 1];
  int sh = 0;
  if (s2 != 0.0 && !(s2 >= 0x1p-900 && s2 <= 0x1p+900)) {
    double a = 0.0;
    for (int i = k + 1 + tid; i < m; i += 256) a = fmax(a, fabs(col[i]));
    a = block_max(a, red);
    if (a > 0.0 && a <= 1.7976931348623157e308) {
      int ex;
      frexp(a, &ex);
      sh = 1 - ex;                                  // largest scaled entry in [1, 2)
      s2 = 0.0;
      for (int i = k + 1 + tid; i < m; i += 256) {
        const double c = ldexp(col[i], sh);
        s2 = fma(c, c, s2);
      }
      s2 = block_sum(s2, red);
      x0 = ldexp(x0, sh);
    }
  }
  const double as = (x0 >= 0.0) ? -sqrt(s2) : sqrt(s2);
  Reflector r;
  r.v0 = x0 - as;
  const double vtv = s2 - x0 * x0 + r.v0 * r.v0;
  r.beta = (s2 > 0.0 && vtv > 0.0) ? 2.0 / vtv : 0.0;
  r.alpha = (r.beta > 0.0) ? ldexp(as, -sh) : col[k + 1];
  r.sh = sh;
  return r;
}

// ---------------------------------------------------------------------------
// Pivot-block inverse by Gauss-Jordan with partial pivoting (in place).  At
// step k the row of largest |a_ik|, i >= k (first on ties), is swapped into
// row k; row k is scaled by the pivot's inverse, and every other row gets
// row_i -= a_ik * row_k with column k replaced by -a_ik / pivot.  The column
// interchanges that undo the row pivoting are applied at the end in reverse.
// ---------------------------------------------------------------------------
template <int C>
__global__ void __launch_bounds__(256) invert_kernel(const InvTask* __restrict__ tasks, DeviceStatus* status) {
  extern __shared__ double sm[];
  const InvTask t = tasks[task_index<C>()];
  const Team<C> team;
  const int m = t.m, lda = t.lda;
  double* A = t.A;
  double* f = sm;                                        // column k (after the swap)
  double* rowk = sm + m;                                 // scaled row k (own columns)
  int* ipiv = reinterpret_cast<int*>(sm + 2 * m);
  int* idx = ipiv + m;
  __shared__ double wbest[8];
  __shared__ int widx[8];
  __shared__ int s_p, s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int k = 0; k < m; ++k) {
    for (int i = tid; i < m; i += 256) f[i] = A[i + (size_t)k * lda];
    __syncthreads();
    double best = -1.0;
    int bi = m;
    for (int i = k + tid; i < m; i += 256) {
      const double v = fabs(f[i]);
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
      s_bad = !(b > 0.0) || p >= m;
      if (s_bad && team.rank == 0) {
        if (b == 0.0) atomicExch(&status->singular, 1);
        else atomicExch(&status->numeric, 1);
      }
      s_p = p;
      ipiv[k] = p;
      if (!s_bad && p != k) { const double x = f[k]; f[k] = f[p]; f[p] = x; }
    }
    __syncthreads();
    if (s_bad) return;                                   // every CTA of the team decides alike
    team.sync();                                         // column k read everywhere before it changes
    const int p = s_p;
    const double inv = 1.0 / f[k];
    for (int j = tid; j < m; j += 256) {
      if (!team.owns(j)) continue;
      const double a = A[k + (size_t)j * lda];
      const double b = (p != k) ? A[p + (size_t)j * lda] : a;
      if (p != k) A[p + (size_t)j * lda] = a;
      const double v = (j == k) ? inv : b * inv;
      rowk[j] = v;
      A[k + (size_t)j * lda] = v;
    }
    __syncthreads();
    for (int j = warp; j < m; j += 8) {
      if (!team.owns(j)) continue;
      const double rj = rowk[j];
      double* col = A + (size_t)j * lda;
      for (int i = lane; i < m; i += 32) {
        if (i == k) continue;
        const double a = (j == k) ? 0.0 : col[i];
        col[i] = fma(-f[i], rj, a);
      }
    }
    team.sync();
  }
  // undo the row pivoting: apply the column swaps (k, ipiv[k]) for k = m-1..0
  if constexpr (C == 1) {
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
  } else {
    if (tid == 0) {
      for (int j = 0; j < m; ++j) idx[j] = j;
      for (int k = m - 1; k >= 0; --k) { const int x = idx[k]; idx[k] = idx[ipiv[k]]; idx[ipiv[k]] = x; }
    }
    for (int j = warp; j < m; j += 8)
      if (team.owns(j))
        for (int i = lane; i < m; i += 32) t.W[i + (size_t)j * m] = A[i + (size_t)j * lda];
    team.sync();
    for (int j = warp; j < m; j += 8)
      if (team.owns(j)) {
        const double* src = t.W + (size_t)idx[j] * m;
        for (int i = lane; i < m; i += 32) A[i + (size_t)j * lda] = src[i];
      }
  }
}

// ---------------------------------------------------------------------------
// Pivot-block inverse on the whole GPU, columns resident in shared memory.
// The same Gauss-Jordan steps and arithmetic as invert_kernel.  CTA b holds
// columns [b cw, b cw + cw) in shared memory for the whole run.  Step k needs
// one thing from another CTA: column k after the pivot search (and the pivot
// row).  Its owner publishes that column to slot k of W and sets flag k to
// pivot + 1; every CTA waits for the flag, reads the column, and updates its
// own columns.  The owner of column k + 1 updates that column first and
// publishes step k + 1 before the rest of its update, so the steps overlap.
// No barrier is needed: the final column interchanges move each CTA's own
// columns straight to their places in A (every CTA has read its columns of A
// before it published its first step, and each CTA waits on every step).
// W: m x m column slots, then the abort word and m step flags (zeroed by the
// launcher).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void publish_pivot(const double* col, int k, int m, double* slot, double* local,
                                              unsigned long long* flag, DeviceStatus* status, double* wbest,
                                              int* widx, unsigned long long* s_own) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double best = -1.0;
  int bi = m;
  for (int i = k + tid; i < m; i += 256) {
    const double v = fabs(col[i]);
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
  double b = wbest[0];
  int p = widx[0];
  for (int w = 1; w < 8; ++w)
    if (wbest[w] > b || (wbest[w] == b && widx[w] < p)) { b = wbest[w]; p = widx[w]; }
  const bool bad = !(b > 0.0) || p >= m;
  if (!bad)
    for (int i = tid; i < m; i += 256) {
      const double v = (i == k) ? col[p] : (i == p) ? col[k] : col[i];
      slot[i] = v;
      local[i] = v;                                // the publisher keeps its own copy
    }
  __syncthreads();
  if (tid == 0) {
    if (bad) {
      if (b == 0.0) atomicExch(&status->singular, 1);
      else atomicExch(&status->numeric, 1);
    }
    __threadfence();
    const unsigned long long v = bad ? kFlagBad : (unsigned long long)p + 1;
    *s_own = v;
    st_release(flag, v);
  }
}

// the block of a resident wave that this CTA works on (tasks ordered by cta0)
template <class T>
__device__ int resident_task(const T* tasks, int ntask, int bid) {
  __shared__ int s_task;
  if (threadIdx.x == 0) {
    int k = 0;
    while (k + 1 < ntask && tasks[k + 1].cta0 <= bid) ++k;
    s_task = k;
  }
  __syncthreads();
  return s_task;
}

// bid: this CTA's index among the CTAs of the resident inverses of its launch
__device__ void invert_resident_body(const InvTask* __restrict__ tasks, int ntask, int bid, DeviceStatus* status,
                                     double* sm) {
  const InvTask t = tasks[resident_task(tasks, ntask, bid)];
  const int m = t.m, lda = t.lda, cw = t.cw;
  const int tid = threadIdx.x;
  const int c0 = (bid - t.cta0) * cw;
  const int nc = min(cw, m - c0);
  double* cols = sm;                              // own columns, leading dimension m
  double* fbuf = sm + (size_t)cw * m;             // column k after the interchange, two buffers
  double* r = fbuf + 2 * (size_t)m;               // row k of the step, own columns
  unsigned long long* abort_word = reinterpret_cast<unsigned long long*>(t.W + (size_t)m * m);
  unsigned long long* flags = abort_word + 1;
  __shared__ double wbest[8];
  __shared__ int widx[8];
  __shared__ unsigned long long s_flag, s_own;
  if (nc <= 0) return;
  for (int j = 0; j < nc; ++j)
    for (int i = tid; i < m; i += 256) cols[(size_t)j * m + i] = t.A[i + (size_t)(c0 + j) * lda];
  __syncthreads();
  if (c0 == 0) publish_pivot(cols, 0, m, t.W, fbuf, &flags[0], status, wbest, widx, &s_own);
  for (int k = 0; k < m; ++k) {
    double* f = fbuf + (size_t)(k & 1) * m;
    // the CTA that published step k already holds its column; the others wait
    // for the flag and read the column from the slot
    const bool mine = k >= c0 && k < c0 + nc;
    if (!mine && tid == 0) s_flag = await_flag(&flags[k], abort_word, status);
    __syncthreads();
    const unsigned long long fl = mine ? s_own : s_flag;
    if (fl == 0 || fl == kFlagBad) return;         // every CTA leaves alike
    const int p = (int)(fl - 1);
    if (!mine) {
      const double* slot = t.W + (size_t)k * m;
      for (int i = tid; i < m; i += 256) f[i] = __ldcg(slot + i);
    }
    __syncthreads();
    const double inv = 1.0 / f[k];
    if (tid < nc) {                                // interchange rows k and p; row k of the result
      double* cj = cols + (size_t)tid * m;
      const double a = cj[k];
      const double b = (p != k) ? cj[p] : a;
      if (p != k) cj[p] = a;
      const double v = (c0 + tid == k) ? inv : b * inv;
      r[tid] = v;
      cj[k] = v;
    }
    __syncthreads();
    const int nx = k + 1;
    const int jx = (nx < m && nx >= c0 && nx < c0 + nc) ? nx - c0 : -1;
    auto update = [&](int j) {
      const double rj = r[j];
      double* cj = cols + (size_t)j * m;
      const bool diag = (c0 + j == k);
      for (int i = tid; i < m; i += 256) {
        if (i == k) continue;
        const double a = diag ? 0.0 : cj[i];
        cj[i] = fma(-f[i], rj, a);
      }
    };
    if (jx >= 0) {                                 // next step's column first, then publish it
      update(jx);
      __syncthreads();
      publish_pivot(cols + (size_t)jx * m, nx, m, t.W + (size_t)nx * m, fbuf + (size_t)(nx & 1) * m, &flags[nx],
                    status, wbest, widx, &s_own);
    }
    for (int j = 0; j < nc; ++j)
      if (j != jx) update(j);
    __syncthreads();
  }
  // column interchanges (k, p_k) for k = m-1..0: position j receives column idx[j]
  int* idx = reinterpret_cast<int*>(fbuf);
  int* pos = idx + m;
  if (tid == 0) {
    for (int j = 0; j < m; ++j) idx[j] = j;
    for (int k = m - 1; k >= 0; --k) {
      const int p = (int)(__ldcg(&flags[k]) - 1);
      const int x = idx[k];
      idx[k] = idx[p];
      idx[p] = x;
    }
    for (int j = 0; j < m; ++j) pos[idx[j]] = j;
  }
  __syncthreads();
  for (int j = 0; j < nc; ++j) {
    double* dst = t.A + (size_t)pos[c0 + j] * lda;
    for (int i = tid; i < m; i += 256) dst[i] = cols[(size_t)j * m + i];
  }
}

// ---------------------------------------------------------------------------
// Householder tridiagonalisation of a Gram matrix on the whole GPU, columns
// resident in shared memory: the reduction of eig_kernel (same arithmetic, in
// the same order, so T is bit-identical) with two exchanges per step.
//  - The owner of column k forms reflector k (v, beta) from its column and
//    publishes it with d_k, e_k to slot k of H (flag k).
//  - Every CTA with columns right of k forms p_j = beta column_j . v for them
//    and writes p_j to the step's p slot, then adds its column count to the
//    step's counter; those CTAs wait until the counter reaches m - k - 1, read
//    all of p, form K and w alike, and apply B -= v w^T + w v^T to their
//    columns -- column k+1 first, whose owner then publishes reflector k+1.
// H: m slots of m + 4 doubles, m p slots of m doubles, then the abort word, m
// reflector flags and m counters (zeroed by the launcher).
// ---------------------------------------------------------------------------
__device__ void publish_reflector(const double* col, int k, int m, double* slot, unsigned long long* flag,
                                  double* red) {
  const int tid = threadIdx.x;
  const Reflector rf = make_reflector(col, k, m, red);
  for (int i = k + 1 + tid; i < m; i += 256) slot[i] = (i == k + 1) ? rf.v0 : (rf.sh ? ldexp(col[i], rf.sh) : col[i]);
  if (tid == 0) {
    slot[m] = col[k];
    slot[m + 1] = rf.alpha;
    slot[m + 2] = rf.beta;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    st_release(flag, 1);
  }
}

// the last two diagonal entries and the last off-diagonal one (no reflector)
__device__ void publish_tail(const double* col, int k, int m, double* slot, unsigned long long* flag) {
  if (threadIdx.x == 0) {
    slot[m] = col[k];
    slot[m + 1] = (k + 1 < m) ? col[k + 1] : 0.0;
    slot[m + 2] = 0.0;
    __threadfence();
    st_release(flag, 1);
  }
}

// bid: this CTA's index among the CTAs of the resident reductions of its launch
__device__ void tridiag_resident_body(const EigTask* __restrict__ tasks, int ntask, int bid, DeviceStatus* status,
                                      double* sm) {
  const EigTask t = tasks[resident_task(tasks, ntask, bid)];
  const int m = t.m, cw = t.cw;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c0 = (bid - t.cta0) * cw;
  const int nc = min(cw, m - c0);
  const size_t ls = (size_t)m + 4;
  double* cols = sm;                              // own columns of G, leading dimension m
  double* v = sm + (size_t)cw * m;                // reflector of the step
  double* w = v + m;                              // p, then w
  double* P = t.H + (size_t)m * ls;               // p slots
  unsigned long long* abort_word = reinterpret_cast<unsigned long long*>(P + (size_t)m * m);
  unsigned long long* vflag = abort_word + 1;
  unsigned long long* cnt = vflag + m;
  __shared__ double red[8];
  __shared__ unsigned long long s_flag;
  if (nc <= 0) return;
  // G's lower triangle is the data; the upper one is its mirror
  for (int j = 0; j < nc; ++j) {
    const int gj = c0 + j;
    for (int i = tid; i < m; i += 256)
      cols[(size_t)j * m + i] = (i >= gj) ? t.G[i + (size_t)gj * m] : t.G[gj + (size_t)i * m];
  }
  __syncthreads();
  auto owns = [&](int col) { return col >= c0 && col < c0 + nc; };
  auto column = [&](int col) { return cols + (size_t)(col - c0) * m; };
  if (m >= 3 && owns(0)) publish_reflector(column(0), 0, m, t.H, &vflag[0], red);
  for (int k = 0; k + 2 < m; ++k) {
    const bool trailing = c0 + nc - 1 > k;        // this CTA has columns right of k
    if (!trailing) break;                         // nothing of it changes any more
    if (tid == 0) s_flag = await_flag(&vflag[k], abort_word, status);
    __syncthreads();
    if (s_flag == 0) return;
    const double* slot = t.H + (size_t)k * ls;
    for (int i = k + 1 + tid; i < m; i += 256) v[i] = __ldcg(slot + i);
    const double bk = __ldcg(slot + m + 2);
    __syncthreads();
    const int nx = k + 1;
    if (bk == 0.0) {
      if (owns(nx) && nx + 2 < m) publish_reflector(column(nx), nx, m, t.H + (size_t)nx * ls, &vflag[nx], red);
      __syncthreads();
      continue;
    }
    // p_j = bk * column_j . v over own columns right of k
    double* pk = P + (size_t)k * m;
    for (int j = c0 + warp; j < c0 + nc; j += 8) {
      if (j <= k) continue;
      const double* cj = column(j);
      double s = 0.0;
      for (int i = k + 1 + lane; i < m; i += 32) s = fma(cj[i], v[i], s);
      s = warp_sum(s);
      if (lane == 0) pk[j] = bk * s;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(&cnt[k], (unsigned long long)(c0 + nc - max(c0, k + 1)));
      const unsigned long long want = (unsigned long long)(m - k - 1);
      const unsigned long long t0 = global_ns();
      s_flag = 1;
      for (unsigned it = 0; ld_acquire(&cnt[k]) < want; ++it) {
        if ((it & 15) == 15) {
          if (ld_acquire(abort_word)) { s_flag = 0; break; }
          if (global_ns() - t0 > kWaitNs) {
            atomicExch(&status->wait_timeout, 1);
            st_release(abort_word, 1);
            s_flag = 0;
            break;
          }
        }
        __nanosleep(32);
      }
    }
    __syncthreads();
    if (s_flag == 0) return;
    double pv = 0.0;
    for (int i = k + 1 + tid; i < m; i += 256) {
      const double pi = __ldcg(pk + i);
      w[i] = pi;
      pv = fma(pi, v[i], pv);
    }
    const double K = 0.5 * bk * block_sum(pv, red);
    for (int i = k + 1 + tid; i < m; i += 256) w[i] = fma(-K, v[i], w[i]);
    __syncthreads();
    auto update = [&](int j) {
      double* cj = column(j);
      const double vj = v[j], wj = w[j];
      for (int i = k + 1 + tid; i < m; i += 256) cj[i] = fma(-v[i], wj, fma(-w[i], vj, cj[i]));
    };
    if (owns(nx)) {
      update(nx);
      __syncthreads();
      if (nx + 2 < m) publish_reflector(column(nx), nx, m, t.H + (size_t)nx * ls, &vflag[nx], red);
    }
    for (int j = max(c0, k + 1); j < c0 + nc; ++j)
      if (j != nx) update(j);
    __syncthreads();
  }
  // the last 2 x 2 block is final once step m - 3 is applied
  if (m >= 2 && owns(m - 2)) publish_tail(column(m - 2), m - 2, m, t.H + (size_t)(m - 2) * ls, &vflag[m - 2]);
  if (owns(m - 1)) publish_tail(column(m - 1), m - 1, m, t.H + (size_t)(m - 1) * ls, &vflag[m - 1]);
}

__global__ void __launch_bounds__(256, 1) invert_resident_kernel(const InvTask* __restrict__ tasks, int ntask,
                                                                 DeviceStatus* status) {
  extern __shared__ double sm[];
  invert_resident_body(tasks, ntask, (int)blockIdx.x, status, sm);
}

__global__ void __launch_bounds__(256, 1) tridiag_resident_kernel(const EigTask* __restrict__ tasks, int ntask,
                                                                  DeviceStatus* status) {
  extern __shared__ double sm[];
  tridiag_resident_body(tasks, ntask, (int)blockIdx.x, status, sm);
}

// Pivot inverses and Householder reductions in one cooperative launch: CTAs
// [0, inv_ctas) work on the inverses, the rest on the reductions.  The two
// kinds of teams share nothing, so blocks of both kinds advance together on
// disjoint SMs (the inverses of a batch's super-nodes do not depend on its
// compression).
__global__ void __launch_bounds__(256, 1) resident_mix_kernel(const InvTask* __restrict__ inv, int ninv, int inv_ctas,
                                                              const EigTask* __restrict__ eig, int neig,
                                                              DeviceStatus* status) {
  extern __shared__ double sm[];
  const int b = (int)blockIdx.x;
  if (b < inv_ctas) invert_resident_body(inv, ninv, b, status, sm);
  else tridiag_resident_body(eig, neig, b - inv_ctas, status, sm);
}

// ---------------------------------------------------------------------------
// Compression spectrum.  M's right singular vectors and singular values are
// the eigenvectors and the square roots of the eigenvalues of G = M^T M:
//  1. Householder reduction G = Q T Q^T to tridiagonal T (reflector k kept in
//     rows k+1.. of column k; its product with a trailing vector uses symmetry,
//     p_i = column_i . v);
//  2. every eigenvalue of T by multisection on Sturm counts (lambda_0 on one
//     warp, the others on groups of lanes) to an absolute width of 2 u ||T||
//     for the kept and reported ones, 1e-7 ||T|| for the rest;
//  3. eigenvectors of the r kept eigenvalues by inverse iteration on T
//     (tridiagonal LU with partial pivoting, two solves from a distinct
//     pseudo-random start), then orthonormalised in order, each against the
//     earlier vectors of its cluster (blocked Gram-Schmidt, orthonormalise());
//  4. back-transformation V = Q Z.
// ---------------------------------------------------------------------------
constexpr int kEigSmemMax = kEigClusterMin - 1;  // largest m whose G sits in shared memory
constexpr int kBisectIters = 64;
constexpr int kInverseIters = 2;

// Number of eigenvalues below x of the unit-norm symmetric tridiagonal (d, e),
// given ne2[i] = -e_i^2: the sign changes of the Sturm sequence of leading
// principal minors p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (p_0 = 1).  A zero
// p_i counts as the sign opposite to p_{i-1} (the pair is renormalised to
// (+-1, -+2^-1000) so the recurrence continues); every 8 steps the pair is
// rescaled by an exact power of two.  Three FP64 operations per step; signs,
// zero tests and exponents are read from the bit patterns.
__device__ __forceinline__ unsigned sign_bit(double v) {
  return (unsigned)((unsigned long long)__double_as_longlong(v) >> 63);
}
__device__ __forceinline__ bool is_zero(double v) { return (__double_as_longlong(v) << 1) == 0; }

__device__ int sturm_count(const double* d, const double* ne2, int m, double x) {
  double pp = 1.0, p = d[0] - x;
  unsigned sp = 0, s;
  if (is_zero(p)) {
    s = 1;
    p = -0x1p-1000;
  } else {
    s = sign_bit(p);
  }
  int cnt = (int)(s != sp);
  for (int i = 1; i < m; ++i) {
    double pn = fma(d[i] - x, p, ne2[i - 1] * pp);
    unsigned sn;
    if (is_zero(pn)) {
      sn = s ^ 1u;
      pp = s ? -1.0 : 1.0;
      pn = s ? 0x1p-1000 : -0x1p-1000;
    } else {
      sn = sign_bit(pn);
      pp = p;
    }
    cnt += (int)(sn != s);
    p = pn;
    s = sn;
    if ((i & 7) == 0) {
      const long long bp = __double_as_longlong(fabs(p)), bq = __double_as_longlong(fabs(pp));
      int ex = (int)(((bp > bq ? bp : bq) >> 52) & 0x7ff) - 1023;
      if (ex > 400 || ex < -400) {
        ex = max(-1000, min(1000, ex));
        const double f = __longlong_as_double((long long)(1023 - ex) << 52);   // 2^-ex, exact
        p *= f;
        pp *= f;
      }
    }
  }
  return cnt;
}


// Eigenvalue number idx (ascending) by multisection: each of the 32 threads of
// warp 0 counts at one of 32 interior points, so the bracket shrinks 33-fold
// per round.  Every thread of the CTA must call it; returns the same value in all.
__device__ double multisect(const double* d, const double* ne2, int m, int idx, double lo, double hi, double tol,
                            int* s_first, double* s_ab) {
  const int tid = threadIdx.x;
  if (tid == 0) { s_ab[0] = lo; s_ab[1] = hi; }
  __syncthreads();
  if (tid < 32) {
    for (int round = 0; round < 16; ++round) {
      const double a = s_ab[0], b = s_ab[1];
      if (!(b - a > tol)) break;
      const double x = a + (b - a) * (double)(tid + 1) / 33.0;
      const unsigned above = __ballot_sync(0xffffffffu, sturm_count(d, ne2, m, x) > idx);
      const int t = above ? __ffs(above) - 1 : 32;            // first point with count > idx
      if (tid == 0) {
        s_ab[0] = (t == 0) ? a : a + (b - a) * (double)t / 33.0;
        s_ab[1] = (t == 32) ? b : a + (b - a) * (double)(t + 1) / 33.0;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  const double v = 0.5 * (s_ab[0] + s_ab[1]);
  __syncthreads();
  (void)s_first;
  return v;
}

__device__ __forceinline__ double start_entry(int j, int i) {
  unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(j * 7919 + i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Inverse iteration for one eigenvalue (run by one thread): x <- (T - shift)^{-1} x,
// scaled.  Six work arrays of m doubles in `scratch`, element i at [i * S].
__device__ void inverse_iteration(const double* d, const double* e, int m, double shift, double tnorm, int j,
                                  double* scratch, size_t S, double* out) {
  double* dl = scratch;
  double* dd = dl + (size_t)m * S;
  double* du = dd + (size_t)m * S;
  double* du2 = du + (size_t)m * S;
  double* x = du2 + (size_t)m * S;
  double* swp = x + (size_t)m * S;                   // 1.0 where rows i, i+1 were interchanged
  for (int i = 0; i < m; ++i) {
    dd[i * S] = d[i] - shift;
    if (i + 1 < m) { dl[i * S] = e[i]; du[i * S] = e[i]; }
  }
  for (int i = 0; i + 1 < m; ++i) {
    const double ddi = dd[i * S], dli = dl[i * S];
    if (fabs(ddi) >= fabs(dli)) {
      swp[i * S] = 0.0;
      const double f = ddi != 0.0 ? dli / ddi : 0.0;
      dl[i * S] = f;
      dd[(i + 1) * S] -= f * du[i * S];
      if (i + 2 < m) du2[i * S] = 0.0;
    } else {
      swp[i * S] = 1.0;
      const double f = ddi / dli;
      dd[i * S] = dli;
      dl[i * S] = f;
      const double tmp = du[i * S];
      const double dn = dd[(i + 1) * S];
      du[i * S] = dn;
      dd[(i + 1) * S] = tmp - f * dn;
      if (i + 2 < m) {
        const double un = du[(i + 1) * S];
        du2[i * S] = un;
        du[(i + 1) * S] = -f * un;
      }
    }
  }
  const double tiny = fmax(2.220446049250313e-16 * tnorm, 1e-300);
  for (int i = 0; i < m; ++i) {                        // keep 1 / pivot (tiny pivots perturbed)
    const double v = dd[i * S];
    dd[i * S] = 1.0 / ((fabs(v) < tiny) ? ((v < 0.0) ? -tiny : tiny) : v);
  }
  for (int i = 0; i < m; ++i) x[i * S] = start_entry(j, i);
  for (int it = 0; it < kInverseIters; ++it) {
    double xi = x[0];
    for (int i = 0; i + 1 < m; ++i) {
      const double xn = x[(i + 1) * S];
      if (swp[i * S] == 0.0) {
        x[i * S] = xi;
        xi = xn - dl[i * S] * xi;
      } else {
        x[i * S] = xn;
        xi = xi - dl[i * S] * xn;
      }
    }
    x[(m - 1) * S] = xi;
    double x1 = x[(m - 1) * S] * dd[(m - 1) * S];
    x[(m - 1) * S] = x1;
    double x2 = 0.0;
    if (m >= 2) {
      x2 = x1;
      x1 = (x[(m - 2) * S] - du[(m - 2) * S] * x2) * dd[(m - 2) * S];
      x[(m - 2) * S] = x1;
    }
    for (int i = m - 3; i >= 0; --i) {
      const double xv = (x[i * S] - du[i * S] * x1 - du2[i * S] * x2) * dd[i * S];
      x[i * S] = xv;
      x2 = x1;
      x1 = xv;
    }
    double mx = 0.0;
    for (int i = 0; i < m; ++i) mx = fmax(mx, fabs(x[i * S]));
    const double sc = mx > 0.0 ? 1.0 / mx : 1.0;
    for (int i = 0; i < m; ++i) x[i * S] *= sc;
  }
  for (int i = 0; i < m; ++i) out[i] = x[i * S];
}

// Classical Gram-Schmidt, twice, of z_j (j0 <= j < j1) against z_c0 .. z_{j-1},
// then normalisation; one vector at a time.  cvec: global (>= m doubles);
// normpart: global (>= team size doubles); cv: shared (>= m doubles).
template <int C>
__device__ void gram_schmidt_each(const Team<C>& team, double* Z, int m, int c0, int j0, int j1, double* cvec,
                                  double* normpart, double* cv, double* red) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int j = j0; j < j1; ++j) {
    double* zj = Z + (size_t)j * m;
    for (int pass = 0; pass < 2 && j > c0; ++pass) {
      for (int i = c0 + team.gwarp(); i < j; i += team.nwarps()) {
        const double* zi = Z + (size_t)i * m;
        double s = 0.0;
        for (int q = lane; q < m; q += 32) s = fma(zi[q], zj[q], s);
        s = warp_sum(s);
        if (lane == 0) cvec[i - c0] = s;
      }
      team.sync();
      for (int i = tid; i < j - c0; i += 256) cv[i] = cvec[i];
      __syncthreads();
      for (int q = team.gthread(); q < m; q += team.nthreads()) {
        double v = zj[q];
        for (int i = c0; i < j; ++i) v = fma(-cv[i - c0], Z[q + (size_t)i * m], v);
        zj[q] = v;
      }
      team.sync();
    }
    double s = 0.0;
    for (int q = team.gthread(); q < m; q += team.nthreads()) s = fma(zj[q], zj[q], s);
    s = block_sum(s, red);
    if constexpr (C != 1) {
      if (tid == 0) normpart[team.rank] = s;
      team.sync();
      s = 0.0;
      for (int c = 0; c < team.size; ++c) s += normpart[c];
    }
    const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int q = team.gthread(); q < m; q += team.nthreads()) zj[q] *= inv;
    team.sync();
  }
}

// Orthonormalisation of the kept eigenvectors Z (m x rank), in order, each
// against the earlier vectors of its cluster (runs of eigenvalues closer than
// gap_tol): the Gram-Schmidt basis of each cluster, computed in blocks of
// kGsBlock vectors.  A block is projected against the cluster's earlier
// vectors (C = Z_prev^T B, B -= Z_prev C) and then orthonormalised within
// itself by a Cholesky factorisation of its Gram matrix (S = B^T B = L L^T,
// B <- B L^-T); both steps twice.  When a pivot of the Cholesky factorisation
// is below kGsWeak times its diagonal entry (a vector almost inside the span
// of the ones before it) the block is redone one vector at a time.  Cg: global
// scratch of kGsBlock (m + kGsBlock) doubles (C, then S).  Every CTA of the
// team factors S alike.
constexpr double kGsWeak = 1e-10;

template <int C>
__device__ void orthonormalise(const Team<C>& team, double* Z, int m, int rank, const double* lam, double gap_tol,
                               double* Cg, double* cv, double* red) {
  constexpr int B = kGsBlock;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = (warp * team.size + team.rank) * 32 + lane;     // warps dealt to the CTAs in turn
  double* Sg = Cg + (size_t)B * m;
  __shared__ double sL[B * B];
  __shared__ double sdinv[B];
  __shared__ double s_rmin;
  __shared__ int s_weak;
  int c0 = 0;
  for (int j0 = 0; j0 < rank;) {
    if (j0 > 0 && lam[j0 - 1] - lam[j0] >= gap_tol) c0 = j0;
    int j1 = j0 + 1;
    while (j1 < rank && j1 - j0 < B && lam[j1 - 1] - lam[j1] < gap_tol) ++j1;
    const int nb = j1 - j0, np = j0 - c0;
    double* Bk = Z + (size_t)j0 * m;
    const double* Zp = Z + (size_t)c0 * m;
    // projection passes (classical Gram-Schmidt against the cluster's earlier
    // vectors) and Cholesky QR passes, each repeated only when needed: a
    // second projection when it removed more than half of a vector's squared
    // norm (the block's vectors have unit norm before it: "twice is enough"),
    // a second Cholesky QR when some pivot left under a quarter of its
    // column's squared norm (then one pass leaves orthogonality ~ kappa^2 u)
    int proj = 0, chol = 0;
    bool project = np > 0;
    for (int round = 0; round < 4; ++round) {
      if (tid == 0) s_weak = 0;
      if (project) {
        // C(i, jj) = z_i . b_jj: one warp per earlier vector i
        for (int i = team.gwarp(); i < np; i += team.nwarps()) {
          const double* zi = Zp + (size_t)i * m;
          double acc[B];
#pragma unroll
          for (int jj = 0; jj < B; ++jj) acc[jj] = 0.0;
          for (int q = lane; q < m; q += 32) {
            const double z = zi[q];
#pragma unroll
            for (int jj = 0; jj < B; ++jj)
              if (jj < nb) acc[jj] = fma(z, Bk[q + (size_t)jj * m], acc[jj]);
          }
#pragma unroll
          for (int jj = 0; jj < B; ++jj)
            if (jj < nb) {
              const double sj = warp_sum(acc[jj]);
              if (lane == 0) Cg[(size_t)i * B + jj] = sj;
            }
        }
        team.sync();
        // b_jj -= sum_i C(i, jj) z_i: one thread per (jj, row)
        for (int u = g; u < nb * m; u += team.nthreads()) {
          const int jj = u / m, q = u - jj * m;
          double v = Bk[q + (size_t)jj * m];
          for (int i = 0; i < np; ++i) v = fma(-Cg[(size_t)i * B + jj], Zp[q + (size_t)i * m], v);
          Bk[q + (size_t)jj * m] = v;
        }
        team.sync();
        ++proj;
      }
      // S = B^T B, lower triangle: one warp per entry
      for (int e = team.gwarp(); e < nb * (nb + 1) / 2; e += team.nwarps()) {
        int a = 0;
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        const int b = e - a * (a + 1) / 2;
        const double* xa = Bk + (size_t)a * m;
        const double* xb = Bk + (size_t)b * m;
        double sv = 0.0;
        for (int q = lane; q < m; q += 32) sv = fma(xa[q], xb[q], sv);
        sv = warp_sum(sv);
        if (lane == 0) Sg[a * B + b] = sv;
      }
      team.sync();
      if (project && proj == 1) {
        double smin = 1.0;
        for (int jj = 0; jj < nb; ++jj) smin = fmin(smin, Sg[jj * B + jj]);
        if (!(smin >= 0.5)) continue;               // project once more (every CTA decides alike)
      }
      project = false;
      // S = L L^T by columns on warp 0 (lane i holds row i of L)
      if (warp == 0) {
        double Lrow[B];
        double rmin = 1.0;
#pragma unroll
        for (int p = 0; p < B; ++p) Lrow[p] = 0.0;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (k >= nb) break;
          double sk = (lane >= k && lane < nb) ? Sg[lane * B + k] : 0.0;
#pragma unroll
          for (int p = 0; p < k; ++p) sk = fma(-Lrow[p], __shfl_sync(0xffffffffu, Lrow[p], k), sk);
          const double piv = __shfl_sync(0xffffffffu, sk, k);
          const double skk = Sg[k * B + k];
          const bool ok = piv > 0.0 && piv <= 1.7976931348623157e308;
          if (lane == 0 && !(piv > kGsWeak * skk)) s_weak = 1;
          rmin = fmin(rmin, ok ? piv / skk : 0.0);
          const double dk = ok ? sqrt(piv) : 0.0;
          const double di = ok ? 1.0 / dk : 0.0;
          if (lane == k) { Lrow[k] = dk; sdinv[k] = di; }
          else if (lane > k && lane < nb) Lrow[k] = sk * di;
        }
        if (lane < nb)
#pragma unroll
          for (int p = 0; p < B; ++p) sL[lane * B + p] = Lrow[p];
        if (lane == 0) s_rmin = rmin;
      }
      __syncthreads();
      if (s_weak) {
        // a column almost inside the span of the ones before it: Gram-Schmidt
        // one vector at a time for this block instead (every CTA decides alike)
        gram_schmidt_each(team, Z, m, c0, j0, j1, Cg, Sg, cv, red);
        break;
      }
      // B <- B L^-T: forward substitution along each row (one thread per row)
      for (int q = g; q < m; q += team.nthreads()) {
        double y[B];
#pragma unroll
        for (int jj = 0; jj < B; ++jj) {
          if (jj >= nb) break;
          double v = Bk[q + (size_t)jj * m];
#pragma unroll
          for (int p = 0; p < jj; ++p) v = fma(-y[p], sL[jj * B + p], v);
          y[jj] = v * sdinv[jj];
          Bk[q + (size_t)jj * m] = y[jj];
        }
      }
      team.sync();
      ++chol;
      if (!(chol == 1 && s_rmin < 0.25)) break;      // else a second Cholesky QR pass
    }
    j0 = j1;
  }
}

template <int C>
__global__ void __launch_bounds__(256) eig_kernel(const EigTask* __restrict__ tasks, DeviceStatus* status,
                                                  int smem_m, int ntask) {
  extern __shared__ double sm[];
  int ti = 0;
  if constexpr (C == kSubTeam) {
    __shared__ int s_task;
    if (threadIdx.x == 0) {
      int k = 0;
      while (k + 1 < ntask && tasks[k + 1].team0 <= (int)blockIdx.x) ++k;
      s_task = k;
    }
    __syncthreads();
    ti = s_task;
  } else {
    ti = task_index<C>();
  }
  const EigTask t = tasks[ti];
  Team<C> team;
  if constexpr (C == kSubTeam) team = Team<C>((int)blockIdx.x - t.team0, t.team_size, t.bar, status);
  const int m = t.m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ double red[8];
  __shared__ double s_lo, s_hi, s_emax;
  __shared__ double wlo[8], whi[8], wem[8];
  if (m == 0) {
    if (tid == 0 && team.rank == 0) *t.rank = 0;
    return;
  }
  double* d = sm;                  // diagonal of T
  double* e = d + m;               // sub-diagonal of T
  double* beta = e + m;            // reflector scalars
  double* lam = beta + m;          // eigenvalues, largest first
  double* wv = lam + m;            // w of the reduction
  double* cv = wv + m;             // p (one CTA) / Gram-Schmidt coefficients
  double* ds = cv + m;             // T scaled to unit norm: diagonal
  double* e2s = ds + m;            // and minus the squared off-diagonal
  double* Gs = e2s + m;
  // global scratch of the cluster form
  double* pg = t.W;                // p
  double* cg_ = t.W + m;           // Gram-Schmidt coefficients and block Gram matrix
  double* inv_scratch = t.W + m + (size_t)kGsBlock * (m + kGsBlock);
  const bool in_smem = (C == 1) && m <= smem_m;

  const int ld = in_smem ? (m | 1) : m;
  double* G = in_smem ? Gs : t.G;
  double* pvec = (C == 1) ? cv : pg;
  // reduced already (the resident kernel): T and the reflectors come from the slots
  const bool pre = (C != 1) && t.H != nullptr;
  const size_t lh = pre ? (size_t)m + 4 : (size_t)ld;
  const double* hv = pre ? t.H : G;               // reflector k at hv + k lh, rows k+1..
  // G's lower triangle is the data; the upper one is filled from it (exactly symmetric)
  if (pre) {
  } else if (in_smem) {
    for (int j = warp; j < m; j += 8)
      for (int i = lane; i < m; i += 32) {
        const double v = (i >= j) ? t.G[i + (size_t)j * m] : t.G[j + (size_t)i * m];
        Gs[i + j * ld] = v;
      }
  } else {
    for (int j = warp; j < m; j += 8) {
      if (!team.owns(j)) continue;
      for (int i = lane; i < j; i += 32) G[i + (size_t)j * ld] = G[j + (size_t)i * ld];
    }
    team.sync();
  }
  __syncthreads();
  long long clk = clock64();
  unsigned long long wall = global_ns();
  auto phase = [&](int ph) {                 // per-phase SM cycles, sampled by thread 0
    if (tid == 0) {
      const long long now = clock64();
      atomicAdd(&status->eig_cycles[ph], (unsigned long long)(now - clk));
      clk = now;
      if (C != 1 && team.rank == 0) {        // wall time on a large block's first CTA
        const unsigned long long w = global_ns();
        atomicAdd(&status->eig_lead_ns[ph], w - wall);
        wall = w;
      }
    }
  };

  // ---- 1. Householder tridiagonalisation
  if (pre) {
    for (int k = tid; k < m; k += 256) {
      const double* slot = t.H + (size_t)k * lh;
      d[k] = slot[m];
      e[k] = slot[m + 1];
      beta[k] = slot[m + 2];
    }
  }
  for (int k = 0; !pre && k + 2 < m; ++k) {
    double* colk = G + (size_t)k * ld;
    const Reflector rf = make_reflector(colk, k, m, red);
    const double dk = colk[k], bk = rf.beta;
    team.sync();                                   // column k read by every CTA
    if (tid == 0) {
      d[k] = dk;
      e[k] = rf.alpha;
      beta[k] = bk;
      if (team.rank == 0) colk[k + 1] = rf.v0;
    }
    if (rf.sh != 0 && team.rank == 0)              // the reflector is kept in column k
      for (int i = k + 2 + tid; i < m; i += 256) colk[i] = ldexp(colk[i], rf.sh);
    team.sync();
    if (bk == 0.0) continue;
    // p_i = bk * column_i . v over own trailing columns
    for (int i = k + 1 + warp; i < m; i += 8) {
      if (!team.owns(i)) continue;
      const double* ci = G + (size_t)i * ld;
      double s = 0.0;
      for (int j = k + 1 + lane; j < m; j += 32) s = fma(ci[j], colk[j], s);
      s = warp_sum(s);
      if (lane == 0) pvec[i] = bk * s;
    }
    team.sync();
    double pv = 0.0;
    for (int i = k + 1 + tid; i < m; i += 256) pv = fma(pvec[i], colk[i], pv);
    const double K = 0.5 * bk * block_sum(pv, red);
    for (int i = k + 1 + tid; i < m; i += 256) wv[i] = fma(-K, colk[i], pvec[i]);
    __syncthreads();
    // own trailing columns: B -= v w^T + w v^T
    for (int j = k + 1 + warp; j < m; j += 8) {
      if (!team.owns(j)) continue;
      const double vj = colk[j], wj = wv[j];
      double* cj = G + (size_t)j * ld;
      for (int i = k + 1 + lane; i < m; i += 32) cj[i] = fma(-colk[i], wj, fma(-wv[i], vj, cj[i]));
    }
    team.sync();
  }
  if (tid == 0 && !pre) {
    if (m >= 2) {
      d[m - 2] = G[(m - 2) + (size_t)(m - 2) * ld];
      e[m - 2] = G[(m - 1) + (size_t)(m - 2) * ld];
      beta[m - 2] = 0.0;
    }
    d[m - 1] = G[(m - 1) + (size_t)(m - 1) * ld];
    e[m - 1] = 0.0;
    beta[m - 1] = 0.0;
  }
  __syncthreads();

  phase(0);
  // ---- 2. eigenvalues by bisection
  // (fmin / fmax drop NaN operands: a non-finite T is detected separately)
  double lo = 1e308, hi = -1e308, emax = 0.0;
  bool t_bad = false;
  for (int i = tid; i < m; i += 256) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
    t_bad |= !(fabs(d[i]) + r <= 1.7976931348623157e308);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i + 1 < m) emax = fmax(emax, e[i] * e[i]);
  }
  if (__syncthreads_or(t_bad) && tid == 0 && team.rank == 0) atomicExch(&status->numeric, 1);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, off));
  }
  if (lane == 0) { wlo[warp] = lo; whi[warp] = hi; wem[warp] = emax; }
  __syncthreads();
  if (tid == 0) {
    double a0 = wlo[0], b0 = whi[0], c0 = wem[0];
    for (int w = 1; w < 8; ++w) { a0 = fmin(a0, wlo[w]); b0 = fmax(b0, whi[w]); c0 = fmax(c0, wem[w]); }
    s_lo = a0; s_hi = b0; s_emax = c0;
  }
  __syncthreads();
  const double tnorm = fmax(fabs(s_lo), fabs(s_hi));
  // work on T scaled by a power of two to unit norm (exact), with e^2 precomputed
  const double sc = (tnorm > 0.0 && tnorm <= 1.7976931348623157e308) ? ldexp(1.0, -ilogb(tnorm)) : 1.0;
  for (int i = tid; i < m; i += 256) {
    ds[i] = d[i] * sc;
    e2s[i] = (i + 1 < m) ? -(e[i] * sc) * (e[i] * sc) : 0.0;   // -e_i^2
  }
  __syncthreads();
  const double los = s_lo * sc, his = s_hi * sc;
  const double abstol = 2.0 * 2.220446049250313e-16 * fmax(fabs(los), fabs(his));
  const double coarse = 1e-7 * fmax(fabs(los), fabs(his));
  const double lo0 = los - abstol, hi0 = his + abstol;
  // the largest eigenvalue first (thread 0 of every CTA, alike), then the rank by
  // one Sturm count at the threshold: #{lambda >= x} = m - count(x); eigenvalues
  // that are kept or reported (sigma >= 1e-3 sigma_0) get full accuracy, the rest
  // a coarse bisection (absolute 1e-7 ||T||)
  __shared__ double s_l0, s_ab[2];
  __shared__ int s_rank2, s_nacc, s_first;
  const double l0m = multisect(ds, e2s, m, m - 1, lo0, hi0, abstol, &s_first, s_ab);
  // eq. curOff6 sums the tail of the spectrum: every eigenvalue at full
  // accuracy, the rank decided after the bisection
  const bool frob = t.trunc_rule == 1;
  if (tid == 0) {
    const double l0 = l0m;
    const int nsv = min(t.rho, m);
    int r = 0;
    if (!frob && nsv > 0 && l0 > 0.0) {
      if (t.eps == 0.0) r = nsv;
      else {
        // lambda_k >= eps^2 lambda_0, and never a zero eigenvalue (the
        // threshold stays above zero if eps^2 lambda_0 underflows)
        const double thr = fmax(t.eps * t.eps * l0, 4.9406564584124654e-324);
        r = min(nsv, m - sturm_count(ds, e2s, m, thr));
      }
    }
    s_l0 = l0;
    s_rank2 = r;
  }
  if (tid == 32) s_nacc = (frob || !(l0m > 0.0)) ? m : m - sturm_count(ds, e2s, m, 1e-6 * l0m);
  __syncthreads();
  if (tid == 0) s_nacc = max(s_nacc, s_rank2);
  __syncthreads();
  const double l0 = s_l0;
  const int nacc = s_nacc;
  int rank = s_rank2;
  // every other eigenvalue by multisection on a group of L lanes: each round
  // the L lanes count at L interior points, so the bracket shrinks (L+1)-fold
  // for the cost of one Sturm count (a warp instruction costs the same for
  // any number of active lanes).  L: the largest power of two up to 32 with
  // the groups filling at most a quarter of the team's threads; warps are
  // dealt to the team's CTAs in turn.
  {
    int L = 1;
    while (L < 32 && (size_t)m * 2 * L <= (size_t)team.nthreads() / 4) L *= 2;
    const int per_warp = 32 / L, grp = lane / L, sub = lane % L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
    const int wg = warp * team.size + team.rank;
    for (int base = wg * per_warp; base < m; base += team.nwarps() * per_warp) {
      const int k = base + grp;                     // descending: k = 0 is lambda_0
      const bool valid = k > 0 && k < m;
      const int idx = m - 1 - k;
      const double tol = k < nacc ? abstol : coarse;
      double a = lo0, b = hi0;
      for (int round = 0; round < kBisectIters; ++round) {
        const bool active = valid && b - a > tol;
        if (!__any_sync(0xffffffffu, active)) break;
        const double x = a + (b - a) * (double)(sub + 1) / (double)(L + 1);
        const bool above = active && sturm_count(ds, e2s, m, x) > idx;
        const unsigned g = (__ballot_sync(0xffffffffu, above) >> (grp * L)) & gmask;
        const int first = g ? __ffs(g) - 1 : L;     // first point with count > idx
        if (active) {
          const double na = (first == 0) ? a : a + (b - a) * (double)first / (double)(L + 1);
          const double nb = (first == L) ? b : a + (b - a) * (double)(first + 1) / (double)(L + 1);
          a = na;
          b = nb;
        }
      }
      if (sub == 0 && k < m) t.sigma[k] = ((k == 0) ? l0 : 0.5 * (a + b)) / sc;   // eigenvalue for now
    }
  }
  team.sync();
  for (int k = tid; k < m; k += 256) lam[k] = t.sigma[k];
  team.sync();
  if (frob) {
    // eq. curOff6: r = the smallest k with sum_{j >= k} sigma_j^2 < (eps N)^2,
    // N^2 = ||all levels below||_F^2; the tail is summed from the smallest
    // singular value up (no cancellation).  Every CTA of the team decides
    // alike from the same eigenvalues.
    if (tid == 0) {
      const int nsv = min(t.rho, m);
      const double bnd = t.eps * sqrt(fmax(*t.below_sq, 0.0));
      const double b2 = bnd * bnd;
      int r = nsv;
      if (b2 > 0.0) {
        double tail = 0.0;
        for (int k = nsv - 1; k >= 0; --k) {
          tail += fmax(lam[k], 0.0) * t.gram_scale;
          if (tail < b2) r = k;
          else break;
        }
      }
      s_rank2 = r;
    }
    __syncthreads();
    rank = s_rank2;
  }
  if (team.rank == 0)
    for (int k = tid; k < m; k += 256) t.sigma[k] = sqrt(fmax(lam[k], 0.0) * t.gram_scale);
  if (tid == 0 && team.rank == 0) {
    *t.rank = rank;
    if (!(tnorm <= 1.7976931348623157e308)) atomicExch(&status->numeric, 1);
    atomicAdd(&status->eig_flops, (unsigned long long)(2.0 * m * (double)m * m + 4.0 * m * (double)rank * rank +
                                                       2.0 * m * (double)m * rank));
  }
  __syncthreads();
  phase(1);
  if (rank == 0) return;                            // same decision in every CTA

  // ---- 3. inverse iteration, one thread per kept eigenvector; warps are dealt
  // to the team's CTAs in turn so that the work spreads over all of them
  double* Z = t.V;                                  // m x rank, leading dimension m
  {
    // the work arrays of the team's threads interleaved (element i of thread
    // g at i S + g), so that a warp's accesses are coalesced; the threads that
    // take a vector have g < min(team threads, rank) <= S
    const int g = (warp * team.size + team.rank) * 32 + lane;
    const size_t S = (size_t)min(team.nthreads(), m);
    for (int j = g; j < rank; j += team.nthreads())
      inverse_iteration(d, e, m, lam[j], tnorm, j, inv_scratch + g, S, Z + (size_t)j * m);
  }
  team.sync();
  phase(2);
  // normalise every vector (one warp each); then orthonormalise them in order,
  // each only against the earlier vectors of its cluster.  Inverse-iteration
  // vectors of eigenvalues a gap g apart are orthogonal to ~u ||T|| / g on their
  // own, so for eps > 0 a cluster is a run of eigenvalues closer than
  // 1e-4 lambda_0 (leaving < 3e-12 non-orthogonality); at eps = 0 (exact
  // factorisation) every vector is orthogonalised against all earlier ones
  for (int j = team.gwarp(); j < rank; j += team.nwarps()) {
    double* zj = Z + (size_t)j * m;
    double s = 0.0;
    for (int q = lane; q < m; q += 32) s = fma(zj[q], zj[q], s);
    s = warp_sum(s);
    const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (int q = lane; q < m; q += 32) zj[q] *= inv;
  }
  team.sync();
  const double gap_tol = t.eps > 0.0 ? 1e-4 * lam[0] : 1.7976931348623157e308;
  orthonormalise(team, Z, m, rank, lam, gap_tol, cg_, cv, red);
  phase(3);
  // ---- 4. V = Q Z with Q = H_0 H_1 ... H_{m-3}: apply H_{m-3} first, in
  // blocks of 8 reflectors a_p = k_hi - p (applied in the order p = 0, 1, ..).
  // Applying H_{a_0} .. H_{a_{p-1}} before H_{a_p} changes v_p^T z by
  // -sum_{l<p} s_l v_p^T v_l, so with the block's Gram c_pl = v_p^T v_l (l < p,
  // rows > a_l; the same for every column, formed first by the team) one pass
  // over a column gives the eight dots d_p = v_p^T z, then s_p = beta_p (d_p -
  // sum_{l<p} s_l c_pl), and a second pass z -= sum_p s_p v_p: the same
  // arithmetic per column, one pass and one batched warp reduction per eight
  // reflectors instead of per reflector.
  constexpr int RB = 8, RT = RB * (RB - 1) / 2;
  const int nblk = (m - 2 + RB - 1) / RB;                  // reflectors 0 .. m-3
  double* cgram = cg_;                                     // free after the Gram-Schmidt
  for (int e2 = team.gwarp(); e2 < nblk * RT; e2 += team.nwarps()) {
    const int q = e2 / RT, w = e2 % RT;
    int p = 1;
    while ((p + 1) * p / 2 <= w) ++p;                      // w = p (p - 1) / 2 + l, l < p
    const int l = w - p * (p - 1) / 2;
    const int khi = m - 3 - RB * q, ap = khi - p, al = khi - l;
    double sdot = 0.0;
    if (ap >= 0) {
      const double* vp = hv + (size_t)ap * lh;
      const double* vl = hv + (size_t)al * lh;
      for (int i = al + 1 + lane; i < m; i += 32) sdot = fma(vp[i], vl[i], sdot);
    }
    sdot = warp_sum(sdot);
    if (lane == 0) cgram[e2] = sdot;
  }
  team.sync();
  for (int col = team.gwarp(); col < rank; col += team.nwarps()) {
    double* zc = Z + (size_t)col * m;
    for (int q = 0; q < nblk; ++q) {
      const int khi = m - 3 - RB * q, n = min(RB, khi + 1);
      const int i0 = khi - n + 2;                          // first row any reflector of the block touches
      double dp[RB];
#pragma unroll
      for (int p = 0; p < RB; ++p) dp[p] = 0.0;
      for (int i = i0 + lane; i < m; i += 32) {
        const double z = zc[i];
#pragma unroll
        for (int p = 0; p < RB; ++p)
          if (p < n && i > khi - p) dp[p] = fma(hv[(size_t)(khi - p) * lh + i], z, dp[p]);
      }
      double sp[RB];
#pragma unroll
      for (int p = 0; p < RB; ++p) dp[p] = warp_sum(dp[p]);
      const double* cq = cgram + (size_t)q * RT;
#pragma unroll
      for (int p = 0; p < RB; ++p) {
        double v = dp[p];
#pragma unroll
        for (int l = 0; l < p; ++l) v = fma(-sp[l], cq[p * (p - 1) / 2 + l], v);
        sp[p] = (p < n) ? beta[khi - p] * v : 0.0;
      }
      for (int i = i0 + lane; i < m; i += 32) {
        double z = zc[i];
#pragma unroll
        for (int p = 0; p < RB; ++p)
          if (p < n && i > khi - p) z = fma(-sp[p], hv[(size_t)(khi - p) * lh + i], z);
        zc[i] = z;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  phase(4);
}

template <class... KArgs, class... Args>
cudaError_t launch_team(void (*kernel)(KArgs...), TeamKind kind, int ctas, size_t smem, cudaStream_t st,
                        Args... args) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (kind == TeamKind::Cluster) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kDenseCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  } else if (kind == TeamKind::Grid || kind == TeamKind::Sub) {
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

int co_resident_ctas(const void* kernel, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess) per_sm = 1;
  return std::max(1, sms * std::max(per_sm, 1));
}

}  // namespace

size_t eig_smem(int m) { return (size_t)8 * m * sizeof(double) + 64; }
size_t inv_smem(int m) { return (size_t)m * (2 * sizeof(double) + 2 * sizeof(int)) + 64; }

int grid_team_size(int m, bool eig) {
  // the inverse: one 16-column chunk per CTA at least; the spectrum: one CTA
  // per SM (its later phases spread rows, eigenvalues and vectors over all);
  // never more than can be co-resident
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int want = eig ? std::max(sms, 1) : std::max(8, (m + 15) / 16);
  const int cap = eig ? co_resident_ctas((const void*)eig_kernel<kGridTeam>, eig_smem(m))
                      : co_resident_ctas((const void*)invert_kernel<kGridTeam>, inv_smem(m));
  return std::min({want, cap, kMaxTeam});
}

cudaError_t launch_invert(const InvTask* tasks, int ntask, int max_m, TeamKind kind, int team,
                          DeviceStatus* status, cudaStream_t st) {
  if (ntask <= 0) return cudaSuccess;
  const size_t smem = inv_smem(max_m);
  if (kind == TeamKind::Grid) return launch_team(invert_kernel<kGridTeam>, kind, team, smem, st, tasks, status);
  if (kind == TeamKind::Cluster)
    return launch_team(invert_kernel<kDenseCluster>, kind, ntask * kDenseCluster, smem, st, tasks, status);
  return launch_team(invert_kernel<1>, kind, ntask, smem, st, tasks, status);
}

namespace {
int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}
// shared memory of a resident CTA holding cw columns of a block of size m
size_t resident_smem(int m, int cw, bool eig) {
  return ((size_t)cw * m + (eig ? 2 * (size_t)m : 2 * (size_t)m + cw)) * sizeof(double);
}
// most columns a resident CTA can hold
int resident_cw_max(int m, bool eig) {
  const size_t cap = kResidentSmemMax / sizeof(double);
  const size_t extra = 2 * (size_t)m;
  if (cap <= extra + 1) return 0;
  return (int)std::min<size_t>((cap - extra) / ((size_t)m + (eig ? 0 : 1)), (size_t)m);
}
}  // namespace

size_t inv_resident_workspace(int m) { return (size_t)m * m + m + 8; }
size_t tridiag_resident_workspace(int m) { return (size_t)m * (m + 4) + (size_t)m * m + 2 * (size_t)m + 8; }

static bool fits_on(int m, bool eig, int sms) {
  if (m < 1) return false;
  const int cw = resident_cw_max(m, eig);
  return cw >= 1 && (m + cw - 1) / cw <= sms;
}

bool resident_fits(int m, bool eig) { return fits_on(m, eig, device_sms()); }

std::vector<std::pair<int, int>> plan_resident_waves(const int* m, int n, bool eig, int* cta0, int* cw, int sms) {
  std::vector<char> kinds((size_t)n, eig ? 1 : 0);
  return plan_mixed_waves(m, kinds.data(), n, cta0, cw, sms);
}

std::vector<std::pair<int, int>> plan_mixed_waves(const int* m, const char* eigs, int n, int* cta0, int* cw,
                                                  int sms) {
  std::vector<std::pair<int, int>> waves;
  if (sms <= 0) sms = device_sms();
  for (int i = 0; i < n; ++i)
    if (!fits_on(m[i], eigs[i], sms)) return {};
  int b = 0;
  while (b < n) {
    // the most blocks whose smallest teams fit on the SMs together
    int e = b, need = 0;
    while (e < n) {
      const int cmax = resident_cw_max(m[e], eigs[e]);
      const int p = (m[e] + cmax - 1) / cmax;
      if (e > b && need + p > sms) break;
      need += p;
      ++e;
    }
    // share the SMs in proportion to the blocks' work (m^3), at least the smallest team each
    double work = 0.0;
    for (int i = b; i < e; ++i) work += (double)m[i] * m[i] * m[i];
    int next = 0;
    for (int i = b; i < e; ++i) {
      const int cmax = resident_cw_max(m[i], eigs[i]);
      const int pmin = (m[i] + cmax - 1) / cmax;
      const int want = (int)((double)sms * m[i] * m[i] * m[i] / work);
      int p = std::min(std::max(pmin, want), m[i]);
      const int rest_min = [&] {
        int r = 0;
        for (int j = i + 1; j < e; ++j) {
          const int cj = resident_cw_max(m[j], eigs[j]);
          r += (m[j] + cj - 1) / cj;
        }
        return r;
      }();
      p = std::max(pmin, std::min(p, sms - next - rest_min));
      const int c = (m[i] + p - 1) / p;
      cw[i] = c;
      cta0[i] = next;
      next += (m[i] + c - 1) / c;
    }
    waves.emplace_back(b, e);
    b = e;
  }
  return waves;
}

template <class T>
static int wave_layout(const T* h, int n, bool eig, size_t* smem) {
  int ctas = 0;
  *smem = 0;
  for (int i = 0; i < n; ++i) {
    ctas = std::max(ctas, h[i].cta0 + (h[i].m + h[i].cw - 1) / h[i].cw);
    *smem = std::max(*smem, resident_smem(h[i].m, h[i].cw, eig));
  }
  return ctas;
}

cudaError_t launch_invert_resident(const InvTask* d_tasks, const InvTask* h_tasks, int n, DeviceStatus* status,
                                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  size_t smem = 0;
  const int ctas = wave_layout(h_tasks, n, false, &smem);
  if (smem > kResidentSmemMax || ctas > co_resident_ctas((const void*)invert_resident_kernel, smem))
    return cudaErrorCooperativeLaunchTooLarge;
  for (int i = 0; i < n; ++i) {
    const InvTask& t = h_tasks[i];
    cudaError_t e = cudaMemsetAsync(t.W + (size_t)t.m * t.m, 0, (size_t)(t.m + 1) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  return launch_team(invert_resident_kernel, TeamKind::Grid, ctas, smem, st, d_tasks, n, status);
}

cudaError_t launch_tridiag_resident(const EigTask* d_tasks, const EigTask* h_tasks, int n, DeviceStatus* status,
                                    cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  size_t smem = 0;
  const int ctas = wave_layout(h_tasks, n, true, &smem);
  if (smem > kResidentSmemMax || ctas > co_resident_ctas((const void*)tridiag_resident_kernel, smem))
    return cudaErrorCooperativeLaunchTooLarge;
  for (int i = 0; i < n; ++i) {
    const EigTask& t = h_tasks[i];
    if (t.H == nullptr) return cudaErrorInvalidValue;
    double* flags = t.H + (size_t)t.m * (t.m + 4) + (size_t)t.m * t.m;
    cudaError_t e = cudaMemsetAsync(flags, 0, (2 * (size_t)t.m + 1) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  return launch_team(tridiag_resident_kernel, TeamKind::Grid, ctas, smem, st, d_tasks, n, status);
}

cudaError_t launch_resident_mix(const InvTask* d_inv, const InvTask* h_inv, int ninv, const EigTask* d_eig,
                                const EigTask* h_eig, int neig, DeviceStatus* status, cudaStream_t st) {
  if (ninv <= 0) return launch_tridiag_resident(d_eig, h_eig, neig, status, st);
  if (neig <= 0) return launch_invert_resident(d_inv, h_inv, ninv, status, st);
  size_t smem_i = 0, smem_e = 0;
  const int ci = wave_layout(h_inv, ninv, false, &smem_i);
  const int ce = wave_layout(h_eig, neig, true, &smem_e);
  const size_t smem = std::max(smem_i, smem_e);
  if (smem > kResidentSmemMax || ci + ce > co_resident_ctas((const void*)resident_mix_kernel, smem))
    return cudaErrorCooperativeLaunchTooLarge;
  for (int i = 0; i < ninv; ++i) {
    const InvTask& t = h_inv[i];
    cudaError_t e = cudaMemsetAsync(t.W + (size_t)t.m * t.m, 0, (size_t)(t.m + 1) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  for (int i = 0; i < neig; ++i) {
    const EigTask& t = h_eig[i];
    if (t.H == nullptr) return cudaErrorInvalidValue;
    double* flags = t.H + (size_t)t.m * (t.m + 4) + (size_t)t.m * t.m;
    cudaError_t e = cudaMemsetAsync(flags, 0, (2 * (size_t)t.m + 1) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  return launch_team(resident_mix_kernel, TeamKind::Grid, ci + ce, smem, st, d_inv, ninv, ci, d_eig, neig, status);
}

int sub_team_capacity(int max_m) {
  return std::min(co_resident_ctas((const void*)eig_kernel<kSubTeam>, eig_smem(max_m)), 2 * device_sms());
}

std::vector<std::pair<int, int>> plan_sub_teams(const int* m, int n, int capacity, int* team0, int* size) {
  std::vector<std::pair<int, int>> waves;
  capacity = std::max(capacity, 1);
  int b = 0;
  while (b < n) {
    const int e = std::min(n, b + capacity);                // at least one CTA per block
    double work = 0.0;
    for (int i = b; i < e; ++i) work += (double)m[i] * m[i] * m[i];
    int next = 0;
    for (int i = b; i < e; ++i) {
      const int rest = e - i - 1;                           // later blocks keep one CTA each
      int p = (int)((double)capacity * m[i] * m[i] * m[i] / work);
      p = std::max(1, std::min({p, kMaxTeam, capacity - next - rest}));
      team0[i] = next;
      size[i] = p;
      next += p;
    }
    waves.emplace_back(b, e);
    b = e;
  }
  return waves;
}

namespace {
// A wait on a flag that nothing sets: await_flag must give up after its time
// limit, set status->wait_timeout and the abort word, and return 0.
__global__ void bounded_wait_selftest_kernel(unsigned long long* words, DeviceStatus* status) {
  if (threadIdx.x == 0) words[2] = await_flag(&words[0], &words[1], status);
}
}  // namespace

cudaError_t launch_bounded_wait_selftest(unsigned long long* words, DeviceStatus* status, cudaStream_t st) {
  bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(words, status);
  return cudaGetLastError();
}

cudaError_t launch_eig(const EigTask* tasks, int ntask, int max_m, TeamKind kind, int team, DeviceStatus* status,
                       cudaStream_t st) {
  if (ntask <= 0) return cudaSuccess;
  const size_t base = eig_smem(max_m);
  if (kind == TeamKind::Grid) return launch_team(eig_kernel<kGridTeam>, kind, team, base, st, tasks, status, 0, ntask);
  if (kind == TeamKind::Sub) return launch_team(eig_kernel<kSubTeam>, kind, team, base, st, tasks, status, 0, ntask);
  if (kind == TeamKind::Cluster)
    return launch_team(eig_kernel<kDenseCluster>, kind, ntask * kDenseCluster, base, st, tasks, status, 0, ntask);
  int smem_m = std::min(max_m, kEigSmemMax);
  size_t smem = base + (size_t)(smem_m | 1) * (smem_m | 1) * sizeof(double);
  if (smem > 227 * 1024) {
    smem_m = 0;
    smem = base;
  }
  return launch_team(eig_kernel<1>, kind, ntask, smem, st, tasks, status, smem_m, ntask);
}

}  // namespace lrs
