// tc_gemm.cu -- the precision form's gather GEMM on the fifth-generation
// tensor cores (sm_103a tcgen05): the block products of Algorithm 1 -- Schur
// updates A_qk -= A_qp (A_pp^{-1} A_pk) and the products A_pp^{-1} A_pk
// (Sec. 2.2), the projections R_k = A_k V, Q_k^T = V^T B_k^T and the Gram
// matrices of the stacked well-separated blocks (Sec. 4.3, eq. lra) -- with
// TF32 operands and FP32 accumulation in tensor memory.
//
// Each operand x (an FP64 block entry) is truncated to FP32 (in integer
// instructions: the FP64 pipe is the scarce one on this chip) and split into
// a TF32 head h = rna_tf32(x) and a TF32 tail l = rna_tf32(x - h); a product
// is formed as h_a h_b + h_a l_b + l_a h_b (the truncation, the tail's
// rounding and the dropped l_a l_b are each at most about 2^-21 |a b|), close
// to FP32 accuracy at three tensor-core products.  Accumulation is FP32 in
// tensor memory over all terms and K chunks of a tile in a fixed order
// (deterministic); the epilogue adds the sum to the block's FP64 value rounded
// to FP32 and writes the FP32 result back as FP64, all in FP32 and integer
// instructions (GB300 issues two FP64 operations per clock per SM, which would
// bound a tile with a short contraction).  The block values are then FP32
// accurate, below the products' own error.
//
// One CTA per 128 x 128 output tile (the tile's rows are the 128 lanes of the
// accumulator, its columns 128 tensor-memory columns), two CTAs per SM.  Eight
// warps stage K chunks of 16 into shared memory (FP64 loads, split, 16-byte stores in the
// tensor core's K-major core-matrix layout, no swizzle); one thread issues the
// tcgen05.mma instructions of a chunk and commits them to the chunk buffer's
// mbarrier, so the warps stage chunk c + 1 into the other buffer while the
// tensor core works on chunk c.  Every wait on an mbarrier is bounded.
#include <cstdint>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace lrs {
namespace {

constexpr int TM = kTcTile, TN = kTcTile;  // output tile
constexpr int KC = 16;                     // K chunk per pipeline stage
constexpr int KS = 8;                      // K of one kind::tf32 MMA (32 bytes)
constexpr int kThreads = 256;
constexpr int kSlab = 128 * KS * 4;        // bytes of one K step of a 128-row operand part
constexpr int kPart = (KC / KS) * kSlab;   // one operand part (head or tail) of a stage: 8 KB
constexpr int kStage = 4 * kPart;          // A head, A tail, B head, B tail: 32 KB
constexpr int kStages = 2;
constexpr int kCtasPerSm = 2;              // co-resident CTAs hide each other's staging latency
constexpr int kTmemCols = 128;             // FP32 accumulator: 128 lanes x TN columns

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N / 8 at bits 17-22,
// M / 16 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

using tc::mbar_wait;
using tc::smem_desc;
using tc::smem_u32;

// FP64 -> FP32 by truncation of the significand, in integer instructions (the
// FP64 pipe, ~2 operations per clock per SM on this chip, stays free): error
// below 2^-23 relative; magnitudes under FP32's normal range become zero,
// over it infinity (NaN stays NaN).
__device__ __forceinline__ float f64_to_f32_trunc(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FF) - (1023 - 127);
  const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  uint32_t bits;
  const bool nan = ((hi >> 20) & 0x7FF) == 0x7FF && ((hi & 0xFFFFFu) | lo);
  if (e <= 0) bits = sign;
  else if (e >= 255) bits = sign | 0x7F800000u | (nan ? 0x400000u : 0u);
  else bits = sign | ((uint32_t)e << 23) | mant;
  return __uint_as_float(bits);
}

// FP64 -> FP32 rounded to nearest (ties to even), in integer instructions;
// magnitudes under FP32's normal range become zero, over it infinity.
__device__ __forceinline__ float f64_to_f32_rn(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FF) - (1023 - 127);
  const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  if (e <= 0) return __uint_as_float(sign);
  const bool nan = ((hi >> 20) & 0x7FF) == 0x7FF && ((hi & 0xFFFFFu) | lo);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u));
  uint32_t bits = ((uint32_t)e << 23) | mant;
  const uint32_t rest = lo & 0x1FFFFFFFu, half = 0x10000000u;   // the 29 dropped bits
  if (rest > half || (rest == half && (bits & 1u))) ++bits;       // a carry may reach the exponent (or infinity)
  return __uint_as_float(sign | bits);
}

// FP32 -> FP64, exact, in integer instructions (FP32 subnormals become zero).
__device__ __forceinline__ double f32_to_f64_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t sign = b & 0x80000000u, e = (b >> 23) & 0xFFu, mant = b & 0x7FFFFFu;
  unsigned long long out;
  if (e == 0) out = (unsigned long long)sign << 32;
  else if (e == 255) out = (unsigned long long)(sign | 0x7FF00000u | (mant ? 0x80000u : 0u)) << 32;
  else out = ((unsigned long long)(sign | ((e + (1023 - 127)) << 20) | (mant >> 3)) << 32) |
             ((unsigned long long)(mant & 7u) << 29);
  return __longlong_as_double((long long)out);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return h;
}

// Stages a 128-row x KC operand chunk (KC / 8 (row, k-quad) items per
// thread): element (r, k) of op(X) is P[r + k ld]
// (kcontig == false) or P[k + r ld] (kcontig == true); rows >= rv and k >= kv
// are zero.  Head and tail parts go to hd and tl in the K-major core-matrix
// layout: byte offset of (r, k) = (k / 8) kSlab + (r / 8) 256 + ((k / 4) % 2)
// 128 + (r % 8) 16 + (k % 4) 4; each thread stores 4 consecutive k at once.
__device__ __forceinline__ void stage_operand(const double* __restrict__ P, int ld, bool kcontig, int rv, int kv,
                                              uint8_t* hd, uint8_t* tl, int tid) {
  constexpr int NI = KC / 8;                         // (row, k-quad) items per thread
  constexpr int NQ = KC / 4;                         // k-quads per row
  double v[NI][4];
  int rr[NI], kq[NI];
#pragma unroll
  for (int p = 0; p < NI; ++p) {
    const int q = tid + kThreads * p;
    int r, g;
    if (!kcontig) { r = q & 127; g = q >> 7; }          // a warp: 32 consecutive rows, one k-quad
    else { r = (q & 7) + 8 * (q / (8 * NQ)); g = (q >> 3) % NQ; }
    rr[p] = r;
    kq[p] = g;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 4 * g + e;
      double x = 0.0;
      if (r < rv && k < kv) x = kcontig ? P[k + (size_t)r * ld] : P[r + (size_t)k * ld];
      v[p][e] = x;
    }
  }
#pragma unroll
  for (int p = 0; p < NI; ++p) {
    const int r = rr[p], g = kq[p];
    const uint32_t off = (uint32_t)((g >> 1) * kSlab + (r >> 3) * 256 + (g & 1) * 128 + (r & 7) * 16);
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float xf = f64_to_f32_trunc(v[p][e]);
      h[e] = tf32_rna(xf);
      l[e] = tf32_rna(xf - __uint_as_float(h[e]));
    }
    *reinterpret_cast<uint4*>(hd + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(tl + off) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    gemm_tc_kernel(const GemmTask* __restrict__ tasks, const GemmTerm* __restrict__ terms, DeviceStatus* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kStages * kStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + kStages);
  __shared__ int s_abort;

  const GemmTask t = tasks[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = t.ti * TM, col0 = t.tj * TN;
  const int m = min(TM, t.rows - row0), n = min(TN, t.cols - col0);

  int total = 0;                                       // K chunks over all terms
  for (int it = 0; it < t.nterm; ++it) total += (terms[t.term0 + it].k + KC - 1) / KC;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    for (int b = 0; b < kStages; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  // chunk cursor: term index and K offset of the next chunk to stage
  int cur_term = 0, cur_k0 = 0;
  auto stage = [&](int buf) {
    while (cur_term < t.nterm && cur_k0 >= terms[t.term0 + cur_term].k) { ++cur_term; cur_k0 = 0; }
    const GemmTerm g = terms[t.term0 + cur_term];
    const bool ta = g.trans & 1, tb = (g.trans >> 1) & 1;
    const int kv = min(KC, g.k - cur_k0);
    uint8_t* base = smem + buf * kStage;
    // op(A) rows row0.., K from cur_k0; op(B)^T rows (columns of op(B)) col0..
    const double* A = ta ? g.A + (size_t)row0 * g.lda + cur_k0 : g.A + row0 + (size_t)cur_k0 * g.lda;
    const double* B = tb ? g.B + col0 + (size_t)cur_k0 * g.ldb : g.B + (size_t)col0 * g.ldb + cur_k0;
    stage_operand(A, g.lda, ta, m, kv, base, base + kPart, tid);
    stage_operand(B, g.ldb, !tb, n, kv, base + 2 * kPart, base + 3 * kPart, tid);
    cur_k0 += KC;
    return kv;
  };

  bool ok = true;
  if (total > 0) {
    int kv = stage(0);
    for (int c = 0; c < total; ++c) {
      const int buf = c & 1;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staged data -> tensor core's view
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a_hd = smem_u32(smem + buf * kStage), a_tl = a_hd + kPart;
        const uint32_t b_hd = a_hd + 2 * kPart, b_tl = a_hd + 3 * kPart;
        const int steps = (kv + KS - 1) / KS;
        for (int s = 0; s < steps; ++s) {
          const uint32_t o = s * kSlab;
          const uint64_t ah = smem_desc(a_hd + o), al = smem_desc(a_tl + o);
          const uint64_t bh = smem_desc(b_hd + o), bl = smem_desc(b_tl + o);
          const uint64_t pa[3] = {ah, ah, al}, pb[3] = {bh, bl, bh};
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {
            const uint32_t acc = (c > 0 || s > 0 || pr > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                "l"(pa[pr]), "l"(pb[pr]), "r"(kIdesc), "r"(acc));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(mbar + buf)));
      }
      if (c + 1 < total) {
        const int nb = (c + 1) & 1;
        // buffer nb was read by the MMAs of chunk c - 1 (commit (c - 1) / 2 on its barrier)
        if (c >= 1 && !mbar_wait(smem_u32(mbar + nb), (uint32_t)(((c - 1) >> 1) & 1))) s_abort = 1;
        __syncthreads();
        if (s_abort) { ok = false; break; }             // uniform: every thread read the same flag
        kv = stage(nb);
      }
    }
    // the last commit covers every MMA issued before it
    const uint32_t last = smem_u32(mbar + ((total - 1) & 1)), lpar = (uint32_t)(((total - 1) >> 1) & 1);
    if (ok && !mbar_wait(last, lpar)) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      ok = false;
      mbar_wait(last, lpar);                            // once more (bounded) before the TMEM is freed
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok) {
    if (status) atomicExch(&status->wait_timeout, 1);
  } else {
    // epilogue: warp w reads lanes 32 (w % 4).. (its rows) and columns 64 (w / 4)..,
    // 16 columns at a time
    const int q = warp & 3, h = warp >> 2;
    const int i = 32 * q + lane;
    const float sign = (t.mode & kSubtract) ? -1.0f : 1.0f;
    double* C = t.C + row0 + i + (size_t)col0 * t.ldc;
    const double* D = t.D ? t.D + row0 + i + (size_t)col0 * t.ldd : nullptr;
#pragma unroll 1
    for (int c4 = 0; c4 < 4; ++c4) {
      uint32_t r[16];
      if (total > 0) {
        const uint32_t a = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * h + 16 * c4);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(a));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) r[e] = 0u;
      }
      if (i < m) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int j = 64 * h + 16 * c4 + e;
          if (j < n) {
            double init = 0.0;
            if (D) init = D[(size_t)j * t.ldd];
            else if (t.mode & kAccumulate) init = C[(size_t)j * t.ldc];
            // FP32 arithmetic on the FP32-rounded init: the products carry ~1e-6
            // relative error already, and FP64 operations would bound the tile
            C[(size_t)j * t.ldc] = f32_to_f64_exact(fmaf(sign, __uint_as_float(r[e]), f64_to_f32_rn(init)));
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace

size_t gemm_tc_smem_bytes() { return (size_t)kStages * kStage + 64; }

cudaError_t launch_gemm_tc(const GemmTask* tasks, int ntask, const GemmTerm* terms, DeviceStatus* status,
                           cudaStream_t st) {
  if (ntask <= 0) return cudaSuccess;
  const int smem = (int)gemm_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  gemm_tc_kernel<<<ntask, kThreads, smem, st>>>(tasks, terms, status);
  return cudaGetLastError();
}

}  // namespace lrs
