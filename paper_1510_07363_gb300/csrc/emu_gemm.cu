// emu_gemm.cu -- the FP64 form's gather GEMM with FP64 products emulated on
// the fifth-generation tensor cores (sm_103a tcgen05, kind::f16 with BF16
// operands): the block products of Algorithm 1 -- Schur updates A_qk -= A_qp
// (A_pp^{-1} A_pk) and the products A_pp^{-1} A_pk (Sec. 2.2), the
// projections R_k = A_k V, Q_k^T = V^T B_k^T and the Gram matrices of the
// stacked well-separated blocks (Sec. 4.3, eq. lra).
//
// GB300 issues two FP64 FMAs per clock per SM; its BF16 tensor cores do about
// 1800 multiply-adds per clock per SM.  The FP64 products are formed by
// Ozaki's error-free splitting scheme on integer slices:
//  - per K chunk of 64, every row i of op(A) gets the largest biased exponent
//    E_i of its entries, and every entry becomes the signed fixed-point
//    integer N = a 2^(1078 - E_i), rounded to nearest (|N| <= 2^56: the
//    row's largest entry keeps all 53 bits, a smaller one the bits above 2^-56
//    of the row's scale), written as eight balanced digits N = sum_s d_s
//    2^(49 - 7 s) with d_0 in [-128, 128] and d_1..d_7 in [-64, 63] -- each
//    exactly a BF16 number; the columns of op(B) likewise with exponents F_j;
//  - the digit products with s + t <= 7 (36 BF16 MMAs per K step) are summed
//    per diagonal d = s + t in eight FP32 accumulators in tensor memory.  A
//    diagonal sums at most 64 x 2 products of magnitude <= 2^13 (pairs with
//    d_0) and 64 x 6 of <= 2^12, so every partial sum is an integer of
//    magnitude at most 2^22 and the FP32 accumulation is exact;
//  - at the end of the chunk the eight accumulators are read back as integers
//    and combined into X = sum_d acc_d 2^(49 - 7 d), the chunk's product in
//    units of 2^(E_i + F_j - 2107) (|X| < 2^69.02), which is rounded to
//    units of 2^cut, cut = 7 + ceil(log2(chunks of the tile)), and added to a
//    running 64-bit integer sum per output (below 2^63 whatever the signs).
//    The running sums keep the largest exponents seen so far (R_i, R_j); a
//    chunk with smaller exponents is shifted into them, a larger one shifts
//    the sum first;
//  - the epilogue converts the sum to FP64 once: C = init + sign sum
//    2^(R_i + R_j - 2107 + cut).
// Error per chunk, against max_k |a_ik| max_k |b_kj|: the rounding of the
// operands (half a unit of 2^-56 of their row's or column's scale, at most
// 2^-49 for the two over 64 products), the dropped diagonals s + t >= 8 (at
// most about 2^-47, and of either sign) and the rounding to 2^cut (at most
// 2^(cut - 62)): below 2^-45 in all for up to 512 chunks, under the worst-case rounding error of an FP64 dot
// product of length 64 (2^-41 of the same); on well-scaled data the error is
// that of FP64.  The order of every operation is fixed, so results are
// deterministic.  Entries that are not finite make their row's or column's
// outputs NaN.
//
// One CTA per 128 x 64 output tile (rows = the 128 lanes of tensor memory;
// the eight diagonal accumulators fill its 512 columns), one CTA per SM.
// Eight warps load a chunk's FP64 operands into registers, agree on the
// exponents through shared memory and write the digits of one K step (16)
// at a time into a two-stage buffer in the tensor core's K-major layout;
// one thread issues the 36 MMAs of a K step and commits them to the stage's
// mbarrier, so the warps split step q + 1 while the tensor core runs step q.
// The next chunk's loads are issued before the chunk's last MMAs are waited
// for.  Every wait on an mbarrier is bounded.
#include <cstdint>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace lrs {
namespace {

using tc::mbar_wait;
using tc::smem_desc;
using tc::smem_u32;

constexpr int EM = kEmuTileM;                  // 128 rows
constexpr int EN = kEmuTileN;                  // 64 columns
constexpr int EK = kEmuChunk;                  // 64: K chunk with one exponent per row / column
constexpr int ES = 8;                          // digits (slices) of 7 bits
constexpr int EKS = 16;                        // K of one kind::f16 MMA
constexpr int ESUB = EK / EKS;                 // K steps per chunk
constexpr int kThreads = 256;
constexpr int kAPart = EM * EKS * 2;           // one digit slice of A for one K step: 4 KB
constexpr int kBPart = EN * EKS * 2;           // of B: 2 KB
constexpr int kStage = ES * (kAPart + kBPart);  // 48 KB
constexpr int kStages = 2;
constexpr int kTmemCols = ES * EN;             // eight FP32 accumulators of 128 x 64
constexpr int kAccOff = kStages * kStage;      // int64 running sums, column-major 128 x 64
constexpr int kBarOff = kAccOff + EM * EN * 8;
constexpr int kSmem = kBarOff + 64;

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, N / 8 at bits 17-22, M / 16 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(EN >> 3) << 17) |
                            ((uint32_t)(EM >> 4) << 24);

// Biased exponent of x as the fixed-point scale sees it: 1 for subnormals, 0
// for zero and for non-finite entries (flagged separately).
__device__ __forceinline__ int scale_exponent(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  if (e == 0x7FF) return 0;
  if (e == 0) return (u << 1) ? 1 : 0;
  return e;
}
__device__ __forceinline__ bool not_finite(double x) {
  return (((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF;
}

// The signed fixed-point value N = x 2^(1078 - er), rounded to nearest (er
// >= the entry's exponent, so |N| <= 2^56), offset by kBias (64 in each of the
// seven lower digit positions) and returned as N + kBias = hi 2^28 + lo, hi
// signed, lo in [0, 2^28).
constexpr long long kBias = 64ll * ((1ll << 42) + (1ll << 35) + (1ll << 28) + (1ll << 21) + (1ll << 14) + (1ll << 7) + 1);
__device__ __forceinline__ void fixed_point(double x, int er, int& hi, uint32_t& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
  const unsigned long long m56 = (e ? (mant | (1ull << 52)) : mant) << 3;
  const int sh = er - (e ? e : 1);
  unsigned long long U;
  if (e == 0x7FF || sh < 0 || sh > 56) U = 0ull;
  else if (sh == 0) U = m56;
  else U = (m56 + (1ull << (sh - 1))) >> sh;
  const long long N = ((u >> 63) ? -(long long)U : (long long)U) + kBias;
  hi = (int)(N >> 28);
  lo = (uint32_t)((unsigned long long)N & 0xFFFFFFFull);
}

// The eight balanced digits of N = (hi 2^28 + lo) - kBias: N = sum_s d_s
// 2^(49 - 7 s) with d_0 = hi >> 21 in [-128, 128] and, for s >= 1, d_s = (the
// s-th 7-bit field) - 64 in [-64, 63].  Balanced digits make the dropped
// products (s + t >= 8) as likely negative as positive.  Each digit is
// returned as the FP32 value d_s (exact: 1.5 2^23 + field is exact in FP32, so
// is the subtraction), whose upper 16 bits are its BF16 encoding.
__device__ __forceinline__ void digits(int hi, uint32_t lo, uint32_t f[ES]) {
  const uint32_t fld[ES] = {0u, (uint32_t)(hi >> 14) & 127u, (uint32_t)(hi >> 7) & 127u, (uint32_t)hi & 127u,
                            lo >> 21, (lo >> 14) & 127u, (lo >> 7) & 127u, lo & 127u};
  f[0] = __float_as_uint(__int_as_float(0x4B400000 + (hi >> 21)) - 12582912.0f);
#pragma unroll
  for (int s = 1; s < ES; ++s) f[s] = __float_as_uint(__int_as_float(0x4B400000 + (int)fld[s]) - 12582976.0f);
}
// two digits (FP32 words) as one BF16 pair: the low half holds the first
__device__ __forceinline__ uint32_t pack2(uint32_t f0, uint32_t f1) { return __byte_perm(f0, f1, 0x7632); }

// An FP32 accumulator as an integer: the sums are integers of magnitude at
// most 2^22, and 1.5 2^23 + v is then exact in FP32.
__device__ __forceinline__ int acc_int(uint32_t v) {
  return __float_as_int(__uint_as_float(v) + 12582912.0f) - 0x4B400000;
}

// x >> s (arithmetic) for any s >= 0
__device__ __forceinline__ long long sra(long long x, int s) { return x >> (s < 63 ? s : 63); }

__global__ void __launch_bounds__(kThreads, 1)
    gemm_emu_kernel(const GemmTask* __restrict__ tasks, const GemmTerm* __restrict__ terms, DeviceStatus* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  long long* accs = reinterpret_cast<long long*>(smem + kAccOff);     // (i, j) at j * EM + i
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kBarOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + kStages);
  __shared__ int sPa[2][EM], sPb[4][EN];       // per-thread partial exponents of a chunk
  __shared__ int sEa[EM], sEb[EN];             // the chunk's exponents
  __shared__ int sRa[EM], sRb[EN];             // exponents of the running sums
  __shared__ int sBadA[EM], sBadB[EN];
  __shared__ int s_abort;

  const GemmTask t = tasks[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = t.ti * EM, col0 = t.tj * EN;
  const int m = min(EM, t.rows - row0), n = min(EN, t.cols - col0);

  int total = 0;                                       // K chunks over all terms
  for (int it = 0; it < t.nterm; ++it) total += (terms[t.term0 + it].k + EK - 1) / EK;
  // low bits cut from each chunk's product: |X| < 2^69.02 per chunk, so the
  // running sums of `total` chunks stay below 2^63 with 7 + ceil(log2 total)
  const int cut = 7 + (total > 1 ? 32 - __clz(total - 1) : 0);

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
  for (int e = tid; e < EM * EN; e += kThreads) accs[e] = 0;
  if (tid < EM) { sRa[tid] = 0; sBadA[tid] = 0; }
  if (tid < EN) { sRb[tid] = 0; sBadB[tid] = 0; }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  // operand registers of one chunk: A row ra, K offsets 16 q + 8 oa + e;
  // B column jb, K offsets 16 q + 4 ob + e
  const int ra = tid & (EM - 1), oa = tid >> 7;
  const int jb = tid & (EN - 1), ob = tid >> 6;
  double av[ESUB][8], bv[ESUB][4];
  int cur_term = 0, cur_k0 = 0;
  auto load = [&]() {
    while (cur_term < t.nterm && cur_k0 >= terms[t.term0 + cur_term].k) { ++cur_term; cur_k0 = 0; }
    const GemmTerm g = terms[t.term0 + cur_term];
    const bool ta = g.trans & 1, tb = (g.trans >> 1) & 1;
    const int kv = min(EK, g.k - cur_k0);
    const double* A = ta ? g.A + (size_t)row0 * g.lda + cur_k0 : g.A + row0 + (size_t)cur_k0 * g.lda;
    const double* B = tb ? g.B + col0 + (size_t)cur_k0 * g.ldb : g.B + (size_t)col0 * g.ldb + cur_k0;
#pragma unroll
    for (int q = 0; q < ESUB; ++q) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = EKS * q + 8 * oa + e;
        double x = 0.0;
        if (ra < m && k < kv) x = ta ? A[k + (size_t)ra * g.lda] : A[ra + (size_t)k * g.lda];
        av[q][e] = x;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = EKS * q + 4 * ob + e;
        double x = 0.0;
        if (jb < n && k < kv) x = tb ? B[jb + (size_t)k * g.ldb] : B[k + (size_t)jb * g.ldb];
        bv[q][e] = x;
      }
    }
    cur_k0 += EK;
  };

  bool ok = true;
  int step = 0;                                        // K steps issued so far (all chunks)
  if (total > 0) load();
  for (int c = 0; c < total && ok; ++c) {
    // ---- the chunk's exponents
    {
      int ea = 0, eb = 0;
      bool bad_a = false, bad_b = false;
#pragma unroll
      for (int q = 0; q < ESUB; ++q) {
#pragma unroll
        for (int e = 0; e < 8; ++e) { ea = max(ea, scale_exponent(av[q][e])); bad_a |= not_finite(av[q][e]); }
#pragma unroll
        for (int e = 0; e < 4; ++e) { eb = max(eb, scale_exponent(bv[q][e])); bad_b |= not_finite(bv[q][e]); }
      }
      sPa[oa][ra] = ea;
      sPb[ob][jb] = eb;
      if (bad_a) sBadA[ra] = 1;
      if (bad_b) sBadB[jb] = 1;
    }
    __syncthreads();
    if (tid < EM) sEa[tid] = max(sPa[0][tid], sPa[1][tid]);
    else if (tid < EM + EN) {
      const int j = tid - EM;
      sEb[j] = max(max(sPb[0][j], sPb[1][j]), max(sPb[2][j], sPb[3][j]));
    }
    __syncthreads();
    const int er = sEa[ra], ec = sEb[jb];
    // ---- K steps: digits into the stage buffer, then 36 MMAs
#pragma unroll
    for (int q = 0; q < ESUB; ++q, ++step) {
      const int buf = step & 1;
      // the buffer was read by the MMAs of step - 2 (commit (step - 2) / 2 on its barrier)
      if (step >= 2 && !mbar_wait(smem_u32(mbar + buf), (uint32_t)(((step - 2) >> 1) & 1))) s_abort = 1;
      __syncthreads();
      if (s_abort) { ok = false; break; }              // uniform: every thread read the same flag
      uint8_t* st = smem + buf * kStage;
      {
        uint32_t w[ES][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          int h0, h1;
          uint32_t l0, l1;
          fixed_point(av[q][e], er, h0, l0);
          fixed_point(av[q][e + 1], er, h1, l1);
          uint32_t d0[ES], d1[ES];
          digits(h0, l0, d0);
          digits(h1, l1, d1);
#pragma unroll
          for (int s = 0; s < ES; ++s) w[s][e >> 1] = pack2(d0[s], d1[s]);
        }
        const uint32_t off = (uint32_t)((ra >> 3) * 256 + oa * 128 + (ra & 7) * 16);
#pragma unroll
        for (int s = 0; s < ES; ++s)
          *reinterpret_cast<uint4*>(st + s * kAPart + off) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
      }
      {
        uint32_t w[ES][2];
#pragma unroll
        for (int e = 0; e < 4; e += 2) {
          int h0, h1;
          uint32_t l0, l1;
          fixed_point(bv[q][e], ec, h0, l0);
          fixed_point(bv[q][e + 1], ec, h1, l1);
          uint32_t d0[ES], d1[ES];
          digits(h0, l0, d0);
          digits(h1, l1, d1);
#pragma unroll
          for (int s = 0; s < ES; ++s) w[s][e >> 1] = pack2(d0[s], d1[s]);
        }
        const uint32_t off =
            (uint32_t)(ES * kAPart + (jb >> 3) * 256 + (ob >> 1) * 128 + (jb & 7) * 16 + (ob & 1) * 8);
#pragma unroll
        for (int s = 0; s < ES; ++s)
          *reinterpret_cast<uint2*>(st + s * kBPart + off) = make_uint2(w[s][0], w[s][1]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // digits -> the tensor core's view
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(st), b0 = a0 + ES * kAPart;
#pragma unroll
        for (int d = 0; d < ES; ++d)
#pragma unroll
          for (int s = 0; s <= d; ++s) {
            const uint64_t ad = smem_desc(a0 + s * kAPart), bd = smem_desc(b0 + (d - s) * kBPart);
            const uint32_t acc = (q > 0 || s > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)(d * EN)),
                "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(mbar + buf)));
      }
    }
    if (!ok) break;
    if (c + 1 < total) load();                         // the next chunk's loads overlap the last MMAs
    // ---- all MMAs of the chunk done (the last commit covers every earlier one)
    const int last = step - 1;
    if (!mbar_wait(smem_u32(mbar + (last & 1)), (uint32_t)((last >> 1) & 1))) s_abort = 1;
    __syncthreads();
    if (s_abort) { ok = false; break; }
    asm volatile("tcgen05.fence::after_thread_sync;");
    // ---- fold the eight diagonals into the running sums: warp w reads lanes
    // 32 (w % 4).. (its rows) and columns 32 (w / 4).. of every diagonal
    {
      const int i = 32 * (warp & 3) + lane, h = warp >> 2;
      const int r_old = sRa[i], e_row = sEa[i];
      const int r_new = max(r_old, e_row);
#pragma unroll 1
      for (int g4 = 0; g4 < 8; ++g4) {
        uint32_t v[ES][4];
#pragma unroll
        for (int d = 0; d < ES; ++d) {
          const uint32_t a = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(d * EN + 32 * h + 4 * g4);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                       : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3])
                       : "r"(a));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 32 * h + 4 * g4 + e;
          const int c_old = sRb[j], e_col = sEb[j];
          const int c_new = max(c_old, e_col);
          int a[ES];
#pragma unroll
          for (int d = 0; d < ES; ++d) a[d] = acc_int(v[d][e]);
          const long long H = (long long)a[0] * (1 << 21) + (long long)a[1] * (1 << 14) + a[2] * 128 + a[3];
          const long long L = (long long)a[4] * (1 << 21) + (long long)a[5] * (1 << 14) + a[6] * 128 + a[7];
          // X = H 2^28 + L rounded to units of 2^cut (2^28 is a multiple of 2^cut)
          const long long X = H * (1ll << (28 - cut)) + ((L + (1ll << (cut - 1))) >> cut);
          long long& sum = accs[j * EM + i];
          sum = sra(sum, (r_new - r_old) + (c_new - c_old)) + sra(X, (r_new - e_row) + (c_new - e_col));
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();                                   // tensor memory read before the next chunk's MMAs
    if (tid < EM) sRa[tid] = max(sRa[tid], sEa[tid]);
    else if (tid < EM + EN) sRb[tid - EM] = max(sRb[tid - EM], sEb[tid - EM]);
  }
  if (!ok && step > 0) {
    // wait (bounded) for the MMAs in flight before the tensor memory is freed
    const int last = step - 1;
    mbar_wait(smem_u32(mbar + (last & 1)), (uint32_t)((last >> 1) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (!ok) {
    if (status && tid == 0) atomicExch(&status->wait_timeout, 1);
  } else {
    // epilogue: C = init + sign * sum * 2^(R_i + R_j - 2107 + cut)
    const int i = 32 * (warp & 3) + lane, h = warp >> 2;
    if (i < m) {
      const int ri = sRa[i];
      const bool bad_i = sBadA[i] != 0;
      double* C = t.C + row0 + i + (size_t)col0 * t.ldc;
      const double* D = t.D ? t.D + row0 + i + (size_t)col0 * t.ldd : nullptr;
      for (int jj = 0; jj < 32; ++jj) {
        const int j = 32 * h + jj;
        if (j >= n) break;
        const long long sum = accs[j * EM + i];
        double v = sum ? ldexp((double)sum, ri + sRb[j] - 2107 + cut) : 0.0;
        if (bad_i || sBadB[j]) v = __longlong_as_double(0x7FF8000000000000ll);
        double init = 0.0;
        if (D) init = D[(size_t)j * t.ldd];
        else if (t.mode & kAccumulate) init = C[(size_t)j * t.ldc];
        C[(size_t)j * t.ldc] = (t.mode & kSubtract) ? init - v : init + v;
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace

int gemm_emu_chunks(const GemmTerm* terms, int nterm) {
  int c = 0;
  for (int i = 0; i < nterm; ++i) c += (terms[i].k + EK - 1) / EK;
  return c;
}

cudaError_t launch_gemm_emu(const GemmTask* tasks, int ntask, const GemmTerm* terms, DeviceStatus* status,
                            cudaStream_t st) {
  if (ntask <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(gemm_emu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  gemm_emu_kernel<<<ntask, kThreads, kSmem, st>>>(tasks, terms, status);
  return cudaGetLastError();
}

}  // namespace lrs
