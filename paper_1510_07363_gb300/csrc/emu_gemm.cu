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
//  - per group of eight K chunks of 64 (512 values of k), every row i of
//    op(A) gets the largest biased exponent E_i of its entries, and every
//    entry becomes the signed fixed-point integer N = a 2^(1077 - E_i),
//    rounded to nearest (|N| <= 2^55: the row's largest entry keeps all 53
//    bits, a smaller one the bits above 2^-55 of the row's scale), written as
//    eight balanced digits N = sum_s d_s 2^(49 - 7 s) with d_0 in [-64, 64] and
//    d_1..d_7 in [-64, 63] -- each exactly a BF16 number; the columns of
//    op(B) likewise with exponents F_j.  A split kernel does this once per
//    distinct operand of a launch, writing the digit slices in the tensor
//    core's K-major core-matrix layout, one 32 KB (A, 128 rows) or 16 KB (B,
//    64 columns) block per tile, K step of 16 and all eight slices;
//  - the product kernel copies those blocks into shared memory with bulk
//    copies (cp.async.bulk, completion on an mbarrier) and forms the 36 digit
//    products with s + t <= 7 per K step in twelve MMAs (tcgen05.mma
//    kind::f16, M = 128, K = 16, N = 64 to 256: A_s against up to four B
//    slices side by side), summed per diagonal d = s + t in eight FP32
//    accumulators in tensor memory over the whole group.  A digit product is
//    at most 2^12 in magnitude and a diagonal has at most eight digit pairs, so
//    it gains at most 2^21 per chunk and 2^24 per group: every partial sum is
//    an integer of magnitude at most 2^24 and the FP32 accumulation is exact;
//  - after a group the eight accumulators are read back as integers and
//    combined into X = sum_d acc_d 2^(49 - 7 d), the group's product in units
//    of 2^(E_i + F_j - 2105), which is rounded to units of 2^cut, cut = 5 +
//    ceil(log2(chunks of the tile)), and added to a running 64-bit integer
//    sum per output (below 2^63 whatever the signs).  The running sums keep
//    the largest exponents seen so far (R_i, R_j); a group with smaller
//    exponents is shifted into them, a larger one shifts the sum first;
//  - the epilogue converts the sum to FP64 once: C = init + sign sum
//    2^(R_i + R_j - 2105 + cut).
// Error per group, against max |a_ik| max |b_kj| over the group's k: the
// rounding of the operands (half a unit of 2^-55 of their row's or column's
// scale, at most 2^-45 for the two over 512 products), the dropped diagonals
// s + t >= 8 (at most 7 2^-45, and of either sign) and the rounding to 2^cut
// (at most 2^(cut - 60), 2^-46 for up to 512 chunks): below 2^-41.5 in all,
// under the worst-case rounding error of an FP64 dot product of length 512
// (2^-35 of the same); on well-scaled data the error is that of FP64.  A group
// whose row or column exponent lies below the running one is added at the
// running scale, and the running sum is shifted when the scale grows: each
// drops bits below one unit of 2^cut there, 2^(cut + R_i + R_j - 2105), at
// most 2^(cut - 59) of max_k |a_ik| max_k |b_kj| over the whole contraction.
// That is zero when every group holds its row's and its column's largest
// exponent, and it bounds a small output's relative accuracy when a row peaks
// in other groups than a column (normwise it stays at the level above).  The
// order of every operation is fixed, so results are deterministic.  Entries
// that are not finite make their row's or column's outputs NaN.
//
// One CTA per 128 x 64 output tile (rows = the 128 lanes of tensor memory;
// the eight diagonal accumulators fill its 512 columns), one CTA per SM, ten
// warps: warp 8 issues the bulk copies into a four-stage ring, warp 9 the
// MMAs (each K step's commit frees its stage; a group's last commit starts the
// recombination), warps 0-7 recombine (warp w reads lanes 32 (w % 4).. and
// columns 32 (w / 4).. of every diagonal) and write the tile.  The copies of
// the next group run while a group is recombined.  Every wait is bounded and
// also gives up once another role of the CTA has given up.
#include <cstdint>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace lrs {
namespace {

using tc::smem_desc;
using tc::smem_u32;

constexpr int EM = kEmuTileM;                  // 128 rows
constexpr int EN = kEmuTileN;                  // 64 columns
constexpr int EK = kEmuChunk;                  // 64: K chunk
constexpr int EG = kEmuGroup;                  // chunks per group (one exponent per row / column)
constexpr int ES = 8;                          // digits (slices) of 7 bits
constexpr int EKS = 16;                        // K of one kind::f16 MMA
constexpr int ESUB = EK / EKS;                 // K steps per chunk
constexpr int kAPart = EM * EKS * 2;           // one digit slice of A for one K step: 4 KB
constexpr int kBPart = EN * EKS * 2;           // of B: 2 KB
constexpr int kABlock = ES * kAPart;           // 32 KB: A's eight slices of one K step
constexpr int kBBlock = ES * kBPart;           // 16 KB
constexpr int kStage = kABlock + kBBlock;      // 48 KB
constexpr int kStages = 4;
constexpr int kTmemCols = ES * EN;             // eight FP32 accumulators of 128 x 64
constexpr int kFlushWarps = 8;
constexpr int kThreads = 32 * (kFlushWarps + 2);   // + the copy warp and the MMA warp
constexpr int kBarOff = kStages * kStage;
constexpr int kSmem = kBarOff + 128;

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, M / 16 at bits 24-28; N / 8 goes to
// bits 17-22 per MMA.
constexpr uint32_t kIdescBase = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(EM >> 4) << 24);

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

// The signed fixed-point value N = x 2^(1077 - er), rounded to nearest (er
// >= the entry's exponent, so |N| <= 2^55), offset by kBias (64 in each of the
// seven lower digit positions) and returned as N + kBias = hi 2^28 + lo, hi
// signed, lo in [0, 2^28).
constexpr long long kBias =
    64ll * ((1ll << 42) + (1ll << 35) + (1ll << 28) + (1ll << 21) + (1ll << 14) + (1ll << 7) + 1);
__device__ __forceinline__ void fixed_point(double x, int er, int& hi, uint32_t& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
  const unsigned long long m55 = (e ? (mant | (1ull << 52)) : mant) << 2;
  const int sh = er - (e ? e : 1);
  unsigned long long U;
  if (e == 0x7FF || sh < 0 || sh > 55) U = 0ull;
  else if (sh == 0) U = m55;
  else U = (m55 + (1ull << (sh - 1))) >> sh;
  const long long N = ((u >> 63) ? -(long long)U : (long long)U) + kBias;
  hi = (int)(N >> 28);
  lo = (uint32_t)((unsigned long long)N & 0xFFFFFFFull);
}

// The eight balanced digits of N = (hi 2^28 + lo) - kBias: N = sum_s d_s
// 2^(49 - 7 s) with d_0 = hi >> 21 in [-64, 64] and, for s >= 1, d_s = (the
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

// x >> s (arithmetic) for any s >= 0
__device__ __forceinline__ long long sra(long long x, int s) { return x >> (s < 63 ? s : 63); }

// ---------------------------------------------------------------------------
// Split kernel: one CTA per (operand, group of 512 k, block of 8 rows).  The
// block's FP64 values go through shared memory (loaded along whichever
// dimension is contiguous), every row's exponent is the largest over the
// group (a warp per row), and each (row, 8 consecutive k) becomes one 16-byte
// store per slice.
// ---------------------------------------------------------------------------
constexpr int kSplitRows = kEmuSplitRows, kSplitK = EG * EK;

__global__ void __launch_bounds__(256) emu_split_kernel(const EmuSplitTask* __restrict__ tasks, int ntask) {
  __shared__ double xs[kSplitRows][kSplitK + 1];
  __shared__ int sE[kSplitRows];
  const int bid = (int)blockIdx.x, tid = threadIdx.x;
  int lo = 0, hi = ntask - 1;                   // the task: the largest cta0 <= bid
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].cta0 <= bid) lo = mid;
    else hi = mid - 1;
  }
  const EmuSplitTask t = tasks[lo];
  const int nrb = t.rows_pad / kSplitRows;
  const int local = bid - t.cta0;
  const int g = local / nrb, r0 = (local % nrb) * kSplitRows, k0 = g * kSplitK;
  const int kv = min(kSplitK, t.k - k0);
  if (t.kcontig) {                              // op(X)(r, k) = P[k + r ld]: threads along k
    for (int e = tid; e < kSplitRows * kSplitK; e += 256) {
      const int kk = e % kSplitK, r = e / kSplitK;
      double x = 0.0;
      if (r0 + r < t.rows && kk < kv) x = t.P[(size_t)(k0 + kk) + (size_t)(r0 + r) * t.ld];
      xs[r][kk] = x;
    }
  } else {                                      // op(X)(r, k) = P[r + k ld]: threads along r
    for (int e = tid; e < kSplitRows * kSplitK; e += 256) {
      const int r = e % kSplitRows, kk = e / kSplitRows;
      double x = 0.0;
      if (r0 + r < t.rows && kk < kv) x = t.P[(size_t)(r0 + r) + (size_t)(k0 + kk) * t.ld];
      xs[r][kk] = x;
    }
  }
  __syncthreads();
  {
    // row r's exponent over the group: a warp per row
    const int r = tid >> 5, sub = tid & 31;
    int emax = 0;
    bool bad = false;
    for (int kk = sub; kk < kSplitK; kk += 32) {
      emax = max(emax, scale_exponent(xs[r][kk]));
      bad |= not_finite(xs[r][kk]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
      bad |= __shfl_xor_sync(0xffffffffu, (int)bad, off) != 0;
    }
    if (sub == 0) {
      sE[r] = emax;
      t.ex[(size_t)g * t.rows_pad + r0 + r] = emax;
      if (bad) atomicOr(&t.bad[r0 + r], 1);
    }
  }
  __syncthreads();
  // digits: item (r, o) holds k = 8 o .. 8 o + 7 of the group (chunk g EG + o / 8,
  // K step (o % 8) / 2, half o % 2 of the step)
  const int nch = (t.k + EK - 1) / EK, ntiles = t.rows_pad / t.tile;
  for (int it = tid; it < kSplitRows * (kSplitK / 8); it += 256) {
    const int r = it % kSplitRows, o = it / kSplitRows;
    const int c = g * EG + o / 8, q = (o % 8) >> 1, h = o & 1;
    if (c >= nch) continue;
    const int er = sE[r];
    uint32_t w[ES][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      int h0, h1;
      uint32_t l0, l1;
      fixed_point(xs[r][8 * o + e], er, h0, l0);
      fixed_point(xs[r][8 * o + e + 1], er, h1, l1);
      uint32_t d0[ES], d1[ES];
      digits(h0, l0, d0);
      digits(h1, l1, d1);
#pragma unroll
      for (int s = 0; s < ES; ++s) w[s][e >> 1] = pack2(d0[s], d1[s]);
    }
    const int row = r0 + r, tt = row / t.tile, rin = row % t.tile;
    const size_t slice = (size_t)t.tile * EKS * 2;                 // bytes of one slice of one K step
    uint8_t* base = t.dig + (((size_t)c * ESUB + q) * ntiles + tt) * ES * slice +
                    (size_t)((rin >> 3) * 256 + h * 128 + (rin & 7) * 16);
#pragma unroll
    for (int s = 0; s < ES; ++s)
      *reinterpret_cast<uint4*>(base + s * slice) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  }
}

// ---------------------------------------------------------------------------
// Product kernel.
// ---------------------------------------------------------------------------
// Bounded wait on an mbarrier phase that also gives up once *abort is set
// (another role of the CTA gave up); false when it gave up (and sets *abort).
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, volatile int* abort) {
  const unsigned long long t0 = tc::now_ns();
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.b32 %0, 1, 0, q;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63) {
      if (*abort || tc::now_ns() - t0 > tc::kWaitNs) {
        *abort = 1;
        return false;
      }
      __nanosleep(64);
    }
  }
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Barrier of the recombining warps (named barrier 1) that also tells each of
// them whether every one passed `ok`: after a wait that gave up in some
// threads and not in others, all of them stop together instead of leaving
// some at a later barrier that the others never reach.
__device__ __forceinline__ bool recombiners_agree(bool ok) {
  uint32_t all;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.and.pred b, 1, %2, a;\n selp.u32 %0, 1, 0, b;\n}"
      : "=r"(all)
      : "r"((uint32_t)ok), "r"(32 * kFlushWarps)
      : "memory");
  return all != 0;
}

__global__ void __launch_bounds__(kThreads, 1)
    gemm_emu_kernel(const GemmTask* __restrict__ tasks, const EmuTerm* __restrict__ eterms, DeviceStatus* status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kBarOff);      // stage loaded (copy bytes arrived)
  uint64_t* empty = full + kStages;                                   // stage read by its MMAs
  uint64_t* grp_done = empty + kStages;                               // a group's MMAs complete
  uint64_t* tmem_free = grp_done + 1;                                 // a group's accumulators read
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tmem_free + 1);
  __shared__ int sEb[EN], sRb[EN], sBadB[EN];
  __shared__ volatile int s_abort;
  __shared__ int s_copied, s_issued;

  const GemmTask t = tasks[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = t.ti * EM, col0 = t.tj * EN;
  const int m = min(EM, t.rows - row0), n = min(EN, t.cols - col0);
  int total = 0;                                       // K chunks over all terms
  for (int it = 0; it < t.nterm; ++it) total += (eterms[t.term0 + it].k + EK - 1) / EK;
  // low bits cut from each group's product: |X| < 2^67.03 per chunk, so the
  // running sums of `total` chunks stay below 2^63 with 5 + ceil(log2 total)
  const int cut = 5 + (total > 1 ? 32 - __clz(total - 1) : 0);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32 * kFlushWarps) {
    for (int b = 0; b < 2 * kStages + 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(full + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_abort = 0;
    s_copied = 0;
    s_issued = 0;
  }
  if (tid < EN) { sRb[tid] = 0; sBadB[tid] = 0; }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  if (warp == kFlushWarps) {
    // ---- copies: stage s of step i holds A's and B's eight slices of one K step
    if (lane == 0) {
      int step = 0;
      for (int it = 0; it < t.nterm && !s_abort; ++it) {
        const EmuTerm e = eterms[t.term0 + it];
        const int nch = (e.k + EK - 1) / EK;
        for (int kq = 0; kq < nch * ESUB; ++kq, ++step) {
          const int st = step % kStages, use = step / kStages;
          if (use > 0 && !wait_phase(smem_u32(empty + st), (uint32_t)((use - 1) & 1), &s_abort)) break;
          const uint32_t fb = smem_u32(full + st), dst = smem_u32(smem + st * kStage);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kStage) : "memory");
          bulk_copy(dst, e.a_dig + ((size_t)kq * e.a_tiles + t.ti) * kABlock, kABlock, fb);
          bulk_copy(dst + kABlock, e.b_dig + ((size_t)kq * e.b_tiles + t.tj) * kBBlock, kBBlock, fb);
          s_copied = step + 1;
        }
        if (s_abort) break;
      }
    }
  } else if (warp == kFlushWarps + 1) {
    // ---- MMAs: 36 per K step into the diagonal accumulators d = s + t
    if (lane == 0) {
      int step = 0, grp = 0;
      for (int it = 0; it < t.nterm && !s_abort; ++it) {
        const int nch = (eterms[t.term0 + it].k + EK - 1) / EK;
        for (int c = 0; c < nch && !s_abort; ++c) {
          const bool first = (c % EG) == 0;
          if (first && grp > 0 && !wait_phase(smem_u32(tmem_free), (uint32_t)((grp - 1) & 1), &s_abort)) break;
          for (int q = 0; q < ESUB; ++q, ++step) {
            const int st = step % kStages, use = step / kStages;
            if (!wait_phase(smem_u32(full + st), (uint32_t)(use & 1), &s_abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(smem + st * kStage), b0 = a0 + kABlock;
            // A_s times the B slices t = t0 .. t0 + cnt - 1 side by side (they are
            // consecutive 64-row groups of shared memory) in one MMA of N = 64 cnt
            // (at most 256), into the accumulators of diagonals s + t0 ..: twelve
            // MMAs per K step instead of 36, each slice of A read once or twice
#pragma unroll
            for (int s = 0; s < ES; ++s)
#pragma unroll
              for (int t0 = 0; t0 < ES - s; t0 += 4) {
                const int cnt = min(4, ES - s - t0);
                const uint64_t ad = smem_desc(a0 + s * kAPart), bd = smem_desc(b0 + t0 * kBPart);
                const uint32_t acc = (first && q == 0 && s == 0) ? 0u : 1u;
                const uint32_t idesc = kIdescBase | ((uint32_t)((EN * cnt) >> 3) << 17);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                        tmem + (uint32_t)((s + t0) * EN)),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
              }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(empty + st)));
            s_issued = step + 1;
          }
          if (s_abort) break;
          if ((c % EG) == EG - 1 || c == nch - 1) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(grp_done)));
            ++grp;
          }
        }
      }
    }
  } else {
    // ---- recombination (warps 0-7) and the epilogue
    const int i = 32 * (warp & 3) + lane, h = warp >> 2;
    long long sum[32];
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) sum[jj] = 0;
    int r_row = 0;
    bool bad_i = false;
    int grp = 0;
    bool stop = false;                                 // the same in every recombining thread
    for (int it = 0; it < t.nterm && !stop; ++it) {
      const EmuTerm e = eterms[t.term0 + it];
      const int nch = (e.k + EK - 1) / EK, ngr = (nch + EG - 1) / EG;
      for (int g = 0; g < ngr; ++g, ++grp) {
        // each thread waits for the group's MMAs itself (a thread that gives up
        // sets s_abort); the exponents are read either way (the split kernel
        // wrote them before this launch)
        const bool ok = wait_phase(smem_u32(grp_done), (uint32_t)(grp & 1), &s_abort);
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int ea = e.a_ex[(size_t)g * e.a_rows_pad + row0 + i];
        if (g == 0) bad_i |= e.a_bad[row0 + i] != 0;
        if (tid < EN) {
          sEb[tid] = e.b_ex[(size_t)g * e.b_rows_pad + col0 + tid];
          if (g == 0 && e.b_bad[col0 + tid]) sBadB[tid] = 1;
        }
        if (!recombiners_agree(ok)) {                  // also the barrier before sEb is read
          stop = true;
          break;
        }
        const int r_new = max(r_row, ea);
#pragma unroll
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
          for (int q4 = 0; q4 < 4; ++q4) {
            const int jj = 4 * g4 + q4, j = 32 * h + jj;
            const int c_old = sRb[j], eb = sEb[j];
            const int c_new = max(c_old, eb);
            int a[ES];
#pragma unroll
            for (int d = 0; d < ES; ++d) a[d] = __float2int_rn(__uint_as_float(v[d][q4]));   // exact: |a| < 2^24
            const long long H = (long long)a[0] * (1 << 21) + (long long)a[1] * (1 << 14) + a[2] * 128 + a[3];
            const long long L = (long long)a[4] * (1 << 21) + (long long)a[5] * (1 << 14) + a[6] * 128 + a[7];
            // X = H 2^28 + L rounded to units of 2^cut (2^28 is a multiple of 2^cut)
            const long long X = H * (1ll << (28 - cut)) + ((L + (1ll << (cut - 1))) >> cut);
            sum[jj] = sra(sum[jj], (r_new - r_row) + (c_new - c_old)) + sra(X, (r_new - ea) + (c_new - eb));
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kFlushWarps));   // every accumulator read
        if (tid == 0) bar_arrive(smem_u32(tmem_free));
        r_row = r_new;
        if (tid < EN) sRb[tid] = max(sRb[tid], sEb[tid]);
      }
    }
    if (!stop) {
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kFlushWarps));     // sRb final everywhere
      // epilogue: C = init + sign * sum * 2^(R_i + R_j - 2105 + cut)
      if (i < m) {
        double* C = t.C + row0 + i + (size_t)col0 * t.ldc;
        const double* D = t.D ? t.D + row0 + i + (size_t)col0 * t.ldd : nullptr;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int j = 32 * h + jj;
          if (j < n) {
            double v = sum[jj] ? ldexp((double)sum[jj], r_row + sRb[j] - 2105 + cut) : 0.0;
            if (bad_i || sBadB[j]) v = __longlong_as_double(0x7FF8000000000000ll);
            double init = 0.0;
            if (D) init = D[(size_t)j * t.ldd];
            else if (t.mode & kAccumulate) init = C[(size_t)j * t.ldc];
            C[(size_t)j * t.ldc] = (t.mode & kSubtract) ? init - v : init + v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (s_abort) {
    // give up: record it, wait (bounded) for the copies and MMAs in flight, then
    // free the tensor memory
    if (tid == 0) {
      if (status) atomicExch(&status->wait_timeout, 1);
      volatile int no_abort = 0;
      const int nc = s_copied, ni = s_issued;
      for (int st = 0; st < kStages && st < nc; ++st) {
        const int last = st + kStages * ((nc - 1 - st) / kStages);
        wait_phase(smem_u32(full + st), (uint32_t)((last / kStages) & 1), &no_abort);
        no_abort = 0;
      }
      if (ni > 0) wait_phase(smem_u32(empty + (ni - 1) % kStages), (uint32_t)(((ni - 1) / kStages) & 1), &no_abort);
    }
    __syncthreads();
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace

cudaError_t launch_gemm_emu(const EmuPlan& plan, const EmuSplitTask* d_split, const GemmTask* d_tasks, int ntask,
                            const EmuTerm* d_eterms, DeviceStatus* status, cudaStream_t st) {
  if (ntask <= 0) return cudaSuccess;
  if (plan.split_ctas > 0) {
    emu_split_kernel<<<plan.split_ctas, 256, 0, st>>>(d_split, (int)plan.split.size());
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaFuncSetAttribute(gemm_emu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  gemm_emu_kernel<<<ntask, kThreads, kSmem, st>>>(d_tasks, d_eterms, status);
  return cudaGetLastError();
}

}  // namespace lrs
