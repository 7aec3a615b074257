// emu_plan.cpp -- host planning of the emulated FP64 products (emu_gemm.cu):
// the distinct operands of a launch, where their digit slices, exponents and
// flags live in one workspace, and the split tasks that fill it.  Plain host
// code, kept apart from the kernels so that it builds without a device
// compiler.
#include <cstdint>
#include <vector>

#include "kernels.cuh"

namespace lrs {
namespace {
constexpr int EM = kEmuTileM;                  // 128 rows of op(A) per tile
constexpr int EN = kEmuTileN;                  // 64 columns of op(B) per tile
constexpr int EK = kEmuChunk;                  // 64: K chunk
constexpr int EG = kEmuGroup;                  // chunks per group (one exponent per row / column)
constexpr int kSplitRows = kEmuSplitRows;      // rows per split CTA
}  // namespace

int gemm_emu_chunks(const GemmTerm* terms, int nterm) {
  int c = 0;
  for (int i = 0; i < nterm; ++i) c += (terms[i].k + EK - 1) / EK;
  return c;
}

void EmuPlan::bind(uint8_t* base) {
  auto at = [base](const void* off) { return base + reinterpret_cast<uintptr_t>(off); };
  for (EmuSplitTask& s : split) {
    s.dig = at(s.dig);
    s.ex = reinterpret_cast<int*>(at(s.ex));
    s.bad = reinterpret_cast<int*>(at(s.bad));
  }
  for (EmuTerm& e : eterms) {
    e.a_dig = at(e.a_dig);
    e.a_ex = reinterpret_cast<const int*>(at(e.a_ex));
    e.a_bad = reinterpret_cast<const int*>(at(e.a_bad));
    e.b_dig = at(e.b_dig);
    e.b_ex = reinterpret_cast<const int*>(at(e.b_ex));
    e.b_bad = reinterpret_cast<const int*>(at(e.b_bad));
  }
}

EmuPlan plan_gemm_emu(const GemmTask* tasks, int ntask, const GemmTerm* terms, int nterms) {
  // a distinct operand: its storage and shape (the same block read the same way
  // by several terms is split once), found through an open-addressing table
  struct Key {
    const double* p;
    int ld, kcontig, rows, k, tile;
    bool operator==(const Key& o) const {
      return p == o.p && ld == o.ld && kcontig == o.kcontig && rows == o.rows && k == o.k && tile == o.tile;
    }
  };
  EmuPlan plan;
  plan.eterms.assign((size_t)nterms, EmuTerm{});
  std::vector<char> seen((size_t)nterms, 0);
  std::vector<Key> keys;
  keys.reserve((size_t)nterms);
  size_t cap = 16;
  while (cap < 4 * (size_t)nterms) cap <<= 1;
  std::vector<int> table(cap, -1);
  auto operand = [&](const Key& k) {
    uint64_t h = (uint64_t)(uintptr_t)k.p * 0x9E3779B97F4A7C15ull;
    h ^= ((uint64_t)(unsigned)k.ld << 32 | (unsigned)k.rows) * 0xC2B2AE3D27D4EB4Full;
    h ^= ((uint64_t)(unsigned)k.k << 8 | (unsigned)(k.tile + k.kcontig)) * 0x165667B19E3779F9ull;
    h ^= h >> 29;
    for (size_t slot = (size_t)h & (cap - 1);; slot = (slot + 1) & (cap - 1)) {
      const int id = table[slot];
      if (id < 0) {
        table[slot] = (int)keys.size();
        keys.push_back(k);
        return (int)keys.size() - 1;
      }
      if (keys[id] == k) return id;
    }
  };
  std::vector<std::pair<int, int>> ops((size_t)nterms);   // per term: A and B operand ids
  for (int ti = 0; ti < ntask; ++ti) {
    const GemmTask& t = tasks[ti];
    for (int j = t.term0; j < t.term0 + t.nterm; ++j) {
      if (seen[j]) continue;
      seen[j] = 1;
      const GemmTerm& g = terms[j];
      const bool ta = g.trans & 1, tb = (g.trans >> 1) & 1;
      // op(A) is rows x k: entry (r, k) at A[k + r lda] when A is stored transposed;
      // op(B)^T is cols x k: entry (j, k) at B[k + j ldb] unless B is stored transposed
      ops[j] = {operand(Key{g.A, g.lda, ta ? 1 : 0, t.rows, g.k, EM}),
                operand(Key{g.B, g.ldb, tb ? 0 : 1, t.cols, g.k, EN})};
    }
  }
  // workspace: digits, then exponents, then the bad flags (zeroed by the caller)
  std::vector<size_t> dig_off(keys.size()), ex_off(keys.size()), bad_off(keys.size());
  size_t off = 0;
  auto round = [](size_t b) { return (b + 255) & ~size_t(255); };
  for (size_t i = 0; i < keys.size(); ++i) {
    const Key& k = keys[i];
    const size_t rows_pad = (size_t)((k.rows + k.tile - 1) / k.tile) * k.tile;
    const size_t nch = (size_t)((k.k + EK - 1) / EK);
    dig_off[i] = off;
    off += round(rows_pad * nch * EK * 16);                          // 8 BF16 digits per entry
  }
  for (size_t i = 0; i < keys.size(); ++i) {
    const Key& k = keys[i];
    const size_t rows_pad = (size_t)((k.rows + k.tile - 1) / k.tile) * k.tile;
    const size_t ngr = (size_t)((k.k + EK * EG - 1) / (EK * EG));
    ex_off[i] = off;
    off += round(rows_pad * ngr * sizeof(int));
  }
  plan.bad_off = off;
  for (size_t i = 0; i < keys.size(); ++i) {
    const Key& k = keys[i];
    const size_t rows_pad = (size_t)((k.rows + k.tile - 1) / k.tile) * k.tile;
    bad_off[i] = off;
    off += round(rows_pad * sizeof(int));
  }
  plan.bad_bytes = off - plan.bad_off;
  plan.bytes = off;
  int cta = 0;
  for (size_t i = 0; i < keys.size(); ++i) {
    const Key& k = keys[i];
    EmuSplitTask s{};
    s.P = k.p;
    s.ld = k.ld;
    s.kcontig = k.kcontig;
    s.rows = k.rows;
    s.k = k.k;
    s.tile = k.tile;
    s.rows_pad = ((k.rows + k.tile - 1) / k.tile) * k.tile;
    s.cta0 = cta;
    s.dig = reinterpret_cast<uint8_t*>(dig_off[i]);
    s.ex = reinterpret_cast<int*>(ex_off[i]);
    s.bad = reinterpret_cast<int*>(bad_off[i]);
    cta += (s.rows_pad / kSplitRows) * ((k.k + EK * EG - 1) / (EK * EG));
    plan.split.push_back(s);
  }
  plan.split_ctas = cta;
  for (int j = 0; j < nterms; ++j) {
    if (!seen[j]) continue;
    const EmuSplitTask& a = plan.split[ops[j].first];
    const EmuSplitTask& b = plan.split[ops[j].second];
    EmuTerm& e = plan.eterms[j];
    e.a_dig = a.dig;
    e.a_ex = a.ex;
    e.a_bad = a.bad;
    e.a_tiles = a.rows_pad / EM;
    e.a_rows_pad = a.rows_pad;
    e.b_dig = b.dig;
    e.b_ex = b.ex;
    e.b_bad = b.bad;
    e.b_tiles = b.rows_pad / EN;
    e.b_rows_pad = b.rows_pad;
    e.k = terms[j].k;
  }
  return plan;
}

}  // namespace lrs
