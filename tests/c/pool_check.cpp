// Host check of the served loop's first-fit sub-allocator (pool.h) against a
// byte map of the same pool: seeded random allocations and releases, and
// after every operation
//   - a successful alloc returns an aligned offset whose block lies inside
//     the pool and overlaps no live block;
//   - the offset is the lowest start of a free run that can hold the
//     rounded-up size (first fit over fully merged free runs), and alloc
//     fails exactly when no such run exists;
//   - used() equals the bytes the live blocks cover.
// Prints "ok <operations>" and exits 0, or prints the first mismatch and
// exits 1.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "pool.h"

namespace {

struct Block {
  size_t off, n;
};

uint64_t state = 0x9E3779B97F4A7C15ull;
uint64_t next_u64() {  // xorshift64*
  state ^= state >> 12;
  state ^= state << 25;
  state ^= state >> 27;
  return state * 0x2545F4914F6CDD1Dull;
}

// lowest start of a free run of at least n units in the map, or -1
long first_run(const std::vector<char>& map, size_t n) {
  size_t run = 0;
  for (size_t i = 0; i < map.size(); ++i) {
    run = map[i] ? 0 : run + 1;
    if (run >= n) return (long)(i + 1 - n);
  }
  return -1;
}

int fail(const char* what, long a, long b) {
  std::printf("mismatch: %s (%ld vs %ld)\n", what, a, b);
  return 1;
}

int run_case(size_t units, int ops, int max_units, uint64_t seed) {
  state = seed;
  const size_t A = stp::kPoolAlign;
  stp::Pool pool;
  pool.reset(units * A);
  std::vector<char> map(units, 0);  // one entry per aligned unit
  std::vector<Block> live;
  size_t live_bytes = 0;
  for (int op = 0; op < ops; ++op) {
    const bool do_alloc = live.empty() || next_u64() % 100 < 55;
    if (do_alloc) {
      // sizes that are and are not multiples of the alignment
      const size_t req = 1 + next_u64() % ((size_t)max_units * A);
      const size_t n_units = stp::pool_align_up(req) / A;
      const long expect = first_run(map, n_units);
      size_t off = 0;
      const bool ok = pool.alloc(req, &off);
      if (ok != (expect >= 0)) return fail("alloc success", ok, expect);
      if (!ok) continue;
      if (off % A) return fail("alignment", (long)off, 0);
      if ((long)(off / A) != expect) return fail("first-fit offset", (long)(off / A), expect);
      for (size_t u = off / A; u < off / A + n_units; ++u) {
        if (u >= units) return fail("block past the pool", (long)u, (long)units);
        if (map[u]) return fail("overlap", (long)u, 1);
        map[u] = 1;
      }
      live.push_back({off, req});
      live_bytes += n_units * A;
    } else {
      const size_t k = next_u64() % live.size();
      const Block b = live[k];
      live[k] = live.back();
      live.pop_back();
      const size_t n_units = stp::pool_align_up(b.n) / A;
      for (size_t u = b.off / A; u < b.off / A + n_units; ++u) map[u] = 0;
      pool.release(b.off, b.n);
      live_bytes -= n_units * A;
    }
    if (pool.used() != live_bytes) return fail("used()", (long)pool.used(), (long)live_bytes);
  }
  // release everything: the free runs merge back into one block of the pool
  for (const Block& b : live) pool.release(b.off, b.n);
  size_t off = 1;
  if (pool.used() != 0) return fail("used() after releasing all", (long)pool.used(), 0);
  if (!pool.alloc(units * A, &off) || off != 0) return fail("whole pool after releasing all", (long)off, 0);
  if (pool.alloc(1, &off)) return fail("alloc in a full pool", 1, 0);
  return 0;
}

}  // namespace

int main() {
  int total = 0;
  const struct { size_t units; int ops, max_units; } cases[] = {
      {1, 200, 1}, {64, 4000, 8}, {1000, 20000, 40}, {4096, 20000, 600}, {300, 20000, 300}};
  for (int c = 0; c < 5; ++c) {
    if (run_case(cases[c].units, cases[c].ops, cases[c].max_units, 0x1234567ull + 977ull * c)) {
      std::printf("case %d\n", c);
      return 1;
    }
    total += cases[c].ops;
  }
  // an empty pool holds nothing
  stp::Pool empty;
  empty.reset(0);
  size_t off = 0;
  if (empty.alloc(1, &off)) return fail("alloc in an empty pool", 1, 0);
  std::printf("ok %d\n", total);
  return 0;
}
