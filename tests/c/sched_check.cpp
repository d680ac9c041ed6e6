// Host check of the served scheduler's policy rules (serve_policy.h): the eviction
// victim against a brute-force reading of the rule over seeded random
// simulation tables, and the half-pool batch bound on its cases.
// Prints "ok <cases>" and exits 0, or the first mismatch and exits 1.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <deque>
#include <vector>

#include "serve_policy.h"

namespace {

struct SimRec {
  bool resident = false, busy = false;
  std::deque<int> pending;
  int64_t last_used = 0;
};

uint64_t state = 0x2545F4914F6CDD1Dull;
uint64_t next_u64() {  // xorshift64*
  state ^= state >> 12;
  state ^= state << 25;
  state ^= state >> 27;
  return state * 0x2545F4914F6CDD1Dull;
}

// The rule read literally: candidates are resident, idle, unprotected and not
// the excluded one; prefer those without requests; the smallest tick wins,
// the lower index on a tie.
int expected_victim(const std::vector<SimRec>& s, const std::vector<char>& prot, int ex) {
  for (int want_idle_queue = 1; want_idle_queue >= 0; --want_idle_queue) {
    int best = -1;
    for (int j = 0; j < (int)s.size(); ++j) {
      if (!s[j].resident || s[j].busy || prot[j] || j == ex) continue;
      if (want_idle_queue && !s[j].pending.empty()) continue;
      if (best < 0 || s[j].last_used < s[best].last_used) best = j;
    }
    if (best >= 0) return best;
  }
  return -1;
}

struct Req {
  double t_arrival;
};
struct ReadyRec {
  bool resident = false;
  std::deque<Req> pending;
};

// The ready order read literally: a stable sort of the FIFO list by the key
// (aged: 0, resident: 1, other: 2); FIFO unchanged for policy 0.
std::vector<int> expected_order(const std::vector<ReadyRec>& s, const std::vector<int>& ready,
                                int policy, double now, double bound) {
  std::vector<int> out(ready);
  if (policy == 0) return out;
  auto key = [&](int i) {
    if (now - s[i].pending.front().t_arrival >= bound) return 0;
    return s[i].resident ? 1 : 2;
  };
  std::stable_sort(out.begin(), out.end(), [&](int a, int b) { return key(a) < key(b); });
  return out;
}

}  // namespace

int main() {
  int cases = 0;
  for (int t = 0; t < 20000; ++t) {
    const int n = 1 + (int)(next_u64() % 12);
    std::vector<SimRec> sims((size_t)n);
    std::vector<char> prot((size_t)n, 0);
    for (int j = 0; j < n; ++j) {
      sims[j].resident = next_u64() % 4 != 0;
      sims[j].busy = next_u64() % 4 == 0;
      if (next_u64() % 2) sims[j].pending.push_back(1);
      sims[j].last_used = (int64_t)(next_u64() % 8);  // ties on purpose
      prot[j] = next_u64() % 5 == 0;
    }
    const int ex = (int)(next_u64() % (uint64_t)(n + 1)) - 1;  // -1: nothing excluded
    const int got = stp::choose_victim(sims, prot, ex);
    const int want = expected_victim(sims, prot, ex);
    if (got != want) {
      std::printf("mismatch: victim %d, expected %d (case %d)\n", got, want, t);
      return 1;
    }
    ++cases;
  }
  struct { size_t size, bytes, add, slots, budget; bool room; } b[] = {
      {0, 0, 900, 3, 1000, true},     // an empty batch takes anything, even > budget/2
      {1, 400, 100, 3, 1000, true},   // 500 <= 500
      {1, 400, 101, 3, 1000, false},  // 501 > 500
      {5, 499, 2, 2, 1000, false},
      {5, 900, 900, 1, 1000, true},   // one slot: no bound
      {2, 0, 0, 8, 0, true},
  };
  for (const auto& c : b) {
    if (stp::batch_has_room(c.size, c.bytes, c.add, c.slots, c.budget) != c.room) {
      std::printf("mismatch: batch bound (%zu, %zu, %zu, %zu, %zu)\n", c.size, c.bytes, c.add,
                  c.slots, c.budget);
      return 1;
    }
    ++cases;
  }
  for (int t = 0; t < 20000; ++t) {
    const int n = 1 + (int)(next_u64() % 10);
    std::vector<ReadyRec> sims((size_t)n);
    for (int j = 0; j < n; ++j) {
      sims[j].resident = next_u64() % 2 != 0;
      sims[j].pending.push_back(Req{(double)(next_u64() % 100) * 1e-3});
    }
    std::vector<int> ready;
    for (int j = 0; j < n; ++j)
      if (next_u64() % 4 != 0) ready.push_back(j);
    for (size_t a = ready.size(); a > 1; --a) std::swap(ready[a - 1], ready[next_u64() % a]);
    const int policy = (int)(next_u64() % 2);
    const double now = 0.1, bound = (double)(next_u64() % 60) * 1e-3;
    std::vector<int> got;
    stp::ready_order(sims, ready, policy, now, bound, &got);
    if (got != expected_order(sims, ready, policy, now, bound)) {
      std::printf("mismatch: ready order (case %d)\n", t);
      return 1;
    }
    ++cases;
  }
  // launch forms: the flop count of one element written out per order, the
  // batch's work against the threshold, and the N = 12 Cartesian rule
  {
    const double fl4 = 36.0 * 1024 + 66.0 * 256 + 108.0 * 64;  // N = 4
    const double got = stp::step_work_ms(4, 1000, false), want = 1000 * fl4 / 1.2e9;
    if (got < want * (1 - 1e-12) || got > want * (1 + 1e-12)) {
      std::printf("mismatch: step work N=4 %g vs %g\n", got, want);
      return 1;
    }
    const double gc = stp::step_work_ms(4, 1000, true);
    if (gc < 1.7 * want * (1 - 1e-12) || gc > 1.7 * want * (1 + 1e-12)) {
      std::printf("mismatch: curvilinear step work\n");
      return 1;
    }
    ++cases;
  }
  for (int t = 0; t < 20000; ++t) {
    const int n = 1 + (int)(next_u64() % 10);
    std::vector<int> N((size_t)n);
    std::vector<int64_t> E((size_t)n);
    std::vector<char> curv((size_t)n);
    double work = 0.0;
    for (int j = 0; j < n; ++j) {
      N[(size_t)j] = 1 + (int)(next_u64() % 12);
      E[(size_t)j] = 1 + (int64_t)(next_u64() % 3000);
      curv[(size_t)j] = next_u64() % 3 == 0;
      const double m = N[(size_t)j];
      work += (curv[(size_t)j] ? 1.7 : 1.0) * (double)E[(size_t)j] *
              (36 * m * m * m * m * m + 66 * m * m * m * m + 108 * m * m * m) / 1.2e9;
    }
    const double thr = (double)(next_u64() % 80);
    const std::vector<char> got = stp::launch_forms(N, E, curv, thr);
    for (int j = 0; j < n; ++j) {
      const bool want = work > thr || (N[(size_t)j] == 12 && !curv[(size_t)j]);
      if ((got[(size_t)j] != 0) != want) {
        std::printf("mismatch: launch form (case %d, set %d)\n", t, j);
        return 1;
      }
    }
    ++cases;
  }
  std::printf("ok %d\n", cases);
  return 0;
}
