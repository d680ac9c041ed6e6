// Host check of the batched plan's launch grouping (csrc/launch_groups.h),
// against properties read off the definition, on seeded random inputs:
//   - every set with units lands in exactly one launch, sets without none;
//   - a launch holds one key, at most max_sets sets, in input order;
//   - each key's sets fill its launches in input order, all full but the last;
//   - first_unit[k] = units of the members before k; count and cost are sums;
//   - every unit of a launch maps, by the kernel's search (the last member
//     whose first unit is <= u), to a member and a unit inside that member;
//   - launches are ordered by cost, longest first, ties in creation order;
//   - branches: each launch goes to the least loaded branch (first of equals),
//     never more branches than launches.
// Prints "ok <cases>" and exits 0, or names the first failure and exits 1.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <utility>
#include <vector>

#include "launch_groups.h"

using stp::GroupInput;
using stp::LaunchGroup;

static unsigned long long g_state = 0x9E3779B97F4A7C15ull;
static unsigned next_u32() {
  g_state = g_state * 6364136223846793005ull + 1442695040888963407ull;
  return (unsigned)(g_state >> 33);
}

#define CHECK(c, what)                                                        \
  do {                                                                        \
    if (!(c)) {                                                               \
      std::printf("FAIL case %d: %s (line %d)\n", cs, what, __LINE__);       \
      return 1;                                                               \
    }                                                                         \
  } while (0)

int main() {
  int cases = 0;
  const int max_sets_list[] = {1, 3, 7, 128};
  for (int cs = 0; cs < 400; ++cs) {
    const int n = (int)(next_u32() % 300);
    const int nkeys = 1 + (int)(next_u32() % 6);
    const int max_sets = max_sets_list[cs % 4];
    std::vector<GroupInput> in((size_t)n);
    for (int i = 0; i < n; ++i) {
      in[(size_t)i].key = (int)(next_u32() % (unsigned)nkeys) * 7 + 2;
      in[(size_t)i].units = (next_u32() % 5 == 0) ? 0 : 1 + (int64_t)(next_u32() % 40);
      // some equal costs, to exercise the order of ties
      in[(size_t)i].unit_cost = (next_u32() % 3 == 0) ? 1.0 : 0.25 * (1 + next_u32() % 16);
    }
    const std::vector<LaunchGroup> g = stp::group_launches(in, max_sets);

    // membership
    std::vector<int> seen((size_t)n, 0);
    for (const LaunchGroup& l : g)
      for (int s : l.sets) {
        CHECK(s >= 0 && s < n, "set index in range");
        ++seen[(size_t)s];
      }
    for (int i = 0; i < n; ++i)
      CHECK(seen[(size_t)i] == (in[(size_t)i].units > 0 ? 1 : 0), "each set with units exactly once");

    // per launch: key, size, order, offsets, sums, unit mapping
    for (const LaunchGroup& l : g) {
      CHECK(!l.sets.empty() && (int)l.sets.size() <= max_sets, "launch size");
      CHECK(l.first_unit.size() == l.sets.size(), "one offset per member");
      int64_t acc = 0;
      double cost = 0.0;
      for (size_t k = 0; k < l.sets.size(); ++k) {
        const GroupInput& s = in[(size_t)l.sets[k]];
        CHECK(s.key == l.key, "one key per launch");
        if (k) CHECK(l.sets[k] > l.sets[k - 1], "members in input order");
        CHECK(l.first_unit[k] == acc, "first unit = units before");
        acc += s.units;
        cost += s.unit_cost * (double)s.units;
      }
      CHECK(l.count == acc, "count = sum of units");
      CHECK(std::fabs(l.cost - cost) <= 1e-9 * (1.0 + cost), "cost = sum of unit costs");
      for (int64_t u = 0; u < l.count; ++u) {
        int lo = 0, hi = (int)l.sets.size() - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (l.first_unit[(size_t)mid] <= u) lo = mid; else hi = mid - 1;
        }
        const int64_t local = u - l.first_unit[(size_t)lo];
        CHECK(local >= 0 && local < in[(size_t)l.sets[(size_t)lo]].units, "unit maps inside its member");
      }
    }

    // chunking per key: launches of a key, in creation order, list the key's
    // sets in input order, every launch full but the last
    std::map<int, std::vector<int>> by_key;
    for (int i = 0; i < n; ++i)
      if (in[(size_t)i].units > 0) by_key[in[(size_t)i].key].push_back(i);
    for (const auto& kv : by_key) {
      std::vector<const LaunchGroup*> ls;
      for (const LaunchGroup& l : g)
        if (l.key == kv.first) ls.push_back(&l);
      // creation order: by first member index
      std::vector<const LaunchGroup*> created = ls;
      for (size_t a = 1; a < created.size(); ++a)
        for (size_t b = a; b > 0 && created[b]->sets[0] < created[b - 1]->sets[0]; --b)
          std::swap(created[b], created[b - 1]);
      const size_t want = (kv.second.size() + (size_t)max_sets - 1) / (size_t)max_sets;
      CHECK(created.size() == want, "launches per key = ceil(sets / max_sets)");
      size_t pos = 0;
      for (size_t c = 0; c < created.size(); ++c) {
        if (c + 1 < created.size()) CHECK((int)created[c]->sets.size() == max_sets, "full chunks");
        for (int s : created[c]->sets) CHECK(s == kv.second[pos++], "chunks follow input order");
      }
    }

    // order: cost non-increasing; ties keep creation order, which is key by
    // key (keys in order of first appearance), each key's chunks in order
    std::map<int, int> key_rank;
    for (int i = 0; i < n; ++i)
      if (in[(size_t)i].units > 0 && !key_rank.count(in[(size_t)i].key))
        key_rank[in[(size_t)i].key] = (int)key_rank.size();
    auto created_rank = [&](const LaunchGroup& l) {
      return (int64_t)key_rank[l.key] * 1000000 + l.sets[0];
    };
    for (size_t k = 1; k < g.size(); ++k) {
      CHECK(g[k - 1].cost >= g[k].cost, "longest first");
      if (g[k - 1].cost == g[k].cost)
        CHECK(created_rank(g[k - 1]) < created_rank(g[k]), "ties in creation order");
    }

    // branches
    const int nbr = 1 + (int)(next_u32() % 5);
    std::vector<double> costs;
    for (const LaunchGroup& l : g) costs.push_back(l.cost);
    const std::vector<int> br = stp::lpt_branches(costs, nbr);
    CHECK(br.size() == costs.size(), "one branch per launch");
    const int nb = std::max(1, std::min<int>(nbr, (int)costs.size()));
    std::vector<double> load((size_t)nb, 0.0);
    for (size_t k = 0; k < costs.size(); ++k) {
      CHECK(br[k] >= 0 && br[k] < nb, "branch in range");
      int best = 0;
      for (int b = 1; b < nb; ++b)
        if (load[(size_t)b] < load[(size_t)best]) best = b;
      CHECK(br[k] == best, "least loaded branch, first of equals");
      load[(size_t)br[k]] += costs[k];
    }
    ++cases;
  }
  std::printf("ok %d\n", cases);
  return 0;
}
