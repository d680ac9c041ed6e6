// Host-side grouping of the batched plan's work (plain C++, no CUDA; checked
// on the CPU by tests/c/launch_groups_check.cpp).
//
// Sets of one shape (equal key) share one persistent launch, at most
// `max_sets` of them per launch (the size of the kernel's parameter table);
// a launch numbers its work units set by set, so member k owns units
// [first_unit[k], first_unit[k] + units). Launches are ordered by estimated
// work, longest first (ties keep their creation order), and spread over
// parallel branches longest-processing-time first: each launch to the branch
// with the least estimated work so far.
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>

namespace stp {

struct GroupInput {
  int key;           // shape identity: sets with equal keys share a kernel
  int64_t units;     // work units of the set (<= 0: the set is left out)
  double unit_cost;  // estimated microseconds per unit
};

struct LaunchGroup {
  int key = 0;
  std::vector<int> sets;            // input indices, in input order
  std::vector<int64_t> first_unit;  // per member: units of the members before it
  int64_t count = 0;                // units of the launch
  double cost = 0.0;                // estimated microseconds of the launch
};

inline std::vector<LaunchGroup> group_launches(const std::vector<GroupInput>& in, int max_sets) {
  std::vector<LaunchGroup> built;
  std::vector<char> done(in.size(), 0);
  for (size_t i = 0; i < in.size(); ++i) {
    if (done[i] || in[i].units <= 0) continue;
    size_t g = 0;
    bool open = false;
    for (size_t j = i; j < in.size(); ++j) {
      if (done[j] || in[j].units <= 0 || in[j].key != in[i].key) continue;
      if (!open || (int)built[g].sets.size() == max_sets) {
        built.emplace_back();
        g = built.size() - 1;
        built[g].key = in[i].key;
        open = true;
      }
      LaunchGroup& l = built[g];
      l.sets.push_back((int)j);
      l.first_unit.push_back(l.count);
      l.count += in[j].units;
      l.cost += in[j].unit_cost * (double)in[j].units;
      done[j] = 1;
    }
  }
  std::stable_sort(built.begin(), built.end(),
                   [](const LaunchGroup& a, const LaunchGroup& b) { return a.cost > b.cost; });
  return built;
}

// Branch of each item (costs in launch order) over at most `nbranches`
// branches, and never more branches than items.
inline std::vector<int> lpt_branches(const std::vector<double>& costs, int nbranches) {
  const int nb = std::max(1, std::min<int>(nbranches, (int)costs.size()));
  std::vector<double> load((size_t)nb, 0.0);
  std::vector<int> out;
  out.reserve(costs.size());
  for (double c : costs) {
    const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    out.push_back(b);
    load[(size_t)b] += c;
  }
  return out;
}

}  // namespace stp
