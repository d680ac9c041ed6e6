// Policy rules of the served loop's scheduler, as plain C++ over any
// simulation record with the fields `resident`, `busy`, `pending` (a
// container of queued requests) and `last_used` (a tick), so that the host
// tests compile them on their own.
#pragma once
#include <cstddef>

namespace stp {

// The simulation to evict so that simulation `exclude` can be admitted:
// resident, not running, not in the batch being formed (protect[j] != 0), and
// not `exclude` itself; among those the least recently used one without queued
// requests, else the least recently used one with requests. -1 if none.
template <class Sims, class Protect>
int choose_victim(const Sims& sims, const Protect& protect, int exclude) {
  int victim = -1;
  const int n = (int)sims.size();
  for (int pass = 0; pass < 2 && victim < 0; ++pass)
    for (int j = 0; j < n; ++j) {
      const auto& c = sims[j];
      if (!c.resident || c.busy || protect[j] || j == exclude) continue;
      if (pass == 0 && !c.pending.empty()) continue;
      if (victim < 0 || c.last_used < sims[victim].last_used) victim = j;
    }
  return victim;
}

// Whether a simulation of `bytes` may join a batch that already holds
// `batch_bytes` in `batch_size` simulations: a batch holds at most half the
// pool when more than one slot can be in flight (its simulations cannot be
// evicted while it runs, and the other half lets the next batch be admitted
// and copied meanwhile), and always at least one simulation.
inline bool batch_has_room(size_t batch_size, size_t batch_bytes, size_t bytes, size_t slots,
                           size_t budget) {
  if (batch_size == 0 || slots <= 1) return true;
  return batch_bytes + bytes <= budget / 2;
}

}  // namespace stp
