// Policy rules of the served loop's scheduler, as plain C++ over any
// simulation record with the fields `resident`, `busy`, `pending` (a
// container of queued requests) and `last_used` (a tick), so that the host
// tests compile them on their own.
#pragma once
#include <cstddef>
#include <vector>

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

// Order in which the ready simulations are offered to the batch being formed.
// `ready` lists simulation ids in the order they became ready (FIFO). Policy 0
// (FIFO): that order. Policy 1 (resident first, with an age bound): first
// every simulation whose oldest request has waited at least `age_bound`
// seconds, then the ones already resident in the pool, then the rest, each
// group in FIFO order - a resident simulation needs no admission copy (and
// evicts nothing), while the age bound keeps a non-resident one from waiting
// without limit behind them. Uses sims[i].resident and
// sims[i].pending.front().t_arrival (every ready simulation has a request).
template <class Sims, class Ready>
void ready_order(const Sims& sims, const Ready& ready, int policy, double now, double age_bound,
                 std::vector<int>* out) {
  out->clear();
  if (policy == 0) {
    for (int i : ready) out->push_back(i);
    return;
  }
  auto aged = [&](int i) { return now - sims[i].pending.front().t_arrival >= age_bound; };
  for (int i : ready)
    if (aged(i)) out->push_back(i);
  for (int i : ready)
    if (!aged(i) && sims[i].resident) out->push_back(i);
  for (int i : ready)
    if (!aged(i) && !sims[i].resident) out->push_back(i);
}

}  // namespace stp
