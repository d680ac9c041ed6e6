// Policy rules of the served loop's scheduler, as plain C++ over any
// simulation record with the fields `resident`, `busy`, `pending` (a
// container of queued requests) and `last_used` (a tick), so that the host
// tests compile them on their own.
#pragma once
#include <cstddef>
#include <cstdint>
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

// Estimated FP64 work of one STP step, in milliseconds at 1.2 TFLOP/s: E
// elements with N nodes per direction, a curvilinear element counted 1.7
// times a Cartesian one (every quantity is differentiated along every
// direction).
inline double step_work_ms(int N, int64_t E, bool curvilinear) {
  const double n = N;
  const double flops = 36.0 * n * n * n * n * n + 66.0 * n * n * n * n + 108.0 * n * n * n;
  return (curvilinear ? 1.7 : 1.0) * (double)E * flops / 1.2e9;
}

// Launch form of each FP64 simulation of a batch: 1 = the per-shape
// persistent launches, 0 = the one allocation-free launch. A batch with more
// than `threshold_ms` of work runs per shape as a whole; an N = 12 Cartesian
// simulation always does (there the allocation-free kernel's body differs
// from the single-set kernel's, and a simulation must round the same in
// every batch).
inline std::vector<char> launch_forms(const std::vector<int>& N, const std::vector<int64_t>& E,
                                      const std::vector<char>& curvilinear, double threshold_ms) {
  double work = 0.0;
  for (size_t k = 0; k < N.size(); ++k) work += step_work_ms(N[k], E[k], curvilinear[k] != 0);
  std::vector<char> out(N.size(), 0);
  for (size_t k = 0; k < N.size(); ++k)
    out[k] = (work > threshold_ms || (N[k] == 12 && !curvilinear[k])) ? 1 : 0;
  return out;
}

}  // namespace stp
