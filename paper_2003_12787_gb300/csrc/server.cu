// Served Space-Time Predictor: a continuously batched request loop over many
// independent simulations whose state stays resident on the device.
//
// Every simulation owns, inside one device pool of a fixed HBM budget, two
// state buffers (q_n and the next average), its material field and its face
// projections. A request advances one simulation by one STP step; the
// corrector is outside the method's hot path, so q_{n+1} := avg_n stands in
// for it and is a swap of the two state buffers' roles (no copy). Requests of
// one simulation run one after another.
//
// The scheduler (progress) repeatedly:
//   1. retires finished batches (event query per in-flight slot): records
//      completion times, swaps the state roles, re-queues simulations that
//      have more requests;
//   2. admits ready simulations into the pool (first-fit sub-allocation);
//      when the budget is exhausted it evicts idle simulations, least
//      recently used first, copying their state and last faces back to
//      pinned host memory. Evictions (device to host) and admissions (host
//      to device: state and material; the faces are not copied in, since the
//      launch that follows every admission overwrites them and reads drain
//      first) run on two copy streams, so the two directions overlap; an
//      admission waits for the evictions issued before it (its memory may be
//      theirs, and a re-admitted simulation's host copy must be complete);
//   3. launches up to 128 ready, resident simulations on a free slot (its
//      own stream and scratch): the FP64 ones, Cartesian and curvilinear
//      (their per-node inverse Jacobians resident beside the material)
//      alike, as one allocation-free persistent launch when the batch is
//      small, else as the batched plan's per-shape persistent launches, one
//      after another on the slot's stream; simulations whose handle runs
//      another precision get a
//      launch of their own (the handle's kernel) on the same stream, between
//      the same timing events.
// New requests therefore join the next launch while earlier launches are
// still on the GPU, and launches on different slots overlap on the device.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "pool.h"
#include "serve_policy.h"
#include "stp_internal.h"

namespace stp {
namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAlign = kPoolAlign;

size_t align_up(size_t x) { return pool_align_up(x); }

struct Request {
  int64_t id;      // index in the caller's trace (or submit order)
  double t_arrival;  // seconds on the server clock
};

struct Sim {
  stp_handle handle = nullptr;
  int N = 0;
  int64_t E = 0;
  size_t bytes_state = 0, bytes_params = 0, bytes_faces = 0, bytes_metric = 0;
  double* host_q = nullptr;       // pinned: state while evicted
  double* host_params = nullptr;  // pinned
  double* host_metric = nullptr;  // pinned (curvilinear simulations only)
  double* host_faces = nullptr;   // pinned: last faces while evicted
  // whether the pinned host copies exist: a simulation added from device
  // buffers that fit the pool starts resident without them, and gets them on
  // its first eviction (the pinned footprint follows what is evicted)
  bool host_backed = false;
  bool resident = false;
  ServedSources* sources = nullptr;  // point sources (owned), or none
  size_t off = 0;  // pool offset of [state0 | state1 | params | faces | metric]
  int cur = 0;     // which state buffer holds q_n
  bool busy = false, queued = false, have_faces = false;
  int64_t last_used = 0, steps = 0;
  std::deque<Request> pending;
  size_t footprint() const {
    return 2 * align_up(bytes_state) + align_up(bytes_params) + align_up(bytes_faces) +
           align_up(bytes_metric);
  }
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t start = nullptr;  // timing events around the launch
  cudaEvent_t done = nullptr;
  unsigned char* scratch = nullptr;
  std::vector<int> sims;
  bool busy = false;
};

}  // namespace

struct Server {
  int device = -1;
  size_t budget = 0;
  unsigned char* pool_base = nullptr;
  Pool pool;
  std::vector<Sim> sims;
  std::vector<Slot> slots;
  std::deque<int> ready;  // simulations with a request, not running, FIFO
  int policy = 1;           // ready order (serve_policy.h): 0 FIFO, 1 resident first
  double age_bound = 0.05;  // seconds a request may wait before it goes first
  cudaStream_t copy_stream = nullptr;   // admissions (host to device)
  cudaStream_t evict_stream = nullptr;  // evictions (device to host)
  cudaEvent_t copy_done = nullptr;
  cudaEvent_t evict_done = nullptr;
  Clock::time_point t0 = Clock::now();
  int64_t tick = 0;
  std::vector<int> order;  // scratch of the ready order
  // statistics
  int64_t completed = 0, batches = 0, admissions = 0, evictions = 0, max_batch = 0,
          batched_requests = 0, next_id = 0;
  double kernel_ms = 0.0;  // sum of the launches' device times (start..done events)
  size_t peak_used = 0;
  // completion records of the current trace: id -> completion time
  std::vector<double>* completion = nullptr;
  std::mutex mu;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  double* state(const Sim& s, int which) const {
    return reinterpret_cast<double*>(pool_base + s.off + which * align_up(s.bytes_state));
  }
  double* params(const Sim& s) const {
    return reinterpret_cast<double*>(pool_base + s.off + 2 * align_up(s.bytes_state));
  }
  double* faces(const Sim& s) const {
    return reinterpret_cast<double*>(pool_base + s.off + 2 * align_up(s.bytes_state) + align_up(s.bytes_params));
  }
  double* metric(const Sim& s) const {
    return reinterpret_cast<double*>(pool_base + s.off + 2 * align_up(s.bytes_state) +
                                     align_up(s.bytes_params) + align_up(s.bytes_faces));
  }

  // Pinned host copies of simulation i (state, material, faces, metric).
  cudaError_t make_host_backing(Sim& s) {
    cudaError_t e = cudaMallocHost(&s.host_q, std::max<size_t>(s.bytes_state, 8));
    if (e == cudaSuccess) e = cudaMallocHost(&s.host_params, std::max<size_t>(s.bytes_params, 8));
    if (e == cudaSuccess) e = cudaMallocHost(&s.host_faces, std::max<size_t>(s.bytes_faces, 8));
    if (e == cudaSuccess && s.bytes_metric) e = cudaMallocHost(&s.host_metric, s.bytes_metric);
    if (e == cudaSuccess) s.host_backed = true;
    return e;
  }

  cudaError_t evict(int i) {
    Sim& s = sims[i];
    cudaError_t e = cudaSuccess;
    if (!s.host_backed) {  // first eviction: the material (and metric) leave the pool too
      if ((e = make_host_backing(s)) != cudaSuccess) return e;
      e = cudaMemcpyAsync(s.host_params, params(s), s.bytes_params, cudaMemcpyDeviceToHost, evict_stream);
      if (e == cudaSuccess && s.bytes_metric)
        e = cudaMemcpyAsync(s.host_metric, metric(s), s.bytes_metric, cudaMemcpyDeviceToHost, evict_stream);
      if (e != cudaSuccess) return e;
    }
    e = cudaMemcpyAsync(s.host_q, state(s, s.cur), s.bytes_state, cudaMemcpyDeviceToHost, evict_stream);
    if (e == cudaSuccess && s.have_faces)
      e = cudaMemcpyAsync(s.host_faces, faces(s), s.bytes_faces, cudaMemcpyDeviceToHost, evict_stream);
    // later admissions (which may reuse this memory or re-admit this
    // simulation) start after these copies
    if (e == cudaSuccess) e = cudaEventRecord(evict_done, evict_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(copy_stream, evict_done, 0);
    if (e != cudaSuccess) return e;
    pool.release(s.off, s.footprint());
    s.resident = false;
    s.cur = 0;
    ++evictions;
    return cudaSuccess;
  }

  // Make simulation i resident; returns false if the budget cannot hold it
  // even after evicting every idle simulation outside `protect`.
  bool admit(int i, const std::vector<char>& protect, bool* copied, cudaError_t* err) {
    Sim& s = sims[i];
    if (s.resident) return true;
    size_t off = 0;
    while (!pool.alloc(s.footprint(), &off)) {
      // least recently used idle resident simulation, preferring ones without requests
      const int victim = choose_victim(sims, protect, i);
      if (victim < 0) return false;
      if ((*err = evict(victim)) != cudaSuccess) return false;
    }
    s.off = off;
    s.resident = true;
    s.cur = 0;
    *err = cudaMemcpyAsync(state(s, 0), s.host_q, s.bytes_state, cudaMemcpyHostToDevice, copy_stream);
    if (*err == cudaSuccess)
      *err = cudaMemcpyAsync(params(s), s.host_params, s.bytes_params, cudaMemcpyHostToDevice, copy_stream);
    if (*err == cudaSuccess && s.bytes_metric)
      *err = cudaMemcpyAsync(metric(s), s.host_metric, s.bytes_metric, cudaMemcpyHostToDevice, copy_stream);
    *copied = true;
    ++admissions;
    peak_used = std::max(peak_used, pool.used());
    return *err == cudaSuccess;
  }

  void submit(int i, int64_t id, double t_arrival) {
    Sim& s = sims[i];
    s.pending.push_back(Request{id, t_arrival});
    if (!s.busy && !s.queued) {
      ready.push_back(i);
      s.queued = true;
    }
  }

  // One scheduler pass. Returns the number of requests completed in it.
  cudaError_t progress(int* n_completed) {
    int done_now = 0;
    cudaError_t e;
    // 1. retire finished launches
    for (Slot& sl : slots) {
      if (!sl.busy) continue;
      e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) return e;
      const double t = now();
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, sl.start, sl.done) == cudaSuccess) kernel_ms += ms;
      for (int i : sl.sims) {
        Sim& s = sims[i];
        const Request r = s.pending.front();
        s.pending.pop_front();
        if (completion && r.id >= 0 && r.id < (int64_t)completion->size()) (*completion)[r.id] = t;
        s.cur ^= 1;  // q_{n+1} := avg_n
        s.busy = false;
        s.have_faces = true;
        s.last_used = ++tick;
        ++s.steps;
        ++done_now;
        if (!s.pending.empty() && !s.queued) {
          ready.push_back(i);
          s.queued = true;
        }
      }
      sl.sims.clear();
      sl.busy = false;
    }
    completed += done_now;
    if (n_completed) *n_completed = done_now;
    // 2./3. admit and launch on every free slot while work is ready
    for (Slot& sl : slots) {
      if (sl.busy || ready.empty()) continue;
      std::vector<char> protect(sims.size(), 0);
      std::vector<int> batch;
      bool copied = false;
      size_t batch_bytes = 0;
      // candidates in the policy's order; the ones taken leave the ready
      // queue, the others keep their FIFO places
      ready_order(sims, ready, policy, now(), age_bound, &order);
      for (int i : order) {
        if ((int)batch.size() >= static_max_sets()) break;
        // at most half the pool per batch, so the next one is admitted meanwhile
        if (!batch_has_room(batch.size(), batch_bytes, sims[i].footprint(), slots.size(), budget))
          break;
        cudaError_t ae = cudaSuccess;
        if (admit(i, protect, &copied, &ae)) {
          protect[i] = 1;
          batch.push_back(i);
          batch_bytes += sims[i].footprint();
        } else {
          if (ae != cudaSuccess) {  // a copy failed: nothing of this batch runs
            for (int j : batch) sims[j].busy = false;
            return ae;  // the ready queue still holds every simulation of the batch
          }
          break;  // does not fit next to this batch: wait
        }
      }
      if (batch.empty()) break;
      {
        std::deque<int> rest;
        for (int i : ready)
          if (!protect[i]) rest.push_back(i);
        ready.swap(rest);
      }
      if (copied) {
        e = cudaEventRecord(copy_done, copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.stream, copy_done, 0);
        if (e != cudaSuccess) {
          requeue_front(batch);
          return e;
        }
      }
      const int n = (int)batch.size();
      std::vector<int> N, own;  // own: simulations launched one by one (not FP64)
      std::vector<int64_t> E;
      std::vector<const double*> q, p, tb, mt;
      std::vector<double*> a, f;
      std::vector<double> dx;
      for (int k = 0; k < n; ++k) {
        Sim& s = sims[batch[k]];
        s.busy = true;
        s.queued = false;
        if (!stp_handle_is_fp64(s.handle)) {  // a launch of its own
          own.push_back(batch[k]);
          continue;
        }
        N.push_back(s.N);
        E.push_back(s.E);
        q.push_back(state(s, s.cur));
        a.push_back(state(s, s.cur ^ 1));
        p.push_back(params(s));
        f.push_back(faces(s));
        tb.push_back(stp_handle_tables(s.handle));
        mt.push_back(s.bytes_metric ? metric(s) : nullptr);  // curvilinear: same launch
        dx.push_back(stp_handle_dx(s.handle));
      }
      // A batch with more than about 50 ms of FP64 work runs as the batched
      // plan's per-shape launches (each body at its single-set kernel's
      // speed: 7 % more requests served on large simulations); a smaller one
      // as the one allocation-free launch, which costs a single launch. N = 12 Cartesian simulations
      // always take the per-shape launch, whose body is the single-set
      // kernel's, so each simulation rounds the same in every batch.
      std::vector<char> curv(N.size());
      for (size_t k = 0; k < N.size(); ++k) curv[k] = mt[k] != nullptr;
      const std::vector<char> form = launch_forms(N, E, curv, 50.0);
      std::vector<size_t> direct, shaped;  // allocation-free launch / per-shape launches
      for (size_t k = 0; k < N.size(); ++k) (form[k] ? shaped : direct).push_back(k);
      int too_big = 0;
      e = cudaEventRecord(sl.start, sl.stream);
      for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        const std::vector<size_t>& idx = pass == 0 ? direct : shaped;
        if (idx.empty()) continue;
        std::vector<int> Ns;
        std::vector<int64_t> Es;
        std::vector<const double*> qs, ps, tbs, mts;
        std::vector<double*> as, fs;
        std::vector<double> dxs;
        for (size_t k : idx) {
          Ns.push_back(N[k]); Es.push_back(E[k]); qs.push_back(q[k]); ps.push_back(p[k]);
          as.push_back(a[k]); fs.push_back(f[k]); tbs.push_back(tb[k]); mts.push_back(mt[k]);
          dxs.push_back(dx[k]);
        }
        e = pass == 0
                ? launch_param_batch((int)Ns.size(), Ns.data(), Es.data(), qs.data(), ps.data(),
                                     as.data(), fs.data(), tbs.data(), sl.scratch,
                                     static_scratch_bytes(), sl.stream, &too_big, mts.data(),
                                     dxs.data())
                : launch_shape_batches((int)Ns.size(), Ns.data(), Es.data(), qs.data(), ps.data(),
                                       as.data(), fs.data(), tbs.data(), mts.data(), dxs.data(),
                                       sl.scratch, static_scratch_bytes(), sl.stream, &too_big);
      }
      for (size_t k = 0; e == cudaSuccess && k < own.size(); ++k) {
        Sim& s = sims[own[k]];
        e = stp_launch_handle(s.handle, s.E, state(s, s.cur), params(s),
                              s.bytes_metric ? metric(s) : nullptr, state(s, s.cur ^ 1), faces(s),
                              sl.stream);
      }
      // point sources: their response added to the new average and faces,
      // on the same stream and before the batch's completion event
      for (int k = 0; e == cudaSuccess && k < n; ++k) {
        Sim& s = sims[batch[k]];
        if (s.sources)
          e = served_sources_launch(s.sources, params(s), s.bytes_metric ? metric(s) : nullptr,
                                    state(s, s.cur ^ 1), faces(s), sl.stream);
      }
      if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
      if (e != cudaSuccess) {
        // nothing of this batch counts as launched: its simulations go back to
        // the front of the ready queue, in their order, so drain() and later
        // passes still see their requests
        requeue_front(batch);
        return e;
      }
      sl.sims = batch;
      sl.busy = true;
      ++batches;
      batched_requests += n;
      max_batch = std::max<int64_t>(max_batch, n);
    }
    return cudaSuccess;
  }

  // Undo the marks of a batch whose launch failed: not running, queued again
  // at the front of the ready queue in their original order.
  void requeue_front(const std::vector<int>& batch) {
    for (auto it = batch.rbegin(); it != batch.rend(); ++it) {
      Sim& s = sims[*it];
      s.busy = false;
      ready.push_front(*it);  // batch members were taken off the queue
      s.queued = true;
    }
  }

  bool idle() const {
    if (!ready.empty()) return false;
    for (const Slot& s : slots)
      if (s.busy) return false;
    return true;
  }

  void release() {
    for (Slot& s : slots) {
      if (s.stream) cudaStreamSynchronize(s.stream);
      cudaFree(s.scratch);
      if (s.done) cudaEventDestroy(s.done);
      if (s.start) cudaEventDestroy(s.start);
      if (s.stream) cudaStreamDestroy(s.stream);
    }
    if (copy_stream) cudaStreamSynchronize(copy_stream);
    if (evict_stream) cudaStreamSynchronize(evict_stream);
    if (copy_done) cudaEventDestroy(copy_done);
    if (evict_done) cudaEventDestroy(evict_done);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    if (evict_stream) cudaStreamDestroy(evict_stream);
    for (Sim& s : sims) {
      cudaFreeHost(s.host_q);
      cudaFreeHost(s.host_params);
      cudaFreeHost(s.host_faces);
      cudaFreeHost(s.host_metric);
      served_sources_free(s.sources);
    }
    cudaFree(pool_base);
  }
};

cudaError_t server_create(int64_t budget, int nslots, Server** out) {
  *out = nullptr;
  Server* s = new (std::nothrow) Server;
  if (!s) return cudaErrorMemoryAllocation;
  cudaGetDevice(&s->device);
  s->budget = (size_t)budget;
  cudaError_t e = cudaMalloc(&s->pool_base, std::max<size_t>(s->budget, kAlign));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->copy_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->evict_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->evict_done, cudaEventDisableTiming);
  s->slots.resize(nslots);
  for (Slot& sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.done);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.start);
    if (e == cudaSuccess) e = cudaMalloc(&sl.scratch, static_scratch_bytes());
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->release();
    delete s;
    return e;
  }
  s->pool.reset(s->budget);
  *out = s;
  return cudaSuccess;
}

void server_destroy(Server* s) {
  if (!s) return;
  s->release();
  delete s;
}

cudaError_t server_add_sim(Server* s, stp_handle h, int N, int64_t E, const double* q0,
                           const double* params, const double* metric, bool device_src, int* id,
                           bool* too_big, ServedSources* sources) {
  *too_big = false;
  Sim sim;
  sim.handle = h;
  sim.sources = sources;  // owned from here on only if this call succeeds
  sim.N = N;
  sim.E = E;
  const size_t n3 = (size_t)N * N * N;
  sim.bytes_state = (size_t)E * n3 * 9 * 8;
  sim.bytes_params = (size_t)E * n3 * 3 * 8;
  sim.bytes_faces = (size_t)E * N * N * 54 * 8;
  sim.bytes_metric = metric ? (size_t)E * n3 * 9 * 8 : 0;
  if (sim.footprint() > s->budget) {
    *too_big = true;
    return cudaErrorInvalidValue;
  }
  size_t off = 0;
  if (device_src && s->pool.alloc(sim.footprint(), &off)) {
    // fits the pool as it is: admitted now by device-to-device copies, with
    // no host copies until its first eviction
    sim.off = off;
    sim.resident = true;
    sim.cur = 0;
    // device-to-device copies return before they complete: they run on the
    // admission stream, which is synchronised before the call returns (the
    // caller may free its buffers then, and the launches that read the pool
    // run on other, non-blocking streams)
    cudaError_t e = cudaMemcpyAsync(s->state(sim, 0), q0, sim.bytes_state, cudaMemcpyDeviceToDevice,
                                    s->copy_stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->params(sim), params, sim.bytes_params, cudaMemcpyDeviceToDevice,
                          s->copy_stream);
    if (e == cudaSuccess && metric)
      e = cudaMemcpyAsync(s->metric(sim), metric, sim.bytes_metric, cudaMemcpyDeviceToDevice,
                          s->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
    if (e != cudaSuccess) {
      s->pool.release(off, sim.footprint());
      return e;
    }
    ++s->admissions;
    s->peak_used = std::max(s->peak_used, s->pool.used());
    *id = (int)s->sims.size();
    s->sims.push_back(sim);
    return cudaSuccess;
  }
  cudaError_t e = s->make_host_backing(sim);
  const cudaMemcpyKind kind = device_src ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  if (e == cudaSuccess) e = cudaMemcpy(sim.host_q, q0, sim.bytes_state, kind);
  if (e == cudaSuccess) e = cudaMemcpy(sim.host_params, params, sim.bytes_params, kind);
  if (e == cudaSuccess && metric) e = cudaMemcpy(sim.host_metric, metric, sim.bytes_metric, kind);
  if (e != cudaSuccess) {
    cudaFreeHost(sim.host_q);
    cudaFreeHost(sim.host_params);
    cudaFreeHost(sim.host_faces);
    cudaFreeHost(sim.host_metric);
    return e;
  }
  *id = (int)s->sims.size();
  s->sims.push_back(sim);
  return cudaSuccess;
}

cudaError_t server_run_trace(Server* s, int64_t n, const double* t_arr, const int* sim_ids,
                             double* latency, double* wall) {
  std::vector<double> completion((size_t)n, -1.0);
  s->completion = &completion;
  s->t0 = Clock::now();
  const int64_t start_completed = s->completed;
  int64_t i = 0;
  cudaError_t e = cudaSuccess;
  while (s->completed - start_completed < n) {
    const double t = s->now();
    while (i < n && t_arr[i] <= t) {
      s->submit(sim_ids[i], i, t_arr[i]);
      ++i;
    }
    int done = 0;
    if ((e = s->progress(&done)) != cudaSuccess) break;
    if (done == 0 && s->idle() && i < n) {
      // nothing in flight: wait for the next arrival without burning a core
      const double wait = t_arr[i] - s->now();
      if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
    }
  }
  if (wall) *wall = s->now();
  s->completion = nullptr;
  for (int64_t k = 0; k < n; ++k) latency[k] = completion[k] - t_arr[k];
  return e;
}

cudaError_t server_drain(Server* s) {
  cudaError_t e = cudaSuccess;
  while (!s->idle())
    if ((e = s->progress(nullptr)) != cudaSuccess) break;
  return e;
}

cudaError_t server_read(Server* s, int id, double* q, double* faces, int64_t* steps) {
  Sim& sim = s->sims[id];
  cudaError_t e = server_drain(s);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s->copy_stream)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s->evict_stream)) != cudaSuccess) return e;
  if (sim.resident) {
    if (q && (e = cudaMemcpy(q, s->state(sim, sim.cur), sim.bytes_state, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return e;
    if (faces && sim.have_faces &&
        (e = cudaMemcpy(faces, s->faces(sim), sim.bytes_faces, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return e;
  } else {
    if (q) std::memcpy(q, sim.host_q, sim.bytes_state);
    if (faces && sim.have_faces) std::memcpy(faces, sim.host_faces, sim.bytes_faces);
  }
  if (steps) *steps = sim.steps;
  return cudaSuccess;
}

void server_stats(const Server* s, int64_t* out) {
  out[0] = s->completed;
  out[1] = s->batches;
  out[2] = s->admissions;
  out[3] = s->evictions;
  out[4] = s->max_batch;
  out[5] = s->batched_requests;
  out[6] = (int64_t)s->pool.used();
  out[7] = (int64_t)s->peak_used;
  out[8] = (int64_t)(s->kernel_ms * 1000.0);  // microseconds
}

void server_submit(Server* s, int id) {
  s->submit(id, -1, s->now());
}

cudaError_t server_progress(Server* s, int* done) { return s->progress(done); }

int server_sims(const Server* s) { return (int)s->sims.size(); }

}  // namespace stp

namespace stp {

void server_set_policy(Server* s, int policy, double age_bound) {
  s->policy = policy;
  s->age_bound = age_bound;
}

}  // namespace stp
