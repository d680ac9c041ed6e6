// Batched persistent FP64 STP: element sets of different orders and sizes,
// replayed from a captured CUDA graph, with shapes picked by an on-device
// autotuner.
//
// The paper's Kernel Generator tailors each kernel to its order at build time
// (Sec. II-D: generated, order-specific kernels; Sec. III: padding and
// alignment chosen per order). Here every shape (order and CTA layout) is a
// persistent kernel of its own with the FP64 element body inlined; a plan
// groups the sets by shape, and each group's launch consumes its (set,
// element range) units through an atomic counter, the sets' descriptors
// travelling in a kernel-parameter table. The groups' launches, longest
// first, share the GPU over parallel graph branches; each order runs the
// shape the autotuner measured fastest for it on this device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "curv_body.cuh"
#include "fp64_eo.cuh"
#include "fp64_group.cuh"
#include "launch_groups.h"

namespace stp {
namespace {

constexpr int kBatchThreads = 512;

// Candidate shapes per N: (N, index, nodes per thread, elements per CTA,
// average in smem, new term parked in global scratch instead of registers).
// Orders 7..11 use the even-odd body instead (STP_BATCH_EO below): every FP64
// path uses the same arithmetic per order, so results agree bit for bit.
#define STP_BATCH_SHAPES(X)                                                                        \
  X(1, 0, 1, 256, true, false) X(2, 0, 1, 64, true, false) X(2, 1, 2, 128, true, false)           \
  X(3, 0, 1, 18, true, false) X(3, 1, 2, 36, true, false) X(4, 0, 1, 8, true, false)              \
  X(4, 1, 2, 16, true, false) X(5, 0, 1, 4, true, false) X(5, 1, 2, 8, true, false)               \
  X(6, 0, 1, 2, true, false) X(6, 1, 2, 4, true, false)

constexpr int kMaxVariants = 2;

// Even-odd candidates: (N, index, threads, threads doing the work, CTAs per
// SM); shape 0 of N = 7, 8, 10 is the single-set kernel's (N = 7, 8: two CTAs per SM).
// N = 12 uses the slot-reusing variant (p and accumulators share 16 arrays):
// (N, index, threads, threads doing the work).
#define STP_BATCH_EO(X) X(7, 0, 352, 343, 2) X(7, 1, 512, 512, 1) X(8, 0, 192, 192, 2) \
  X(8, 1, 512, 512, 1) X(9, 0, 512, 486, 1) X(9, 1, 512, 512, 1) X(10, 0, 640, 640, 1)  \
  X(10, 1, 512, 512, 1) X(11, 0, 512, 444, 1) X(11, 1, 512, 512, 1)
#define STP_BATCH_EO_SLOTS(X) X(12, 0, 576, 576) X(12, 1, 512, 512)

struct ShapeInfo {
  int valid = 0, epc = 1;
  size_t smem = 0;
  size_t scratch = 0;  // bytes of global scratch per CTA (parked new terms)
  int threads = kBatchThreads;
};

// host-side table of the candidate shapes
struct ShapeTable {
  ShapeInfo s[kMaxNodes + 1][kMaxVariants];
  ShapeTable() {
#define X(n, v, npt, epc, avg, rg)                                                   \
  s[n][v] = ShapeInfo{1, epc, Fp64Shape<n, npt, epc, avg>::SMEM,                     \
                      rg ? sizeof(double) * 9 * (size_t)Fp64Shape<n, npt, epc, avg>::S * epc : 0};
    STP_BATCH_SHAPES(X)
#undef X
#define X(n, v, nt, use, minb) s[n][v] = ShapeInfo{1, 1, EoShape<n>::SMEM, 0, nt};
    STP_BATCH_EO(X)
#undef X
#define X(n, v, nt, use) s[n][v] = ShapeInfo{1, 1, EoSlotShape<n>::SMEM, 0, nt};
    STP_BATCH_EO_SLOTS(X)
#undef X
  }
};
const ShapeTable& shapes() {
  static ShapeTable t;
  return t;
}

struct SetDev {
  const double* q;
  const double* params;
  double* avg;
  double* faces;
  const double* tables;
  int64_t E;
  int N;
  int variant;
  const double* metric;  // curvilinear set: per-node inverse Jacobians; NULL: Cartesian
  double dx;             // the handle's dx (curvilinear sets)
  int64_t first_unit;    // work units of the launch's sets before this one
  int epc;               // elements per work unit
  int pad;
};

// Shared memory and threads of order N's curvilinear shape (0 for other N):
// the single-set kernel's.
size_t curv_batch_smem(int N) {
  switch (N) {
#define X(n_, nt_, nodes_, a_, lean_, greg_, db_) \
  case n_: return CurvShape<n_, a_, db_>::SMEM;
    STP_CURV_SHAPES(X)
#undef X
    default: return 0;
  }
}

int curv_batch_threads(int N) {
  switch (N) {
#define X(n_, nt_, nodes_, a_, lean_, greg_, db_) \
  case n_: return nt_;
    STP_CURV_SHAPES(X)
#undef X
    default: return 0;
  }
}

// Set descriptors of one launch, passed as a kernel parameter: read from the
// parameter space, the buffer pointers reach the element bodies as they do in
// the single-set kernels. Loaded from a device array instead, the same bodies
// ran 7 % slower (N = 12, measured on GB300), spilled or not, persistent or not.
constexpr int kParamSets = 128;
struct SetTable {
  SetDev sets[kParamSets];
};

// The body of one shape over one work unit. Every shape gets a persistent
// kernel of its own (order_kernel<Unit>) with its body inlined, so that its
// register allocation is that of its single-set kernel (hosting every body
// in one kernel, as calls or inlined, capped them at that kernel's 128
// registers and spilled the large-N ones).
template <int N, int NPT, int EPC, bool AVG, bool RG>
struct GroupUnit {
  static constexpr int NT = kBatchThreads, MINB = 1;
  static __device__ __forceinline__ void run(double* smem, const SetDev& sd, int64_t e0,
                                             double* rbuf) {
    fp64_group<N, NPT, EPC, AVG, kBatchThreads, RG>(smem, sd.q, sd.params, sd.avg, sd.faces,
                                                    sd.tables, e0, sd.E, rbuf);
  }
};

template <int N, int THREADS, int USE, int BLOCKS_PER_SM>
struct EoUnit {
  static constexpr int NT = THREADS, MINB = BLOCKS_PER_SM;
  static __device__ __forceinline__ void run(double* smem, const SetDev& sd, int64_t e0, double*) {
    if (e0 < sd.E)
      fp64_element_eo<N, THREADS, USE>(smem, sd.q, sd.params, sd.avg, sd.faces, sd.tables, e0);
  }
};

template <int N, int THREADS, int USE>
struct EoSlotsUnit {
  static constexpr int NT = THREADS, MINB = 1;
  static __device__ __forceinline__ void run(double* smem, const SetDev& sd, int64_t e0, double*) {
    if (e0 < sd.E)
      fp64_element_eo_slots<N, THREADS, USE>(smem, sd.q, sd.params, sd.avg, sd.faces,
                                                   sd.tables, e0);
  }
};

template <int N, int THREADS, int NODES, int A, bool LEAN, bool GREG, bool DB>
struct CurvUnit {
  static constexpr int NT = THREADS, MINB = 1;
  static __device__ __forceinline__ void run(double* smem, const SetDev& sd, int64_t e0, double*) {
    if (e0 < sd.E)
      curv_element<N, THREADS, NODES, A, LEAN, GREG, DB>(
          smem, sd.q, sd.params, sd.metric, sd.avg, sd.faces, sd.tables, sd.dx, e0);
  }
};

// Persistent kernel of one shape: its CTAs take units of its own work list
// (the units of up to kParamSets sets of that shape, set by set; a unit's
// set is found from the sets' first units) through an atomic counter until
// the list is exhausted.
template <class Unit>
__global__ void __launch_bounds__(Unit::NT, Unit::MINB)
order_kernel(const __grid_constant__ SetTable tb, int nsets, int nunits,
             unsigned int* __restrict__ counter, double* __restrict__ scratch,
             int64_t scratch_doubles_per_cta) {
  double* rbuf = scratch ? scratch + blockIdx.x * scratch_doubles_per_cta : nullptr;
  extern __shared__ double smem[];
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) cur = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int u = cur;
    __syncthreads();  // everyone has read cur before thread 0 may overwrite it
    if (u >= nunits) break;
    int lo = 0, hi = nsets - 1;  // the last set whose first unit is <= u
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tb.sets[mid].first_unit <= u) lo = mid; else hi = mid - 1;
    }
    const SetDev& sd = tb.sets[lo];
    Unit::run(smem, sd, (u - sd.first_unit) * sd.epc, rbuf);
  }
}

using OrderKernel = void (*)(const SetTable, int, int, unsigned int*, double*, int64_t);

// Kernel of order N's Cartesian shape v.
OrderKernel cart_kernel(int N, int v) {
  switch (N * kMaxVariants + v) {
#define X(n_, v_, npt_, epc_, avgsm_, rg_) \
  case n_ * kMaxVariants + v_: return order_kernel<GroupUnit<n_, npt_, epc_, avgsm_, rg_>>;
    STP_BATCH_SHAPES(X)
#undef X
#define X(n_, v_, nt_, use_, minb_) \
  case n_ * kMaxVariants + v_: return order_kernel<EoUnit<n_, nt_, use_, minb_>>;
    STP_BATCH_EO(X)
#undef X
#define X(n_, v_, nt_, use_) \
  case n_ * kMaxVariants + v_: return order_kernel<EoSlotsUnit<n_, nt_, use_>>;
    STP_BATCH_EO_SLOTS(X)
#undef X
    default: return nullptr;
  }
}

// Kernel of order N's curvilinear shape.
OrderKernel curv_kernel(int N) {
  switch (N) {
#define X(n_, nt_, nodes_, a_, lean_, greg_, db_) \
  case n_: return order_kernel<CurvUnit<n_, nt_, nodes_, a_, lean_, greg_, db_>>;
    STP_CURV_SHAPES(X)
#undef X
    default: return nullptr;
  }
}

__global__ void fill_kernel(double* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// ---- autotuner ----------------------------------------------------------------

struct Tuned {
  int variant = -1;
  double us_per_element = 0.0;
  double us[kMaxVariants] = {0.0, 0.0};
};
std::mutex g_tune_mutex;
Tuned g_tuned[8][kMaxNodes + 1];  // [device][N]

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// One launch of a shape's persistent kernel over its part of the work list
// (stream operations only, so it can be captured into a graph); the caller
// resets the counter and has raised the kernel's dynamic shared-memory limit
// to at least smem (prepare_kernel).
cudaError_t launch_order(OrderKernel k, int threads, const SetTable& tb, int nsets, int nunits,
                         unsigned int* d_counter, double* scratch, size_t scratch_per_cta,
                         size_t smem, int ctas, cudaStream_t st) {
  k<<<ctas, threads, std::max<size_t>(smem, 1), st>>>(
      tb, nsets, nunits, d_counter, scratch, (int64_t)(scratch_per_cta / sizeof(double)));
  return cudaGetLastError();
}

// Raises kernel k's shared-memory limit to smem; *per_sm = its CTAs per SM.
cudaError_t prepare_kernel(OrderKernel k, int threads, size_t smem, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)std::max<size_t>(smem, 1));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads,
                                                      std::max<size_t>(smem, 1));
  if (e == cudaSuccess && *per_sm < 1) e = cudaErrorInvalidConfiguration;
  return e;
}

}  // namespace

int batch_variants_mask(int N, int* epc_out) {
  int mask = 0;
  for (int v = 0; v < kMaxVariants; ++v)
    if (N >= 1 && N <= kMaxNodes && shapes().s[N][v].valid) {
      mask |= 1 << v;
      if (epc_out) epc_out[v] = shapes().s[N][v].epc;
    }
  return mask;
}

int batch_variants(int N, int* epc_out) {
  int n = 0;
  for (int v = 0; v < kMaxVariants; ++v)
    if (N >= 1 && N <= kMaxNodes && shapes().s[N][v].valid) {
      if (epc_out) epc_out[n] = shapes().s[N][v].epc;
      ++n;
    }
  return n;
}

// Time every candidate shape of order N on a synthetic set (zero state,
// unit material) with its persistent kernel; keep the fastest per device.
cudaError_t autotune(int N, const double* tables, int* variant, double* us_per_element,
                     double* us_all) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 8 || N < 1 || N > kMaxNodes) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  Tuned& t = g_tuned[dev][N];
  if (t.variant < 0) {
    const int sms = sm_count();
    // about 1.5e10 algorithmic flops (~12 ms) per timed launch, at least 4 units per SM
    const double F = 36.0 * std::pow(N, 5) + 66.0 * std::pow(N, 4) + 108.0 * std::pow(N, 3);
    int64_t E = (int64_t)std::max(1.5e10 / F, 0.0);
    int maxepc = 1;
    for (int v = 0; v < kMaxVariants; ++v)
      if (shapes().s[N][v].valid) maxepc = std::max(maxepc, shapes().s[N][v].epc);
    E = std::max<int64_t>(E, (int64_t)4 * sms * maxepc);
    E = std::min<int64_t>(E, 100000);
    const size_t n3 = (size_t)N * N * N;
    double *q = nullptr, *p = nullptr, *a = nullptr, *f = nullptr;
    unsigned int* d_counter = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t e) { if (err == cudaSuccess && e != cudaSuccess) err = e; return err == cudaSuccess; };
    chk(cudaMalloc(&q, E * n3 * 9 * 8));
    chk(cudaMalloc(&p, E * n3 * 3 * 8));
    chk(cudaMalloc(&a, E * n3 * 9 * 8));
    chk(cudaMalloc(&f, E * (size_t)N * N * 54 * 8));
    chk(cudaMalloc(&d_counter, sizeof(unsigned int)));
    size_t scr = 0;
    for (int v = 0; v < kMaxVariants; ++v)
      if (shapes().s[N][v].valid) scr = std::max(scr, shapes().s[N][v].scratch);
    double* scratch = nullptr;
    if (scr) chk(cudaMalloc(&scratch, scr * (size_t)sms * 4));  // up to 4 CTAs of 512 threads per SM
    chk(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    chk(cudaEventCreate(&e0));
    chk(cudaEventCreate(&e1));
    if (err == cudaSuccess) {
      chk(cudaMemsetAsync(q, 0, E * n3 * 9 * 8, st));
      fill_kernel<<<1024, 256, 0, st>>>(p, (int64_t)(E * n3 * 3), 1.0);
      chk(cudaGetLastError());
    }
    double best = 1e300;
    for (int v = 0; v < kMaxVariants && err == cudaSuccess; ++v) {
      const ShapeInfo& si = shapes().s[N][v];
      if (!si.valid) continue;
      SetTable tb{};
      tb.sets[0] = SetDev{q, p, a, f, tables, E, N, v, nullptr, 0.0, 0, si.epc, 0};
      const int nunits = (int)((E + si.epc - 1) / si.epc);
      float ms_best = 1e30f;
      const OrderKernel k = cart_kernel(N, v);
      int per_sm = 1;
      chk(prepare_kernel(k, si.threads, si.smem, &per_sm));
      const int ctas = (int)std::min<int64_t>((int64_t)per_sm * sms, nunits);
      for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
        chk(cudaMemsetAsync(d_counter, 0, sizeof(unsigned int), st));
        chk(cudaEventRecord(e0, st));
        chk(launch_order(k, si.threads, tb, 1, nunits, d_counter, scratch, scr, si.smem, ctas, st));
        chk(cudaEventRecord(e1, st));
        chk(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_best = std::min(ms_best, ms);  // first launch warms up
      }
      const double us = 1e3 * ms_best / (double)E;
      t.us[v] = us;
      if (us < best) { best = us; t.variant = v; t.us_per_element = us; }
    }
    if (st) cudaStreamSynchronize(st);
    cudaFree(q); cudaFree(p); cudaFree(a); cudaFree(f);
    cudaFree(d_counter); cudaFree(scratch);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (err != cudaSuccess) { t.variant = -1; return err; }
  }
  if (variant) *variant = t.variant;
  if (us_per_element) *us_per_element = t.us_per_element;
  if (us_all)
    for (int v = 0; v < kMaxVariants; ++v) us_all[v] = t.us[v];
  return cudaSuccess;
}

// ---- launches -----------------------------------------------------------------

namespace {

// One persistent launch: up to kParamSets sets of one shape (one order,
// Cartesian shape v or curvilinear), their units numbered set by set.
struct Launch {
  OrderKernel kernel = nullptr;
  int threads = kBatchThreads;
  SetTable table{};
  int nsets = 0;
  size_t smem = 0, scratch_per_cta = 0, scratch_off = 0;  // scratch_off in doubles
  int64_t count = 0;  // work units
  double cost = 0.0;  // estimated us of the whole launch
  int ctas = 0, branch = 0;
};

// A shape's kernel, block size, shared memory and parking scratch per CTA.
struct ShapeRef {
  OrderKernel kernel = nullptr;
  int threads = kBatchThreads;
  size_t smem = 0, scratch_per_cta = 0;
};

// Shape of a set: its kernel, block size, shared memory, parking scratch per
// CTA, elements per unit and estimated us per unit. variant < 0 for a
// Cartesian set picks the autotuned shape (tuning the order first when
// `tune`, else the cached choice or a default that allocates nothing).
cudaError_t set_shape(int N, const double* tables, bool curvilinear, int variant, bool tune,
                      ShapeRef* shape, int* v_out, int* epc, double* unit_us) {
  if (N < 1 || N > kMaxNodes) return cudaErrorInvalidValue;
  const double F = 36.0 * std::pow(N, 5) + 66.0 * std::pow(N, 4) + 108.0 * std::pow(N, 3);
  if (curvilinear) {
    shape->kernel = curv_kernel(N);
    shape->threads = curv_batch_threads(N);
    shape->smem = curv_batch_smem(N);
    shape->scratch_per_cta = 0;
    *v_out = 0;
    *epc = 1;
    *unit_us = 1.7 * F / 1.2e6;  // every quantity along every direction
    return shape->kernel ? cudaSuccess : cudaErrorInvalidValue;
  }
  int v = variant;
  double us = F / 1.2e6;  // FP64-bound estimate
  if (v < 0 && tune) {
    cudaError_t err = autotune(N, tables, &v, &us, nullptr);
    if (err != cudaSuccess) return err;
  } else if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (dev >= 0 && dev < 8 && g_tuned[dev][N].variant >= 0) {
      v = g_tuned[dev][N].variant;
      us = g_tuned[dev][N].us_per_element;
    } else {
      // the shapes the autotuner picks on GB300
      static const int kDefault[kMaxNodes + 1] = {0, 0, 0, 0, 0, 1, 1, 0, 0, 1, 0, 1, 0};
      v = kDefault[N];
    }
  }
  if (v < 0 || v >= kMaxVariants || !shapes().s[N][v].valid) return cudaErrorInvalidValue;
  const ShapeInfo& si = shapes().s[N][v];
  shape->kernel = cart_kernel(N, v);
  shape->threads = si.threads;
  shape->smem = si.smem;
  shape->scratch_per_cta = si.scratch;
  *v_out = v;
  *epc = si.epc;
  *unit_us = us * si.epc;
  return shape->kernel ? cudaSuccess : cudaErrorInvalidValue;
}

// Groups the sets by shape into launches (at most kParamSets sets each, in set
// order), longest first; sets without elements are left out (launch_groups.h).
cudaError_t build_launches(int nsets, const int* N, const int64_t* E, const double* const* q,
                           const double* const* params, double* const* avg,
                           double* const* faces, const double* const* tables,
                           const int* forced_variant, const double* const* metrics,
                           const double* dx, bool tune, std::vector<Launch>* out) {
  constexpr int kCurvKey = (kMaxNodes + 1) * kMaxVariants;
  std::vector<ShapeRef> shape((size_t)nsets);
  std::vector<SetDev> sets((size_t)nsets);
  std::vector<GroupInput> in((size_t)nsets);
  for (int i = 0; i < nsets; ++i) {
    const bool curv = metrics && metrics[i];
    int v = 0, epc = 1;
    double unit_us = 0.0;
    cudaError_t err = set_shape(N[i], tables[i], curv, forced_variant ? forced_variant[i] : -1,
                                tune, &shape[i], &v, &epc, &unit_us);
    if (err != cudaSuccess) return err;
    sets[i] = SetDev{q[i], params[i], avg[i], faces[i], tables[i], E[i], N[i], v,
                     curv ? metrics[i] : nullptr, curv && dx ? dx[i] : 0.0, 0, epc, 0};
    in[i] = GroupInput{curv ? kCurvKey + N[i] : N[i] * kMaxVariants + v,
                       E[i] > 0 ? (E[i] + epc - 1) / epc : 0, unit_us};
  }
  const std::vector<LaunchGroup> groups = group_launches(in, kParamSets);
  out->reserve(out->size() + groups.size());
  for (const LaunchGroup& g : groups) {
    if (g.count > 0x7fffffffLL) return cudaErrorInvalidValue;
    out->emplace_back();
    Launch& l = out->back();
    const ShapeRef& sh = shape[(size_t)g.sets[0]];
    l.kernel = sh.kernel;
    l.threads = sh.threads;
    l.smem = sh.smem;
    l.scratch_per_cta = sh.scratch_per_cta;
    l.nsets = (int)g.sets.size();
    for (int k = 0; k < l.nsets; ++k) {
      l.table.sets[k] = sets[(size_t)g.sets[(size_t)k]];
      l.table.sets[k].first_unit = g.first_unit[(size_t)k];
    }
    l.count = g.count;
    l.cost = g.cost;
  }
  return cudaSuccess;
}

// CTAs per SM of each kernel at its shared memory, set up once per device.
std::mutex g_occ_mutex;
std::vector<std::pair<std::pair<int, OrderKernel>, int>> g_occ;

cudaError_t kernel_ctas_per_sm(OrderKernel k, int threads, size_t smem, int* per_sm) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_occ_mutex);
  for (const auto& e : g_occ)
    if (e.first.first == dev && e.first.second == k) { *per_sm = e.second; return cudaSuccess; }
  cudaError_t err = prepare_kernel(k, threads, smem, per_sm);
  if (err == cudaSuccess) g_occ.push_back({{dev, k}, *per_sm});
  return err;
}

}  // namespace

// ---- plans ------------------------------------------------------------------

constexpr int kMaxBranches = 4;

struct BatchPlan {
  int device = -1;
  int nsets = 0, nunits = 0, ctas = 0;
  size_t smem = 0;
  unsigned int* d_counter = nullptr;  // one per launch
  double* d_scratch = nullptr;        // parked new terms of the large-N shapes, per CTA
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

void destroy_plan(BatchPlan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  cudaFree(p->d_counter);
  cudaFree(p->d_scratch);
  delete p;
}

// Groups the sets by shape (at most kParamSets per launch) and captures into a
// CUDA graph the counters' reset and one persistent launch per group, spread
// over up to kMaxBranches parallel branches (longest first, each to the
// branch with the least estimated work). Launches on different branches run
// concurrently: one shape's CTAs take the SMs that another's finished CTAs
// free, so no SM waits out a shape's tail. forced_variant[i] < 0 = autotuned.
cudaError_t create_plan(int nsets, const int* N, const int64_t* E, const double* const* q,
                        const double* const* params, double* const* avg, double* const* faces,
                        const double* const* tables, const int* forced_variant, BatchPlan** out,
                        const double* const* metrics, const double* dx) {
  *out = nullptr;
  BatchPlan* p = new (std::nothrow) BatchPlan;
  if (!p) return cudaErrorMemoryAllocation;
  cudaGetDevice(&p->device);
  std::vector<Launch> launches;
  cudaError_t err = build_launches(nsets, N, E, q, params, avg, faces, tables, forced_variant,
                                   metrics, dx, true, &launches);
  // grids, branches, scratch
  size_t scratch_doubles = 0;
  int64_t units = 0;
  if (err == cudaSuccess) {
    const int sms = sm_count();
    std::vector<double> costs;
    for (const Launch& l : launches) costs.push_back(l.cost);
    const std::vector<int> branch = lpt_branches(costs, kMaxBranches);
    for (size_t li = 0; li < launches.size(); ++li) {
      Launch& l = launches[li];
      int per_sm = 1;
      if ((err = kernel_ctas_per_sm(l.kernel, l.threads, l.smem, &per_sm)) != cudaSuccess) break;
      l.ctas = (int)std::min<int64_t>((int64_t)per_sm * sms, l.count);
      l.branch = branch[li];
      l.scratch_off = scratch_doubles;
      scratch_doubles += l.scratch_per_cta / sizeof(double) * (size_t)l.ctas;
      p->ctas += l.ctas;
      p->smem = std::max(p->smem, l.smem);
      units += l.count;
    }
  }
  if (err == cudaSuccess && units > 0x7fffffffLL) err = cudaErrorInvalidValue;
  p->nsets = nsets;
  p->nunits = (int)units;
  if (err == cudaSuccess)
    err = cudaMalloc(&p->d_counter, sizeof(unsigned int) * std::max<size_t>(1, launches.size()));
  if (err == cudaSuccess && scratch_doubles)
    err = cudaMalloc(&p->d_scratch, sizeof(double) * scratch_doubles);
  // capture: reset, fork, one launch per group on its branch, join
  cudaStream_t st = nullptr;
  cudaStream_t br[kMaxBranches] = {nullptr};
  cudaEvent_t fork = nullptr, join[kMaxBranches] = {nullptr};
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (int b = 0; b < kMaxBranches && err == cudaSuccess; ++b) {
    err = cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming);
  }
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    cudaError_t le = cudaSuccess;
    if (!launches.empty()) {
      le = cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned int) * launches.size(), st);
      if (le == cudaSuccess) le = cudaEventRecord(fork, st);
      bool used[kMaxBranches] = {false};
      for (const Launch& l : launches) used[l.branch] = true;
      for (int b = 0; b < kMaxBranches && le == cudaSuccess; ++b)
        if (used[b]) le = cudaStreamWaitEvent(br[b], fork, 0);
      for (size_t li = 0; li < launches.size() && le == cudaSuccess; ++li) {
        const Launch& l = launches[li];
        le = launch_order(l.kernel, l.threads, l.table, l.nsets, (int)l.count, p->d_counter + li,
                          p->d_scratch ? p->d_scratch + l.scratch_off : nullptr, l.scratch_per_cta,
                          l.smem, l.ctas, br[l.branch]);
      }
      for (int b = 0; b < kMaxBranches && le == cudaSuccess; ++b)
        if (used[b]) {
          le = cudaEventRecord(join[b], br[b]);
          if (le == cudaSuccess) le = cudaStreamWaitEvent(st, join[b], 0);
        }
    }
    err = cudaStreamEndCapture(st, &p->graph);
    if (le != cudaSuccess) err = le;
  }
  if (err == cudaSuccess) err = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (fork) cudaEventDestroy(fork);
  for (int b = 0; b < kMaxBranches; ++b) {
    if (join[b]) cudaEventDestroy(join[b]);
    if (br[b]) cudaStreamDestroy(br[b]);
  }
  if (st) cudaStreamDestroy(st);
  if (err != cudaSuccess) {
    cudaGetLastError();
    destroy_plan(p);
    return err;
  }
  *out = p;
  return cudaSuccess;
}

// The same per-shape persistent launches issued directly on `stream`, one
// after another, with caller-provided scratch (counters, then the parking
// areas): no allocation, no graph. Used by the served loop for large batches.
cudaError_t launch_shape_batches(int nsets, const int* N, const int64_t* E,
                                 const double* const* q, const double* const* params,
                                 double* const* avg, double* const* faces,
                                 const double* const* tables, const double* const* metrics,
                                 const double* dx, unsigned char* scratch, size_t scratch_bytes,
                                 cudaStream_t stream, int* too_big) {
  *too_big = 0;
  std::vector<Launch> launches;
  cudaError_t err = build_launches(nsets, N, E, q, params, avg, faces, tables, nullptr, metrics,
                                   dx, false, &launches);
  if (err != cudaSuccess || launches.empty()) return err;
  constexpr size_t kCounters = 256;  // bytes of counters at the start of scratch
  if (launches.size() * sizeof(unsigned int) > kCounters) { *too_big = 1; return cudaErrorInvalidValue; }
  const int sms = sm_count();
  size_t off = kCounters;
  for (Launch& l : launches) {
    int per_sm = 1;
    if ((err = kernel_ctas_per_sm(l.kernel, l.threads, l.smem, &per_sm)) != cudaSuccess) return err;
    l.ctas = (int)std::min<int64_t>((int64_t)per_sm * sms, l.count);
    l.scratch_off = off;  // bytes here
    off += l.scratch_per_cta * (size_t)l.ctas;
  }
  if (off > scratch_bytes) { *too_big = 1; return cudaErrorInvalidValue; }
  unsigned int* counters = reinterpret_cast<unsigned int*>(scratch);
  if ((err = cudaMemsetAsync(counters, 0, sizeof(unsigned int) * launches.size(), stream)) != cudaSuccess)
    return err;
  for (size_t li = 0; li < launches.size() && err == cudaSuccess; ++li) {
    const Launch& l = launches[li];
    double* park = l.scratch_per_cta ? reinterpret_cast<double*>(scratch + l.scratch_off) : nullptr;
    err = launch_order(l.kernel, l.threads, l.table, l.nsets, (int)l.count, counters + li, park,
                       l.scratch_per_cta, l.smem, l.ctas, stream);
  }
  return err;
}

cudaError_t launch_plan(BatchPlan* p, cudaStream_t stream) {
  if (p->nunits == 0) return cudaSuccess;
  return cudaGraphLaunch(p->exec, stream);
}

void plan_info(const BatchPlan* p, int* units, int* ctas, size_t* smem) {
  if (units) *units = p->nunits;
  if (ctas) *ctas = p->ctas;
  if (smem) *smem = p->smem;
}

}  // namespace stp
