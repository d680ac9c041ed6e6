// Batched FP64 predictor that allocates nothing: stp_batch_run_static.
//
// Who needs it: code that must not call cudaMalloc at the point where it runs
// the predictor - for example a caller that owns every byte of device memory
// through its own pool and forbids other allocations, a host thread that may
// not take the implicit device synchronisation cudaMalloc/cudaFree can bring,
// or a process that has already handed the rest of the device to someone
// else. The regular batched path (stp_batch_create) allocates its work list,
// its work counter and its scratch buffers; this entry point instead keeps its
// scratch (the work counter and the per-CTA parking area for new Taylor terms)
// in one fixed-size array that is part of the library's device image, and
// passes the set descriptors as kernel parameters.
//
// The paper has no counterpart to this entry point.
#include <algorithm>
#include <mutex>

#include "curv_body.cuh"
#include "fp64_eo.cuh"
#include "fp64_group.cuh"

namespace stp {
namespace {

constexpr int kStaticThreads = 512;
constexpr int kStaticMaxSets = 128;
// Scratch for one call: the work counter (first 256 bytes), then one parking
// area per CTA of 9*S*EPC doubles for the order whose shape parks new terms
// (N = 12: 124.5 KB per CTA). 24 MiB covers one CTA per SM for
// every order up to 190 SMs.
constexpr size_t kStaticScratchBytes = (size_t)24 << 20;
constexpr size_t kCounterBytes = 256;

// File-scope scratch. Every GPU that loads the library holds it until the
// process exits. In host code its name is only a host-side stand-in: the
// device address comes from cudaGetSymbolAddress (see scratch_address).
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// One fixed shape per order (512 threads): (N, nodes per thread, elements per
// CTA, average in smem, new terms parked in scratch).
#define STP_STATIC_SHAPES(X)                                                                      \
  X(1, 1, 256, true, false) X(2, 1, 64, true, false) X(3, 1, 18, true, false)                    \
  X(4, 1, 8, true, false) X(5, 1, 4, true, false) X(6, 1, 2, true, false)                       \
  X(12, 4, 1, false, true)
// Orders 7..11: the even-odd body (N, threads doing the work), as on every other
// FP64 path. N = 12 keeps the per-node body here, which parks its new terms in
// the scratch array; at N = 12 this path (and the served one, which launches
// this kernel) therefore agrees with stp_predict to rounding, not bit for bit.
#define STP_STATIC_EO(X) X(7, 343) X(8, 384) X(9, 512) X(10, 512) X(11, 512)

struct StaticSet {
  const double* q;
  const double* params;
  double* avg;
  double* faces;
  const double* tables;
  int64_t E;
  int64_t first_unit;  // units of the sets before this one
  int N;
  int epc;
  const double* metric;  // curvilinear set: per-node inverse Jacobians; NULL: Cartesian
  double dx;             // the handle's dx (curvilinear sets)
};

struct StaticBatch {
  StaticSet sets[kStaticMaxSets];
  int nsets;
  int64_t nunits;
};

template <int N, int USE>
__device__ __noinline__ void static_unit_eo(double* smem, const StaticSet& sd, int64_t e0) {
  if (e0 < sd.E)
    fp64_element_eo<N, kStaticThreads, USE>(smem, sd.q, sd.params, sd.avg, sd.faces, sd.tables, e0);
}

template <int N, int NPT, int EPC, bool AVG, bool RG>
__device__ __noinline__ void static_unit(double* smem, const StaticSet& sd, int64_t e0, double* rbuf) {
  fp64_group<N, NPT, EPC, AVG, kStaticThreads, RG>(smem, sd.q, sd.params, sd.avg, sd.faces,
                                                   sd.tables, e0, sd.E, rbuf);
}

template <int N, int NODES, int A, bool LEAN>
__device__ __noinline__ void static_unit_curv(double* smem, const StaticSet& sd, int64_t e0) {
  if (e0 < sd.E)
    curv_element<N, kStaticThreads, NODES, A, LEAN, false, false>(
        smem, sd.q, sd.params, sd.metric, sd.avg, sd.faces, sd.tables, sd.dx, e0);
}

__global__ void __launch_bounds__(kStaticThreads, 1)
static_batch_kernel(const __grid_constant__ StaticBatch b, unsigned char* scratch,
                    int64_t park_doubles_per_cta) {
  extern __shared__ double smem[];
  __shared__ long long cur;
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(scratch);
  double* rbuf = reinterpret_cast<double*>(scratch + kCounterBytes) + blockIdx.x * park_doubles_per_cta;
  for (;;) {
    if (threadIdx.x == 0) cur = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t u = cur;
    __syncthreads();
    if (u >= b.nunits) break;
    int lo = 0, hi = b.nsets - 1;  // last set whose first unit is <= u
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.sets[mid].first_unit <= u) lo = mid; else hi = mid - 1;
    }
    const StaticSet& sd = b.sets[lo];
    const int64_t e0 = (u - sd.first_unit) * sd.epc;
    if (sd.metric) {  // a curvilinear set, one element per unit
      switch (sd.N) {
#define X(n_, nodes_, a_, lean_) \
  case n_: static_unit_curv<n_, nodes_, a_, lean_>(smem, sd, e0); break;
        STP_CURV512_SHAPES(X)
#undef X
        default: break;
      }
      continue;
    }
    switch (sd.N) {
#define X(n_, npt_, epc_, avg_, rg_) \
  case n_: static_unit<n_, npt_, epc_, avg_, rg_>(smem, sd, e0, rbuf); break;
      STP_STATIC_SHAPES(X)
#undef X
#define X(n_, use_) \
  case n_: static_unit_eo<n_, use_>(smem, sd, e0); break;
      STP_STATIC_EO(X)
#undef X
      default: break;
    }
  }
}

struct StaticShape {
  int epc = 0;
  size_t smem = 0, park = 0;
};

StaticShape static_shape(int N, bool curvilinear) {
  if (curvilinear) {
    switch (N) {
#define X(n_, nodes_, a_, lean_) \
  case n_: return StaticShape{1, CurvShape<n_, a_, false>::SMEM, 0};
      STP_CURV512_SHAPES(X)
#undef X
      default: return StaticShape{};
    }
  }
  switch (N) {
#define X(n_, npt_, epc_, avg_, rg_)                                                              \
  case n_:                                                                                       \
    return StaticShape{epc_, Fp64Shape<n_, npt_, epc_, avg_>::SMEM,                              \
                       rg_ ? sizeof(double) * 9 * (size_t)Fp64Shape<n_, npt_, epc_, avg_>::S * epc_ \
                           : 0};
    STP_STATIC_SHAPES(X)
#undef X
#define X(n_, use_) \
  case n_: return StaticShape{1, EoShape<n_>::SMEM, 0};
    STP_STATIC_EO(X)
#undef X
    default: return StaticShape{};
  }
}

// Largest dynamic shared memory over every shape of the kernel. The kernel's
// attribute is set to this one value (never to a call's own need), so calls
// on different host threads - the allocation-free entry and the served loop
// - cannot lower it between another call's set and its launch.
size_t max_static_smem() {
  size_t m = 1;
#define X(n_, npt_, epc_, avg_, rg_) m = std::max(m, (size_t)Fp64Shape<n_, npt_, epc_, avg_>::SMEM);
  STP_STATIC_SHAPES(X)
#undef X
#define X(n_, use_) m = std::max(m, (size_t)EoShape<n_>::SMEM);
  STP_STATIC_EO(X)
#undef X
#define X(n_, nodes_, a_, lean_) m = std::max(m, (size_t)CurvShape<n_, a_, false>::SMEM);
  STP_CURV512_SHAPES(X)
#undef X
  return m;
}

// Identity of the calling thread's current CUDA context, through the driver
// entry points the runtime exposes (no link-time dependency on the driver
// library). A context created after cudaDeviceReset, or after the primary
// context was released and retained again, gets a new identifier, and the
// module holding the scratch array may then sit at a new address.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
std::once_flag g_driver_once;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

bool current_context_id(unsigned long long* id) {
  std::call_once(g_driver_once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
  });
  if (!g_ctx_get_current || !g_ctx_get_id) return false;
  void* ctx = nullptr;
  if (g_ctx_get_current(&ctx) != 0 || !ctx) return false;
  return g_ctx_get_id(ctx, id) == 0;
}

// Per device: the context the cached address belongs to, and the address.
struct ScratchAddr {
  unsigned long long ctx_id = 0;
  unsigned char* addr = nullptr;
};
std::mutex g_addr_mutex;
ScratchAddr g_addr[64];

// Device address of the scratch array for the current context of device
// `dev` (which must be current). The set-up - cudaGetSymbolAddress, and the
// kernel's shared-memory attribute - runs on the first call in each context
// and is cached with that context's identifier; a later call in a new context
// (after a device reset) repeats it. If the context's identity cannot be
// read, the address is looked up on every call.
cudaError_t scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  // a runtime call on the kernel makes the device's context current (creating
  // it on first use) before its identity is read
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, static_batch_kernel);
  if (e != cudaSuccess) return e;
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  ScratchAddr& c = g_addr[dev];
  if (!have_id || !c.addr || c.ctx_id != id) {
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_static_scratch)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(static_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)max_static_smem())) != cudaSuccess)
      return e;
    c.addr = static_cast<unsigned char*>(p);
    c.ctx_id = have_id ? id : 0;
  }
  *out = c.addr;
  return cudaSuccess;
}

}  // namespace

size_t static_scratch_bytes() { return kStaticScratchBytes; }
int static_max_sets() { return kStaticMaxSets; }

// One persistent launch over up to 128 sets described in kernel parameters,
// with the given scratch (work counter + parking areas). Inputs validated by
// the caller. Returns cudaErrorInvalidValue with *too_big = 1 when nsets or
// the needed scratch exceed the limits.
cudaError_t launch_param_batch(int nsets, const int* N, const int64_t* E, const double* const* q,
                               const double* const* params, double* const* avg,
                               double* const* faces, const double* const* tables,
                               unsigned char* scratch, size_t scratch_bytes, cudaStream_t stream,
                               int* too_big, const double* const* metrics, const double* dx) {
  *too_big = 0;
  if (nsets < 0 || nsets > kStaticMaxSets) { *too_big = 1; return cudaErrorInvalidValue; }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  StaticBatch b;
  b.nsets = nsets;
  int64_t units = 0;
  size_t smem = 1, park = 0;
  for (int i = 0; i < nsets; ++i) {
    const double* m = metrics ? metrics[i] : nullptr;
    const StaticShape sh = static_shape(N[i], m != nullptr);
    if (sh.epc == 0) return cudaErrorInvalidValue;
    b.sets[i] = StaticSet{q[i], params[i], avg[i], faces[i], tables[i], E[i], units, N[i], sh.epc,
                          m, m && dx ? dx[i] : 0.0};
    units += (E[i] + sh.epc - 1) / sh.epc;
    if (E[i] > 0) {
      smem = std::max(smem, sh.smem);
      park = std::max(park, sh.park);
    }
  }
  b.nunits = units;
  if (units == 0) return cudaSuccess;
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the attribute is the largest shape's, set to that one value on every call
  // (an idempotent set, so a call on another thread cannot lower it)
  if ((e = cudaFuncSetAttribute(static_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)max_static_smem())) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, static_batch_kernel,
                                                         kStaticThreads, smem)) != cudaSuccess)
    return e;
  int64_t ctas = (int64_t)std::max(1, per_sm) * sms;
  ctas = std::min<int64_t>(ctas, units);
  if (kCounterBytes + (size_t)ctas * park > scratch_bytes) { *too_big = 1; return cudaErrorInvalidValue; }
  // the counter must start at zero; the parking areas need no clearing (each
  // parked value is written before it is read within the same work unit)
  if ((e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), stream)) != cudaSuccess) return e;
  static_batch_kernel<<<(unsigned)ctas, kStaticThreads, smem, stream>>>(
      b, scratch, (int64_t)(park / sizeof(double)));
  return cudaGetLastError();
}

}  // namespace stp

namespace stp {

// sets_N/E/...: validated by the caller. The persistent launch uses the
// array below its top `reserve_top` bytes (which hold the caller's
// point-source data, see static_scratch_top). Returns cudaErrorInvalidValue
// with *too_big = 1 when the call needs more scratch than that.
cudaError_t run_static_batch(int nsets, const int* N, const int64_t* E, const double* const* q,
                             const double* const* params, double* const* avg,
                             double* const* faces, const double* const* tables,
                             cudaStream_t stream, int* too_big, size_t reserve_top,
                             const double* const* metrics, const double* dx) {
  *too_big = 0;
  if (reserve_top > kStaticScratchBytes - kCounterBytes) {
    *too_big = 1;
    return cudaErrorInvalidValue;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  unsigned char* scratch = nullptr;
  if ((e = scratch_address(dev, &scratch)) != cudaSuccess) return e;
  return launch_param_batch(nsets, N, E, q, params, avg, faces, tables, scratch,
                            kStaticScratchBytes - reserve_top, stream, too_big, metrics, dx);
}

// Device address of the top `bytes` of the static array (bytes a multiple of
// 256): where the allocation-free path keeps point-source data.
cudaError_t static_scratch_top(size_t bytes, unsigned char** out) {
  if (bytes > kStaticScratchBytes - kCounterBytes || (bytes & 255u)) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  unsigned char* scratch = nullptr;
  if ((e = scratch_address(dev, &scratch)) != cudaSuccess) return e;
  *out = scratch + (kStaticScratchBytes - bytes);
  return cudaSuccess;
}

}  // namespace stp
