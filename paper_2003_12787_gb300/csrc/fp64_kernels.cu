// FP64 Space-Time Predictor kernels for sm_103a.
//
// One CTA owns EPC whole elements (EPC = 1 from N = 6 up). The element's
// current Taylor term lives in shared memory in structure-of-arrays layout
// p[quantity][node]; every thread owns NPT nodes and, per Cauchy-Kowalewsky
// step, forms the 18 directional derivatives its node needs straight from
// shared memory, combines them with the node's elastic coefficients and adds
// the new term to the running time average. This is the sum-factorised,
// dimension-by-dimension scheme of Sec. IV (SplitCK) with the time average
// accumulated on the fly, mapped onto one SM: the O(N^3 m) live set sits in
// shared memory, the per-node result in registers.
//
// On GB300 the FP64 pipe retires about two DFMA per clock per SM while the
// SM can issue four warp-instructions per clock, so the kernel is built to
// minimise FP64 instructions (elastic sparsity: 6 of 9 quantities per
// direction; dt/((k+2) dx) folded into per-step copies of D; coefficient
// products shared between outputs) and leaves shared-memory traffic, address
// arithmetic and synchronisation in the shadow of the FP64 pipe.
//
// Taylor bookkeeping: r_k = dt^k/(k+1)! q^(k) satisfies r_0 = q,
// r_{k+1} = dt/(k+2) * L r_k with L q = -sum_d B_d (D_d q)/dx, and the time
// average of Eq. (exahypeTimeAverage) divided by dt is sum_{k=0..N} r_k.
#include "fp64_eo.cuh"
#include "fp64_group.cuh"

namespace stp {
namespace {

template <int N, int NPT, int EPC, bool AVG_SMEM>
__global__ void __launch_bounds__(Fp64Shape<N, NPT, EPC, AVG_SMEM>::BLOCK,
                                  Fp64Shape<N, NPT, EPC, AVG_SMEM>::MINB)
fp64_stp_kernel(const double* __restrict__ q, const double* __restrict__ params,
                double* __restrict__ out_avg, double* __restrict__ out_faces,
                const double* __restrict__ tables, int64_t E) {
  extern __shared__ double smem[];
  fp64_group<N, NPT, EPC, AVG_SMEM, Fp64Shape<N, NPT, EPC, AVG_SMEM>::BLOCK>(
      smem, q, params, out_avg, out_faces, tables, (int64_t)blockIdx.x * EPC, E);
}

// Even-odd kernel: one element per CTA of NT threads (USE doing the work).
template <int N, int NT, int USE, int MINB>
__global__ void __launch_bounds__(NT, MINB)
fp64_eo_kernel(const double* __restrict__ q, const double* __restrict__ params,
               double* __restrict__ out_avg, double* __restrict__ out_faces,
               const double* __restrict__ tables, int64_t E) {
  extern __shared__ double smem[];
  fp64_element_eo<N, NT, USE>(smem, q, params, out_avg, out_faces, tables, (int64_t)blockIdx.x);
}

template <int N, int NT, int USE>
__global__ void __launch_bounds__(NT, 1)
fp64_eo_slots_kernel(const double* __restrict__ q, const double* __restrict__ params,
                     double* __restrict__ out_avg, double* __restrict__ out_faces,
                     const double* __restrict__ tables, int64_t E) {
  extern __shared__ double smem[];
  fp64_element_eo_slots<N, NT, USE>(smem, q, params, out_avg, out_faces, tables, (int64_t)blockIdx.x);
}

template <int N, int NT, int USE>
cudaError_t launch_eo_slots(int64_t E, const double* q, const double* params, double* out_avg,
                            double* out_faces, const double* tables, cudaStream_t stream) {
  constexpr size_t smem = EoSlotShape<N>::SMEM;
  static_assert(smem <= 232448, "shared memory budget of one CTA exceeded");
  auto kern = fp64_eo_slots_kernel<N, NT, USE>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (E > 0x7fffffffLL) return cudaErrorInvalidValue;
  kern<<<(unsigned)E, NT, smem, stream>>>(q, params, out_avg, out_faces, tables, E);
  return cudaGetLastError();
}

template <int N, int NT, int USE, int MINB>
cudaError_t launch_eo(int64_t E, const double* q, const double* params, double* out_avg,
                      double* out_faces, const double* tables, cudaStream_t stream) {
  constexpr size_t smem = EoShape<N>::SMEM;
  static_assert(smem <= 232448, "shared memory budget of one CTA exceeded");
  auto kern = fp64_eo_kernel<N, NT, USE, MINB>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (E > 0x7fffffffLL) return cudaErrorInvalidValue;
  kern<<<(unsigned)E, NT, smem, stream>>>(q, params, out_avg, out_faces, tables, E);
  return cudaGetLastError();
}

template <int N, int NPT, int EPC, bool AVG_SMEM>
cudaError_t launch_shape(int64_t E, const double* q, const double* params, double* out_avg,
                         double* out_faces, const double* tables, cudaStream_t stream) {
  using Sh = Fp64Shape<N, NPT, EPC, AVG_SMEM>;
  static_assert(Sh::SMEM <= 232448, "shared memory budget of one CTA exceeded");
  auto kern = fp64_stp_kernel<N, NPT, EPC, AVG_SMEM>;
  // per device context; cheap, and legal while a stream is being captured
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  if (err != cudaSuccess) return err;
  const int64_t blocks = (E + EPC - 1) / EPC;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  kern<<<(unsigned)blocks, Sh::BLOCK, Sh::SMEM, stream>>>(q, params, out_avg, out_faces, tables, E);
  return cudaGetLastError();
}

// Launch shapes per N: nodes per thread, elements per CTA, average in smem.
#define STP_FP64_SHAPES(X) \
  X(1, 1, 64, true)        \
  X(2, 1, 32, true)        \
  X(3, 1, 8, true)         \
  X(4, 1, 4, true)         \
  X(5, 1, 2, true)         \
  X(6, 1, 1, true)         \
  X(7, 2, 1, true)         \
  X(8, 2, 1, true)         \
  X(9, 2, 1, true)         \
  X(10, 2, 1, true)        \
  X(11, 2, 1, false)       \
  X(12, 2, 1, false)

}  // namespace

// Orders that use the even-odd kernel: (N, threads, working threads, CTAs/SM).
// The batched, allocation-free and served paths use the even-odd body for the
// same orders, so every FP64 path rounds alike. From N = 9 on, CTAs with every
// thread working beat the thread counts fitted to the 9 N^2 line tasks; the
// counts below are the fastest of a sweep on GB300 (N = 10: 640 threads,
// 12.29 ms for 4096 elements against 13.02 with 512 and 13.20 with 300 of 320;
// N = 12: 576, 14.39 against 14.58 with 512 and 14.79 with 432 of 448).
#define STP_FP64_EO_SHAPES(X) X(7, 352, 343, 2) X(8, 192, 192, 2) X(9, 512, 512, 1) \
  X(10, 640, 640, 1) X(11, 512, 512, 1)

int fp64_elements_per_cta(int N) {
  switch (N) {
#define X(n, npt, epc, avg) case n: return epc;
    STP_FP64_SHAPES(X)
#undef X
    default: return 1;
  }
}

cudaError_t launch_fp64(int N, int64_t E, const double* q, const double* params,
                        double* out_avg, double* out_faces, const double* tables,
                        cudaStream_t stream) {
  switch (N) {
#define X(n, nt, use, minb) \
  case n: return launch_eo<n, nt, use, minb>(E, q, params, out_avg, out_faces, tables, stream);
    STP_FP64_EO_SHAPES(X)
#undef X
    case 12: return launch_eo_slots<12, 576, 576>(E, q, params, out_avg, out_faces, tables, stream);
    default: break;
  }
  switch (N) {
#define X(n, npt, epc, avg) \
  case n: return launch_shape<n, npt, epc, avg>(E, q, params, out_avg, out_faces, tables, stream);
    STP_FP64_SHAPES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stp
