// FP64 Space-Time Predictor on curvilinear elements: one element per CTA,
// with launch shapes per order. The element body (the chain rule through the
// per-node inverse Jacobian, Sec. VI's curvilinear setting) is curv_element
// in curv_body.cuh, which the batched persistent kernel runs too.
#include "curv_body.cuh"

namespace stp {
namespace {

// One element per CTA.
template <int N, int NT, int NODES, int A, bool LEAN, bool GREG, bool DB>
__global__ void __launch_bounds__(NT, 1)
curv_eo_kernel(const double* __restrict__ q, const double* __restrict__ params,
               const double* __restrict__ metric, double* __restrict__ out_avg,
               double* __restrict__ out_faces, const double* __restrict__ tables, double dx) {
  extern __shared__ double smem[];
  curv_element<N, NT, NODES, A, LEAN, GREG, DB>(smem, q, params, metric, out_avg, out_faces, tables,
                                               dx, blockIdx.x);
}

template <int N, int NT, int NODES, int A, bool LEAN, bool GREG, bool DB>
cudaError_t launch_curv_n(int64_t E, const double* q, const double* params, const double* metric,
                          double* out_avg, double* out_faces, const double* tables, double dx,
                          cudaStream_t stream) {
  constexpr size_t smem = CurvShape<N, A, DB>::SMEM;
  static_assert(smem <= 232448, "shared memory budget of one CTA exceeded");
  auto kern = curv_eo_kernel<N, NT, NODES, A, LEAN, GREG, DB>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (E > 0x7fffffffLL) return cudaErrorInvalidValue;
  kern<<<(unsigned)E, NT, smem, stream>>>(q, params, metric, out_avg, out_faces, tables, dx);
  return cudaGetLastError();
}

}  // namespace

// Launch shapes per N: threads, nodes per thread, quantities per line pass,
// lean register state, metric in registers, double buffer (measured on GB300 among 2-6
// candidates per N; from N = 7 on, enough threads that the 9 N^2 line tasks of
// a pass take one or two even rounds).
#define STP_CURV_SHAPES(X)                                                                     \
  X(1, 32, 1, 9, false, false, false) X(2, 32, 1, 9, false, false, false)                       \
  X(3, 32, 1, 9, false, false, false) X(4, 64, 1, 9, false, false, false)                       \
  X(5, 128, 1, 9, false, false, false) X(6, 224, 1, 9, false, false, false)                     \
  X(7, 448, 1, 9, false, true, true) X(8, 576, 1, 9, false, false, true)                        \
  X(9, 384, 2, 9, false, true, true) X(10, 512, 2, 9, true, true, false)                        \
  X(11, 448, 3, 9, true, false, false) X(12, 448, 4, 5, true, false, false)

cudaError_t launch_curvilinear(int N, int64_t E, const double* q, const double* params,
                               const double* metric, double* out_avg, double* out_faces,
                               const double* tables, double dx, cudaStream_t stream) {
  if (E <= 0) return cudaSuccess;
  switch (N) {
#define X(n, nt, nodes, a, lean, greg, db)                                                     \
  case n:                                                                                      \
    return launch_curv_n<n, nt, nodes, a, lean, greg, db>(E, q, params, metric, out_avg,      \
                                                          out_faces, tables, dx, stream);
    STP_CURV_SHAPES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stp
