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

// Launch shapes per N: STP_CURV_SHAPES (curv_body.cuh).
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
