// Float-float STP on curvilinear elements: launch shapes and dispatch (the
// kernel is in ff_curv.cuh).
#include "ff_curv.cuh"

namespace stp {

// Launch shapes per N: threads, nodes per thread, quantities per line pass,
// lean register state, metric in registers, double buffer (measured on GB300
// among 2-5 candidates per N; keeping the metric and the average in
// registers beats a line task per thread at N = 8, unlike the FP64 kernel).
#define STP_FF_CURV_SHAPES(X)                                                                  \
  X(2, 32, 1, 9, false, true, false) X(3, 32, 1, 9, false, true, false)                       \
  X(4, 64, 1, 9, false, true, false) X(5, 128, 1, 9, false, true, false)                      \
  X(6, 224, 1, 9, false, true, false) X(7, 448, 1, 9, false, true, false)                     \
  X(8, 512, 1, 9, false, true, true) X(9, 384, 2, 9, false, true, true)                       \
  X(10, 512, 2, 9, true, true, false) X(11, 448, 3, 9, true, false, false)                    \
  X(12, 448, 4, 5, true, false, false)

cudaError_t launch_ff_curvilinear(int N, int64_t E, const double* q, const double* params,
                                  const double* metric, double* out_avg, double* out_faces,
                                  const double* tables, double dx, cudaStream_t stream) {
  if (E <= 0) return cudaSuccess;
  switch (N) {
#define X(n, nt, nodes, a, lean, greg, db)                                                     \
  case n:                                                                                      \
    return launch_ff_curv_n<n, nt, nodes, a, lean, greg, db>(E, q, params, metric, out_avg,   \
                                                             out_faces, tables, dx, stream);
    STP_FF_CURV_SHAPES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stp
