// Dispatch of the mixed-precision STP over N (instantiations in mixed_n*.cu).
#include "tc_kernels.cuh"

namespace stp {

#define STP_MIXED_EXTERN(n)                                                                    \
  extern template cudaError_t launch_mixed_for<n>(int, int64_t, const double*, const double*, \
                                                  double*, double*, const double*,            \
                                                  const double*, double, int, unsigned int*,       \
                                                  cudaStream_t);
STP_MIXED_EXTERN(2) STP_MIXED_EXTERN(3) STP_MIXED_EXTERN(4) STP_MIXED_EXTERN(5) STP_MIXED_EXTERN(6)
STP_MIXED_EXTERN(7) STP_MIXED_EXTERN(8) STP_MIXED_EXTERN(9) STP_MIXED_EXTERN(10)
STP_MIXED_EXTERN(11) STP_MIXED_EXTERN(12)
#undef STP_MIXED_EXTERN

cudaError_t launch_mixed(int N, int variant, int64_t E, const double* q, const double* params,
                         double* out_avg, double* out_faces, const double* tables,
                         const double* Dref, double dt_over_dx, int eD, unsigned int* status,
                         cudaStream_t stream) {
  switch (N) {
#define X(n) \
  case n:    \
    return launch_mixed_for<n>(variant, E, q, params, out_avg, out_faces, tables, Dref, dt_over_dx, eD, status, stream);
    X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stp
