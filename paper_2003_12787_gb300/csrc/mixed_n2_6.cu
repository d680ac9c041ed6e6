// Explicit instantiations of the tensor-core STP kernels for N = 2, 3, 4, 5, 6.
#include "tc_kernels.cuh"

namespace stp {
template cudaError_t launch_mixed_for<2>(int, int64_t, const double*, const double*, double*,
                                          double*, const double*, const double*, double, int, unsigned int*,
                                          cudaStream_t);
template cudaError_t launch_mixed_for<3>(int, int64_t, const double*, const double*, double*,
                                          double*, const double*, const double*, double, int, unsigned int*,
                                          cudaStream_t);
template cudaError_t launch_mixed_for<4>(int, int64_t, const double*, const double*, double*,
                                          double*, const double*, const double*, double, int, unsigned int*,
                                          cudaStream_t);
template cudaError_t launch_mixed_for<5>(int, int64_t, const double*, const double*, double*,
                                          double*, const double*, const double*, double, int, unsigned int*,
                                          cudaStream_t);
template cudaError_t launch_mixed_for<6>(int, int64_t, const double*, const double*, double*,
                                          double*, const double*, const double*, double, int, unsigned int*,
                                          cudaStream_t);
}  // namespace stp
