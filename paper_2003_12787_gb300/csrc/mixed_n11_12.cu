// Explicit instantiations of the tensor-core STP kernels for N = 11, 12.
#include "tc_kernels.cuh"

namespace stp {
template cudaError_t launch_mixed_for<11>(int, int64_t, const double*, const double*, double*,
                                          double*, const double*, const double*, double, int, unsigned int*,
                                          cudaStream_t);
template cudaError_t launch_mixed_for<12>(int, int64_t, const double*, const double*, double*,
                                          double*, const double*, const double*, double, int, unsigned int*,
                                          cudaStream_t);
}  // namespace stp
