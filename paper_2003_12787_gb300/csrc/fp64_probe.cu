// FP64 throughput probe: eight independent DFMA chains per thread over a grid
// of four 256-thread CTAs per SM. It measures what the FP64 pipe of the
// device retires, the denominator of the FP64 path's roofline.
#include "stp_internal.h"

namespace stp {
namespace {

__global__ void fp64_peak_kernel(double* sink, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 123.456) sink[0] = s;  // keeps the loop alive; never true in practice
}

}  // namespace

cudaError_t launch_fp64_peak(double* sink, int blocks, int threads, int iters,
                             cudaStream_t stream) {
  fp64_peak_kernel<<<blocks, threads, 0, stream>>>(sink, iters, 1.0000001, 1e-9);
  return cudaGetLastError();
}

}  // namespace stp
