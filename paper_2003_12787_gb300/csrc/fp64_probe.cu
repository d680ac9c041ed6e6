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

// FP64 tensor-core (DMMA) throughput probe: four independent accumulator
// fragments per warp of the warp-level m8n8k4 FP64 MMA (512 flop per warp
// instruction), the alternative to DFMA for the FP64 contractions.
__global__ void dmma_peak_kernel(double* sink, int iters, double a, double b) {
  double c[4][2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    c[j][0] = threadIdx.x * 1e-3 + j;
    c[j][1] = threadIdx.x * 2e-3 - j;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[j][0]), "+d"(c[j][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1];
  if (s == 123.456) sink[0] = s;  // keeps the loop alive; never true in practice
}

}  // namespace

cudaError_t launch_dmma_peak(double* sink, int blocks, int threads, int iters,
                             cudaStream_t stream) {
  dmma_peak_kernel<<<blocks, threads, 0, stream>>>(sink, iters, 1e-9, 1e-9);
  return cudaGetLastError();
}

cudaError_t launch_fp64_peak(double* sink, int blocks, int threads, int iters,
                             cudaStream_t stream) {
  fp64_peak_kernel<<<blocks, threads, 0, stream>>>(sink, iters, 1.0000001, 1e-9);
  return cudaGetLastError();
}

}  // namespace stp
