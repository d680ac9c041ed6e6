// Point sources: the response of the elements that hold sources, added to the
// STP outputs after the main launch.
//
// The linear PDE carries a source term (Sec. II-A), projected onto the nodal
// basis; in the STP its time derivatives enter every Cauchy-Kowalewsky order
// (the generic STP figure adds derive(pointSource, time, order o) to each
// term): q^(k+1) = L q^(k) + s^(k). A source is a Dirac delta at a reference
// position of its element times a vector over the quantities times a time
// function f, so with the diagonal (quadrature) mass matrix
//   s^(k)_node = phi_node(pos) / (w_node h^3) * amp * f^(k)(t_n).
// The STP is linear, so the average with sources is the source-free average
// plus the STP response to the sources alone (zero initial state), which is
// non-zero only on the elements holding sources. This kernel computes that
// response, in FP64 with the per-node step of the FP64 kernels, and adds it
// (and its face projections) to the outputs: in the Taylor bookkeeping of the
// FP64 kernels, r_0 = 0 and
//   r_{k+1} = dt/(k+2) L r_k + dt^(k+1)/(k+2)! s^(k),   avg += sum_k r_k.
// On curvilinear elements (metric given) L is the curvilinear operator and the
// node volume of the mass matrix is w_node |det J_node| = w_node / |det G_node|:
// the host passes phi_node(pos) / w_node and the kernel multiplies by
// |det G_node|.
#include "ck_curv.cuh"
#include "stp_internal.h"

namespace stp {
namespace {

constexpr int kSourceThreads = 512;

template <int N, bool CURV>
__global__ void __launch_bounds__(kSourceThreads, 1)
source_kernel(const SourceGroup* __restrict__ groups, const double* __restrict__ proj,
              const double* __restrict__ amp, const double* __restrict__ cf,
              const double* __restrict__ tables, const double* __restrict__ params,
              const double* __restrict__ metric, double dx, double* __restrict__ out_avg,
              double* __restrict__ out_faces, double* __restrict__ scratch) {
  constexpr int N3 = N * N * N, S = N3 | 1, LDD = N | 1, M = kQuantities;
  constexpr int NODES = (N3 + kSourceThreads - 1) / kSourceThreads;
  extern __shared__ double smem[];
  double* sD = smem;                  // [N steps][N rows][LDD]
  double* sPhi = sD + N * N * LDD;    // phi0[N], phi1[N]
  double* sp = sPhi + 2 * N;          // r_k [9][S]
  const SourceGroup g = groups[blockIdx.x];
  const int tid = threadIdx.x;
  double* avg_src = scratch + (size_t)blockIdx.x * M * N3;  // [node][9]
  for (int i = tid; i < N * N * N; i += kSourceThreads) {
    const int row = i / N, col = i - row * N;
    sD[row * LDD + col] = tables[i];
  }
  for (int i = tid; i < 2 * N; i += kSourceThreads) sPhi[i] = tables[N3 + i];
  for (int i = tid; i < M * S; i += kSourceThreads) sp[i] = 0.0;
  for (int i = tid; i < M * N3; i += kSourceThreads) avg_src[i] = 0.0;
  double c[NODES][4];
  const double* pe = params + g.element * (int64_t)(kParams * N3);
  const double* ge = CURV ? metric + g.element * (int64_t)(9 * N3) : nullptr;
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * kSourceThreads;
    c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0;
    if (n < N3) {
      elastic_coefficients(pe[3 * n], pe[3 * n + 1], pe[3 * n + 2], &c[j][0], &c[j][1], &c[j][2],
                           &c[j][3]);
      if (CURV) {  // the step tables hold D dt/((k+2) dx)
#pragma unroll
        for (int i = 0; i < 4; ++i) c[j][i] *= dx;
      }
    }
  }
  __syncthreads();

  for (int k = 0; k < N; ++k) {
    double r[NODES][M];
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * kSourceThreads;
      if (n >= N3) continue;
      double gn[9];  // the node's metric (curvilinear)
      double vol_inv = 1.0;  // |det G_node| (curvilinear), else folded into proj
      if (CURV) {
#pragma unroll
        for (int i = 0; i < 9; ++i) gn[i] = __ldg(ge + 9 * n + i);
        vol_inv = fabs(gn[0] * (gn[4] * gn[8] - gn[5] * gn[7]) - gn[1] * (gn[3] * gn[8] - gn[5] * gn[6]) +
                       gn[2] * (gn[3] * gn[7] - gn[4] * gn[6]));
      }
      if (k == 0) {
#pragma unroll
        for (int s = 0; s < M; ++s) r[j][s] = 0.0;  // r_0 = 0
      } else {
        const int x = n % N, y = (n / N) % N, z = n / (N * N);
        if (CURV)
          ck_node_curv_fp64<N, S, LDD>(sp, sD + k * N * LDD, x, y, z, gn, c[j][0], c[j][1], c[j][2],
                                       c[j][3], r[j]);
        else
          ck_node_fp64<N, S, LDD>(sp, sD + k * N * LDD, x, y, z, c[j][0], c[j][1], c[j][2],
                                  c[j][3], r[j]);
      }
      for (int i = g.first; i < g.first + g.count; ++i) {
        const double w = proj[(size_t)i * N3 + n] * vol_inv * cf[(size_t)i * N + k];
#pragma unroll
        for (int s = 0; s < M; ++s) r[j][s] = fma(w, amp[(size_t)i * M + s], r[j][s]);
      }
#pragma unroll
      for (int s = 0; s < M; ++s) avg_src[n * M + s] += r[j][s];
    }
    __syncthreads();  // every thread has read r_k
    if (k + 1 < N) {
#pragma unroll
      for (int j = 0; j < NODES; ++j) {
        const int n = tid + j * kSourceThreads;
        if (n >= N3) continue;
#pragma unroll
        for (int s = 0; s < M; ++s) sp[s * S + n] = r[j][s];
      }
      __syncthreads();
    }
  }
  __syncthreads();  // avg_src complete (global, this block's own area)

  double* ga = out_avg + g.element * (int64_t)(M * N3);
  for (int f = tid; f < M * N3; f += kSourceThreads) ga[f] += avg_src[f];
  double* fe = out_faces + g.element * (int64_t)(6 * N * N * M);
  for (int o = tid; o < 6 * N * N * M; o += kSourceThreads) {
    const int s = o % M;
    int rest = o / M;
    const int bb = rest % N;
    rest /= N;
    const int aa = rest % N;
    const int f = rest / N;
    const int d = f >> 1;
    const double* phi = sPhi + (f & 1) * N;
    int base, stride;
    if (d == 0) { base = (aa * N + bb) * N; stride = 1; }
    else if (d == 1) { base = aa * N * N + bb; stride = N; }
    else { base = aa * N + bb; stride = N * N; }
    double a = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) a = fma(phi[i], avg_src[(base + i * stride) * M + s], a);
    fe[o] += a;
  }
}

template <int N, bool CURV>
cudaError_t launch_sources_n(int ngroups, const SourceGroup* groups, const double* proj,
                             const double* amp, const double* cf, const double* tables,
                             const double* params, const double* metric, double dx,
                             double* out_avg, double* out_faces, double* scratch,
                             cudaStream_t stream) {
  constexpr int N3 = N * N * N;
  constexpr size_t smem = sizeof(double) * (size_t)(N * N * (N | 1) + 2 * N + kQuantities * (N3 | 1));
  static_assert(smem <= 232448, "shared memory budget of one CTA exceeded");
  auto kern = source_kernel<N, CURV>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)ngroups, kSourceThreads, smem, stream>>>(groups, proj, amp, cf, tables, params,
                                                           metric, dx, out_avg, out_faces, scratch);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sources(int N, int ngroups, const SourceGroup* groups, const double* proj,
                           const double* amp, const double* cf, const double* tables,
                           const double* params, const double* metric, double dx,
                           double* out_avg, double* out_faces, double* scratch,
                           cudaStream_t stream) {
  if (ngroups <= 0) return cudaSuccess;
  switch (N) {
#define X(n)                                                                                     \
  case n:                                                                                        \
    return metric ? launch_sources_n<n, true>(ngroups, groups, proj, amp, cf, tables, params,    \
                                              metric, dx, out_avg, out_faces, scratch, stream)   \
                  : launch_sources_n<n, false>(ngroups, groups, proj, amp, cf, tables, params,   \
                                               nullptr, dx, out_avg, out_faces, scratch, stream);
    X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stp
