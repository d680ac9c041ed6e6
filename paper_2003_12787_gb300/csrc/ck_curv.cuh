// Curvilinear CK step pieces shared by the FP64 curvilinear kernels and the
// point-source correction (device code).
//
// With the inverse Jacobian G[d][j] = dxi_d/dx_j of the element map, the
// physical derivative is d/dx_j = sum_d G[d][j] d/dxi_d. A node's nine partial
// sums collect, over the reference directions d, the products of G's row d
// with the reference derivatives of the quantities:
//   part[v_i] = sum_j dsigma_ij/dx_j, part[s_ii] = dv_i/dx_i,
//   part[s_ij] = dv_i/dx_j + dv_j/dx_i (i < j),
// and the node's elastic coefficients turn them into the new term.
#pragma once
#include "ck_fp64.cuh"

namespace stp {

// Adds the contributions of quantity s, whose derivative along reference
// direction d is a, to a node's partial sums; (g0, g1, g2) = G[d][0..2]. The
// sums are indexed by the output they feed: part[v_i] = sum_j dsigma_ij/dx_j,
// part[s_ii] = dv_i/dx_i, part[s_ij] = dv_i/dx_j + dv_j/dx_i.
__device__ __forceinline__ void curv_add(int s, double a, double g0, double g1, double g2,
                                         double part[9]) {
  switch (s) {
    case kV1:
      part[kS11] = fma(g0, a, part[kS11]);
      part[kS12] = fma(g1, a, part[kS12]);
      part[kS13] = fma(g2, a, part[kS13]);
      break;
    case kV2:
      part[kS12] = fma(g0, a, part[kS12]);
      part[kS22] = fma(g1, a, part[kS22]);
      part[kS23] = fma(g2, a, part[kS23]);
      break;
    case kV3:
      part[kS13] = fma(g0, a, part[kS13]);
      part[kS23] = fma(g1, a, part[kS23]);
      part[kS33] = fma(g2, a, part[kS33]);
      break;
    case kS11: part[kV1] = fma(g0, a, part[kV1]); break;
    case kS22: part[kV2] = fma(g1, a, part[kV2]); break;
    case kS33: part[kV3] = fma(g2, a, part[kV3]); break;
    case kS12:
      part[kV1] = fma(g1, a, part[kV1]);
      part[kV2] = fma(g0, a, part[kV2]);
      break;
    case kS13:
      part[kV1] = fma(g2, a, part[kV1]);
      part[kV3] = fma(g0, a, part[kV3]);
      break;
    default:  // kS23
      part[kV2] = fma(g2, a, part[kV2]);
      part[kV3] = fma(g1, a, part[kV3]);
      break;
  }
}

// New term of one node from its partial sums (coefficients already scaled
// like the step tables' derivatives).
__device__ __forceinline__ void curv_pointwise(const double part[9], double invrho, double lam,
                                               double mu, double mu2, double r[9]) {
  const double ltr = __dmul_rn(lam, (part[kS11] + part[kS22]) + part[kS33]);
  r[kV1] = __dmul_rn(invrho, part[kV1]);
  r[kV2] = __dmul_rn(invrho, part[kV2]);
  r[kV3] = __dmul_rn(invrho, part[kV3]);
  r[kS11] = fma(mu2, part[kS11], ltr);
  r[kS22] = fma(mu2, part[kS22], ltr);
  r[kS33] = fma(mu2, part[kS33], ltr);
  r[kS12] = __dmul_rn(mu, part[kS12]);
  r[kS13] = __dmul_rn(mu, part[kS13]);
  r[kS23] = __dmul_rn(mu, part[kS23]);
}

// One curvilinear CK step at node (x, y, z) straight from shared memory:
// p[quantity * S + node] (node = (z*N + y)*N + x), Dk the step's derivative
// matrix (row stride LDD), g the node's metric (9, row-major), coefficients
// scaled by dx (Dk holds D dt/((k+2) dx)). 27 dot products of length N.
template <int N, int S, int LDD>
__device__ __forceinline__ void ck_node_curv_fp64(const double* __restrict__ p,
                                                  const double* __restrict__ Dk, int x, int y,
                                                  int z, const double g[9], double invrho,
                                                  double lam, double mu, double mu2, double r[9]) {
  double part[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) part[c] = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int i = d == 0 ? x : d == 1 ? y : z;
    const double* row = Dk + i * LDD;
    const int base = d == 0 ? (z * N + y) * N : d == 1 ? z * N * N + x : y * N + x;
    const int stride = d == 0 ? 1 : d == 1 ? N : N * N;
    // not unrolled: the point-source correction that uses this step runs on
    // a few elements, and the fully unrolled form multiplies compile time
#pragma unroll 1
    for (int s = 0; s < 9; ++s) {
      double a = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) a = fma(row[l], p[s * S + base + l * stride], a);
      curv_add(s, a, g[3 * d], g[3 * d + 1], g[3 * d + 2], part);
    }
  }
  curv_pointwise(part, invrho, lam, mu, mu2, r);
}

}  // namespace stp
