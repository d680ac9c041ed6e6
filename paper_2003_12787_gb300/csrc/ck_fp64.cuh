// One FP64 Cauchy-Kowalewsky step at one node (device code shared by the
// FP64 and the mixed-precision kernels).
//
// p holds the current term r_k of one element in shared memory as
// p[quantity * S + node], node = (z*N + y)*N + x. Dk is the step's derivative
// matrix D * dt/((k+2) dx) with row stride LDD. The result is
//   r_{k+1}(node) = A_x (Dk p)_x + A_y (Dk p)_y + A_z (Dk p)_z
// with the elastic coefficient matrices A_d of q_t = sum_d A_d dq/dx_d
// (velocity-stress form): only the 6 quantities each direction couples are
// differentiated, and the cross-direction sums are single DFMA chains.
#pragma once

namespace stp {

// Quantity slots of the state vector.
enum : int { kV1 = 0, kV2, kV3, kS11, kS22, kS33, kS12, kS13, kS23 };

template <int N, int S, int LDD>
__device__ __forceinline__ void ck_node_fp64(const double* __restrict__ p,
                                             const double* __restrict__ Dk, int x, int y, int z,
                                             double invrho, double lam, double mu, double mu2,
                                             double r[9]) {
  const double* Dx = Dk + x * LDD;
  const double* Dy = Dk + y * LDD;
  const double* Dz = Dk + z * LDD;
  const double* px = p + (z * N + y) * N;  // + l
  const double* py = p + z * N * N + x;    // + l*N
  const double* pz = p + y * N + x;        // + l*N*N
  double v1 = 0.0, v2 = 0.0, v3 = 0.0, s12 = 0.0, s13 = 0.0, s23 = 0.0;
  double a = 0.0, b = 0.0, c = 0.0;  // dv1/dx, dv2/dy, dv3/dz
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const double d = Dx[l];
    v1 = fma(d, px[kS11 * S + l], v1);
    v2 = fma(d, px[kS12 * S + l], v2);
    v3 = fma(d, px[kS13 * S + l], v3);
    a = fma(d, px[kV1 * S + l], a);
    s12 = fma(d, px[kV2 * S + l], s12);
    s13 = fma(d, px[kV3 * S + l], s13);
  }
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const double d = Dy[l];
    const int o = l * N;
    v1 = fma(d, py[kS12 * S + o], v1);
    v2 = fma(d, py[kS22 * S + o], v2);
    v3 = fma(d, py[kS23 * S + o], v3);
    s12 = fma(d, py[kV1 * S + o], s12);
    b = fma(d, py[kV2 * S + o], b);
    s23 = fma(d, py[kV3 * S + o], s23);
  }
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const double d = Dz[l];
    const int o = l * N * N;
    v1 = fma(d, pz[kS13 * S + o], v1);
    v2 = fma(d, pz[kS23 * S + o], v2);
    v3 = fma(d, pz[kS33 * S + o], v3);
    s13 = fma(d, pz[kV1 * S + o], s13);
    s23 = fma(d, pz[kV2 * S + o], s23);
    c = fma(d, pz[kV3 * S + o], c);
  }
  // products rounded on their own: no kernel that inlines this step may fuse
  // them into its later additions, so every FP64 path gives the same bits
  const double ltr = __dmul_rn(lam, (a + b) + c);
  r[kV1] = __dmul_rn(invrho, v1);
  r[kV2] = __dmul_rn(invrho, v2);
  r[kV3] = __dmul_rn(invrho, v3);
  r[kS11] = fma(mu2, a, ltr);
  r[kS22] = fma(mu2, b, ltr);
  r[kS33] = fma(mu2, c, ltr);
  r[kS12] = __dmul_rn(mu, s12);
  r[kS13] = __dmul_rn(mu, s13);
  r[kS23] = __dmul_rn(mu, s23);
}

// Lame coefficients of one node from (rho, cp, cs): 1/rho, lambda, mu, 2 mu.
// Every product is rounded on its own (no contraction into an FMA), so every
// kernel that inlines this gets the same bits whatever the compiler fuses.
__device__ __forceinline__ void elastic_coefficients(double rho, double cp, double cs,
                                                     double* invrho, double* lam, double* mu,
                                                     double* mu2) {
  const double cs2 = __dmul_rn(cs, cs);
  const double m = __dmul_rn(rho, cs2);
  *invrho = 1.0 / rho;
  *lam = __dmul_rn(rho, __dsub_rn(__dmul_rn(cp, cp), 2.0 * cs2));
  *mu = m;
  *mu2 = m + m;
}

}  // namespace stp
