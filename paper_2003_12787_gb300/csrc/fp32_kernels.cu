// FP32 variant of the Space-Time Predictor on the CUDA cores (precision
// STP_PRECISION_FP32).
//
// Same Taylor bookkeeping as the FP64 kernels: r_0 = q,
// r_{k+1} = dt/(k+2) * L r_k with L q = -sum_d B_d (D_d q)/dx, and the time
// average of Eq. (exahypeTimeAverage) divided by dt is sum_{k=0..N} r_k.
// The paper's kernels are FP64 throughout; this variant splits the arithmetic
// like the library's tensor-core variants, with FP32 in place of the
// BF16/FP16 slices:
//   * r_1 = dt/2 L q in FP64 (the correction pass); r_0 + r_1 in FP64;
//   * r_2 .. r_N from per-node FP32 FMA chains (state, step matrices and
//     coefficients rounded to FP32), their sum accumulated in FP32;
//   * time average = (r_0 + r_1) + FP32 tail, in FP64, and the face
//     projections of Sec. II-B in FP64.
// The contractions are K = N long, too short to feed the tensor cores
// efficiently once the slice conversions and the scatter of the results back
// to the nodes are paid; the FP32 pipe (64 FP32 FMA per DFMA on GB300) makes
// the tail cheap, so the FP64 first term dominates the run time.
//
// The per-node step is the dimension-split scheme of Sec. IV (SplitCK).
// One CTA owns EPC elements; every thread owns NPT nodes of one element. The
// element's current term lives in shared memory as p[quantity][node] (FP64
// for the first step, then FP32 in the same bytes). r_0 + r_1 of the owned
// nodes is parked in the output average (global memory, read back by the
// same thread at the end), the FP32 tail in registers.
#include "ck_fp64.cuh"
#include "stp_internal.h"

namespace stp {
namespace {

constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }

template <int N, int NPT, int EPC>
struct Fp32Shape {
  static constexpr int N3 = N * N * N;
  static constexpr int T = cdiv(N3, NPT);  // threads per element
  static constexpr int BLOCK = T * EPC;
  static constexpr int S = N3 | 1;         // odd row stride (doubles or floats)
  static constexpr int LDD = N | 1;
  // doubles: step-0 matrix [N][LDD], phi0, phi1, EPC x p[9][S];
  // then floats: step matrices [N][N][LDD]
  static constexpr int DOUBLES = N * LDD + 2 * N + EPC * kQuantities * S;
  static constexpr size_t SMEM = sizeof(double) * (size_t)DOUBLES + sizeof(float) * (size_t)(N * N * LDD);
};

template <int N, int NPT, int EPC>
__global__ void __launch_bounds__(Fp32Shape<N, NPT, EPC>::BLOCK, 1)
fp32_stp_kernel(const double* __restrict__ q, const double* __restrict__ params,
                double* __restrict__ out_avg, double* __restrict__ out_faces,
                const double* __restrict__ tables, int64_t E) {
  using Sh = Fp32Shape<N, NPT, EPC>;
  constexpr int N3 = Sh::N3, T = Sh::T, S = Sh::S, LDD = Sh::LDD;
  constexpr int M = kQuantities;
  extern __shared__ double smem[];
  double* sD0 = smem;                  // [N][LDD], FP64 step-0 matrix
  double* sPhi = sD0 + N * LDD;        // phi0[N], phi1[N]
  double* sP = sPhi + 2 * N;           // EPC x p[M][S]
  float* sDf = reinterpret_cast<float*>(sP + EPC * M * S);  // [N][N][LDD] FP32 step matrices

  const int tid = threadIdx.x;
  const int el = tid / T;
  const int lt = tid - el * T;
  const int64_t e = (int64_t)blockIdx.x * EPC + el;
  const bool active = e < E;
  double* sp = sP + el * M * S;
  float* spf = reinterpret_cast<float*>(sp);  // FP32 term, in the bytes of the FP64 one
  double* gavg = out_avg + e * (int64_t)(M * N3);

  for (int i = tid; i < N * N; i += Sh::BLOCK) {
    const int row = i / N, col = i - row * N;
    sD0[row * LDD + col] = tables[i];
  }
  for (int i = tid; i < N * N * N; i += Sh::BLOCK) {
    const int row = i / N, col = i - row * N;  // row = k*N + r
    sDf[row * LDD + col] = __double2float_rn(tables[i]);
  }
  for (int i = tid; i < 2 * N; i += Sh::BLOCK) sPhi[i] = tables[N3 + i];

  if (active) {
    const double* qe = q + e * (int64_t)(M * N3);
    for (int f = lt; f < M * N3; f += T) {  // coalesced AoS read, SoA scatter
      const int n = f / M, s = f - n * M;
      sp[s * S + n] = __ldg(qe + f);
    }
  }
  double cd[NPT][4];
  float cf[NPT][4];
  const double* pe = params + e * (int64_t)(kParams * N3);
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int n = lt + j * T;
    cd[j][0] = cd[j][1] = cd[j][2] = cd[j][3] = 0.0;
    if (active && n < N3)
      elastic_coefficients(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2),
                           &cd[j][0], &cd[j][1], &cd[j][2], &cd[j][3]);
#pragma unroll
    for (int c = 0; c < 4; ++c) cf[j][c] = __double2float_rn(cd[j][c]);
  }
  __syncthreads();

  // Step 0 in FP64: r_1 from q; r_0 + r_1 parked in the output average.
  float r[NPT][M];
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int n = lt + j * T;
    if (!active || n >= N3) continue;
    const int x = n % N, y = (n / N) % N, z = n / (N * N);
    double r1[M];
    ck_node_fp64<N, S, LDD>(sp, sD0, x, y, z, cd[j][0], cd[j][1], cd[j][2], cd[j][3], r1);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      gavg[n * M + s] = sp[s * S + n] + r1[s];
      r[j][s] = __double2float_rn(r1[s]);
    }
  }
  __syncthreads();  // every thread has read q
  float acc[NPT][M];
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int n = lt + j * T;
#pragma unroll
    for (int s = 0; s < M; ++s) acc[j][s] = 0.f;
    if (!active || n >= N3) continue;
#pragma unroll
    for (int s = 0; s < M; ++s) spf[s * S + n] = r[j][s];
  }
  __syncthreads();  // r_1 (FP32) visible

  for (int k = 1; k < N; ++k) {
    const float* Dk = sDf + k * N * LDD;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const int n = lt + j * T;
      if (!active || n >= N3) continue;
      const int x = n % N, y = (n / N) % N, z = n / (N * N);
      ck_node_fp32<N, S, LDD>(spf, Dk, x, y, z, cf[j][0], cf[j][1], cf[j][2], cf[j][3], r[j]);
#pragma unroll
      for (int s = 0; s < M; ++s) acc[j][s] += r[j][s];
    }
    __syncthreads();  // every thread has read r_k
    if (k + 1 < N) {
#pragma unroll
      for (int j = 0; j < NPT; ++j) {
        const int n = lt + j * T;
        if (!active || n >= N3) continue;
#pragma unroll
        for (int s = 0; s < M; ++s) spf[s * S + n] = r[j][s];
      }
      __syncthreads();  // r_{k+1} visible
    }
  }

  // Time average in FP64 (the FP32 term is no longer read), then the faces.
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int n = lt + j * T;
    if (!active || n >= N3) continue;
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const double v = gavg[n * M + s] + (double)acc[j][s];
      gavg[n * M + s] = v;
      sp[s * S + n] = v;
    }
  }
  __syncthreads();
  if (active) {
    double* fe = out_faces + e * (int64_t)(6 * N * N * M);
    for (int o = lt; o < 6 * N * N * M; o += T) {
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
      for (int i = 0; i < N; ++i) a = fma(phi[i], sp[s * S + base + i * stride], a);
      fe[o] = a;
    }
  }
}

template <int N, int NPT, int EPC>
cudaError_t launch_fp32_shape(int64_t E, const double* q, const double* params, double* out_avg,
                              double* out_faces, const double* tables, cudaStream_t stream) {
  using Sh = Fp32Shape<N, NPT, EPC>;
  static_assert(Sh::SMEM <= 232448, "shared memory budget of one CTA exceeded");
  static_assert(Sh::BLOCK <= 1024, "too many threads per CTA");
  auto kern = fp32_stp_kernel<N, NPT, EPC>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  if (err != cudaSuccess) return err;
  const int64_t blocks = (E + EPC - 1) / EPC;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  kern<<<(unsigned)blocks, Sh::BLOCK, Sh::SMEM, stream>>>(q, params, out_avg, out_faces, tables, E);
  return cudaGetLastError();
}

}  // namespace

// Launch shape per N: (N, nodes per thread, elements per CTA).
#define STP_FP32_SHAPES(X)                                                                  \
  X(2, 1, 64) X(3, 1, 16) X(4, 1, 8) X(5, 1, 4) X(6, 1, 4) X(7, 1, 2) X(8, 1, 1) X(9, 1, 1) \
  X(10, 1, 1) X(11, 2, 1) X(12, 3, 1)

cudaError_t launch_fp32(int N, int64_t E, const double* q, const double* params, double* out_avg,
                        double* out_faces, const double* tables, cudaStream_t stream) {
  switch (N) {
#define X(n, npt, epc) \
  case n: return launch_fp32_shape<n, npt, epc>(E, q, params, out_avg, out_faces, tables, stream);
    STP_FP32_SHAPES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stp
