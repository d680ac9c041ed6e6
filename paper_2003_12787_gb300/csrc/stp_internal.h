// Internal declarations shared by the translation units of the CUDA library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/stp.h"

namespace stp {

constexpr int kQuantities = 9;  // v1 v2 v3 s11 s22 s33 s12 s13 s23
constexpr int kParams = 3;      // rho cp cs
constexpr int kMaxNodes = 12;

// Host-side tables of the reference element for N nodes per dimension, in
// double precision, computed in extended precision (tables.cpp).
struct HostTables {
  int N = 0;
  int family = STP_NODES_GAUSS_LEGENDRE;
  double nodes[kMaxNodes];
  double D[kMaxNodes * kMaxNodes];  // D[i*N+j] = phi_j'(xi_i)
  double phi0[kMaxNodes];
  double phi1[kMaxNodes];
  double weights[kMaxNodes];  // quadrature weights on [0,1] (sum 1)
};

// Nodes (Gauss-Legendre or Gauss-Lobatto, see stp_node_family), derivative
// matrix and face vectors. Returns false for an unknown family, Gauss-Lobatto
// with N < 2, or a Newton iteration that did not converge (never for
// N <= 12).
bool make_tables(int N, HostTables* t, int family = STP_NODES_GAUSS_LEGENDRE);

// Per-step scaled derivative matrices: Dk[k][i][j] = D[i][j] * dt / ((k+2) dx)
// for k = 0..N-1, rounded once from extended precision.
void make_step_matrices(const HostTables& t, double dx, double dt, double* Dk);

// Device tables: [N][N][N] step matrices, then phi0[N], phi1[N], then the
// unscaled D[N][N], then the tensor-core operand tiles of D (make_tc_tiles).
// N^3 + N^2 + 2N is even, so the tile region starts 16-byte aligned.
constexpr int kTcChunkBytes = 1024;   // 32 rows (N) x 16 K of 16-bit values
constexpr int kTcOperandBytes = 2 * kTcChunkBytes;  // K = 32: two chunks
constexpr int kTcRegionBytes = 2 * 3 * kTcOperandBytes;  // FP16 then BF16; T = 1, 2, 3
inline int table_offset_D(int N) { return N * N * N + 2 * N; }
inline int table_offset_tc(int N) { return table_offset_D(N) + N * N; }
inline int table_doubles(int N) { return table_offset_tc(N) + kTcRegionBytes / 8; }

// Tensor-core operand tiles of D (tc_kernels.cuh), for N <= 10. D 2^(W-1-eD)
// is written as balanced base-2^W digits B_0 + B_1 2^-W + ... (W = 10 for
// FP16, 8 for BF16; |B_t| <= 2^(W-1)), each digit an exact 16-bit value. The
// state's T digits sit side by side along K (digit s at k = N s + l), so one
// operand per T (1, 2, 3) holds, for output i and digit s, three column
// blocks of N columns: [L0: B_0 if s = 0 | X: B_(1-s) 2^c | Y: B_(2-s) 2^(c-W)]
// (zero where the index is negative or s >= T); c = 6 for FP16 (keeps every
// value a normal FP16 number), 0 for BF16. Each operand is two K-major
// no-swizzle chunks of 16 K (k = 0..15, 16..31) x 32 rows. Returns false if
// a value is not exactly representable (never for 2 <= N <= 10).
bool make_tc_tiles(const HostTables& t, int eD, unsigned char* out);

// Kernel launchers (fp64_kernels.cu). Return cudaSuccess or the launch error.
cudaError_t launch_fp64(int N, int64_t E, const double* q, const double* params,
                        double* out_avg, double* out_faces, const double* tables,
                        cudaStream_t stream);
// Elements per CTA the FP64 kernel uses for N nodes (chunk sizes are multiples).
int fp64_elements_per_cta(int N);

// Mixed-precision kernel (mixed_kernels.cu); variant 1..4 = BF16x2, BF16x3,
// FP16x2, FP16x3; 2 <= N <= 12. eD = binary exponent of max |D| (frexp).
// status receives bit 0 on a bounded-wait timeout.
cudaError_t launch_mixed(int N, int variant, int64_t E, const double* q, const double* params,
                         double* out_avg, double* out_faces, const double* tables,
                         const double* Dref, double dt_over_dx, int eD, unsigned int* status,
                         cudaStream_t stream);

// FP32 variant (fp32_kernels.cu): first CK term in float-float, later terms in
// FP32 on the CUDA cores; 2 <= N <= 12. status receives bit 0 when a bounded
// wait on a bulk copy gave up.
cudaError_t launch_fp32(int N, int64_t E, const double* q, const double* params, double* out_avg,
                        double* out_faces, const double* tables, unsigned int* status,
                        cudaStream_t stream);

// Float-float variant (ff_kernels.cu): every step in float-float on the FP32
// pipes; ff_supported(N) is true for 2 <= N <= 12.
bool ff_supported(int N);
cudaError_t launch_ff(int N, int64_t E, const double* q, const double* params, double* out_avg,
                      double* out_faces, const double* tables, cudaStream_t stream);

// FP64 STP on curvilinear elements (curvilinear.cu): metric [E][N][N][N][9]
// holds the per-node inverse Jacobian dxi_d/dx_j at 3d + j; tables are the
// handle's (step matrices scaled by 1/dx, undone with dx).
cudaError_t launch_curvilinear(int N, int64_t E, const double* q, const double* params,
                               const double* metric, double* out_avg, double* out_faces,
                               const double* tables, double dx, cudaStream_t stream);
// The same in float-float, and with steps 1..N-1 in FP32 (ff_curvilinear.cu),
// 2 <= N <= 12.
cudaError_t launch_ff_curvilinear(int N, int64_t E, const double* q, const double* params,
                                  const double* metric, double* out_avg, double* out_faces,
                                  const double* tables, double dx, cudaStream_t stream);
cudaError_t launch_fp32_curvilinear(int N, int64_t E, const double* q, const double* params,
                                    const double* metric, double* out_avg, double* out_faces,
                                    const double* tables, double dx, cudaStream_t stream);

// Bounded-wait self-test (selftest.cu): one CTA waits on an mbarrier nothing
// arrives at, for `limit` polls, then sets bit 1 of *status.
cudaError_t launch_wait_selftest(unsigned int* status, int limit, cudaStream_t stream);

// Point sources (sources.cu): after the STP of a set, adds the response of
// the point sources to the outputs of the elements holding them (FP64, one
// CTA per such element). groups[g] = (element, first source, source count);
// per source: proj[N^3] (phi_node(pos) / (w_node h^3)), amp[9], cf[N]
// (dt^(k+1)/(k+2)! f^(k)). scratch: 9 N^3 doubles per group.
struct SourceGroup {
  int64_t element;
  int first, count;
};
// metric (may be NULL): curvilinear elements; proj then omits the node
// volume, which the kernel takes from |det G| (dx rescales the coefficients).
cudaError_t launch_sources(int N, int ngroups, const SourceGroup* groups, const double* proj,
                           const double* amp, const double* cf, const double* tables,
                           const double* params, const double* metric, double dx,
                           double* out_avg, double* out_faces, double* scratch,
                           cudaStream_t stream);

// Batched persistent FP64 launch (batch.cu).
struct BatchPlan;
// Candidate shapes of order N for the batched kernel; fills epc_out[v] with
// the elements per CTA of each; returns their number.
int batch_variants(int N, int* epc_out);
// Bit v set when candidate shape v exists for order N; epc_out[v] filled.
int batch_variants_mask(int N, int* epc_out);
// Measures (once per device and N, then cached) every candidate shape on a
// synthetic set and returns the fastest; us_all[v] gets each candidate's
// microseconds per element (may be NULL).
cudaError_t autotune(int N, const double* tables, int* variant, double* us_per_element,
                     double* us_all);
// metrics[i] (when metrics and it are not NULL) makes set i curvilinear, with
// the handle's dx[i]; such sets run the curvilinear body in the same launch.
cudaError_t create_plan(int nsets, const int* N, const int64_t* E, const double* const* q,
                        const double* const* params, double* const* avg, double* const* faces,
                        const double* const* tables, const int* forced_variant, BatchPlan** out,
                        const double* const* metrics = nullptr, const double* dx = nullptr);
cudaError_t launch_plan(BatchPlan* p, cudaStream_t stream);
// The sets' FP64 STPs as per-shape persistent launches issued one after
// another on `stream`, with caller-provided scratch (256 bytes of counters,
// then parking areas); metrics[i] (when metrics and it are not NULL) makes
// set i curvilinear with the handle's dx[i]. Allocates nothing; *too_big = 1
// (cudaErrorInvalidValue) when the scratch is too small. Shapes: the
// autotuner's cached choice per order, else the default GB300 choice.
cudaError_t launch_shape_batches(int nsets, const int* N, const int64_t* E,
                                 const double* const* q, const double* const* params,
                                 double* const* avg, double* const* faces,
                                 const double* const* tables, const double* const* metrics,
                                 const double* dx, unsigned char* scratch, size_t scratch_bytes,
                                 cudaStream_t stream, int* too_big);
void plan_info(const BatchPlan* p, int* units, int* ctas, size_t* smem);
void destroy_plan(BatchPlan* p);

// Batched FP64 launch with all scratch in a fixed-size static device array
// (noalloc.cu). *too_big = 1 when nsets or the needed scratch exceed it.
// metrics[i] (when metrics and it are not NULL) makes set i curvilinear, with
// the handle's dx[i]: one element per work unit of the same launch.
cudaError_t run_static_batch(int nsets, const int* N, const int64_t* E, const double* const* q,
                             const double* const* params, double* const* avg,
                             double* const* faces, const double* const* tables,
                             cudaStream_t stream, int* too_big, size_t reserve_top = 0,
                             const double* const* metrics = nullptr, const double* dx = nullptr);
// Device address of the top `bytes` (a multiple of 256) of that static array.
cudaError_t static_scratch_top(size_t bytes, unsigned char** out);

// The same launch with caller-provided scratch (counter + per-CTA parking);
// scratch_bytes = param_batch_scratch_bytes() suffices for one CTA per SM on
// up to ~190 SMs. At most param_batch_max_sets() sets.
cudaError_t launch_param_batch(int nsets, const int* N, const int64_t* E, const double* const* q,
                               const double* const* params, double* const* avg,
                               double* const* faces, const double* const* tables,
                               unsigned char* scratch, size_t scratch_bytes, cudaStream_t stream,
                               int* too_big, const double* const* metrics = nullptr,
                               const double* dx = nullptr);
size_t static_scratch_bytes();
int static_max_sets();

// Device tables of a handle (stp_api.cu).
const double* stp_handle_tables(stp_handle h);
double stp_handle_dx(stp_handle h);
// Whether the handle's steps are the FP64 ones (its precision, or N = 1).
bool stp_handle_is_fp64(stp_handle h);
// One launch of the handle's configured kernel (its precision; curvilinear
// when metric is not NULL) on stream st.
cudaError_t stp_launch_handle(stp_handle h, int64_t E, const double* q, const double* params,
                              const double* metric, double* avg, double* faces, cudaStream_t st);

// Point-source data of one served simulation, prepared and uploaded once
// (stp_api.cu): the sources' response, added after every STP step of the
// simulation to its new average and faces on stream st.
struct ServedSources;
cudaError_t served_sources_launch(const ServedSources* src, const double* params,
                                  const double* metric, double* avg, double* faces, cudaStream_t st);
void served_sources_free(ServedSources* src);

// Served predictor (server.cu); see include/stp.h for the behaviour.
// server_add_sim takes ownership of `sources` (may be NULL) when it succeeds.
struct Server;
cudaError_t server_create(int64_t budget, int nslots, Server** out);
void server_destroy(Server* s);
cudaError_t server_add_sim(Server* s, stp_handle h, int N, int64_t E, const double* q0,
                           const double* params, const double* metric, bool device_src, int* id,
                           bool* too_big, ServedSources* sources = nullptr);
cudaError_t server_run_trace(Server* s, int64_t n, const double* t_arr, const int* sim_ids,
                             double* latency, double* wall);
cudaError_t server_drain(Server* s);
cudaError_t server_read(Server* s, int id, double* q, double* faces, int64_t* steps);
void server_stats(const Server* s, int64_t* out);
void server_submit(Server* s, int id);
cudaError_t server_progress(Server* s, int* done);
int server_sims(const Server* s);
void server_set_policy(Server* s, int policy, double age_bound);

// Corrector on a periodic grid of gx*gy*gz cubes (corrector.cu): q_out = q +
// dt (A.(D avg)/dx - lift of the Rusanov fluctuations of the face values);
// q_out may be q. face_params: [E][6][N][N][3] from launch_face_params.
cudaError_t launch_corrector(int N, int gx, int gy, int gz, const HostTables& t, double dx,
                             double dt, const double* tables, const double* q,
                             const double* params, const double* face_params, const double* avg,
                             const double* faces, double* q_out, cudaStream_t stream);
// Face projection of the per-node material (rho, cp, cs) with phi(0), phi(1).
cudaError_t launch_face_params(int N, int64_t E, const double* tables, const double* params,
                               double* out, cudaStream_t stream);

cudaError_t launch_fp64_peak(double* sink, int blocks, int threads, int iters,
                             cudaStream_t stream);
// The same with the warp-level FP64 MMA (m8n8k4, 512 flop per warp instruction).
cudaError_t launch_dmma_peak(double* sink, int blocks, int threads, int iters,
                             cudaStream_t stream);

}  // namespace stp
