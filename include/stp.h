/*
 * stp.h - C ABI of the GB300 (sm_103a) linear ADER-DG Space-Time Predictor.
 *
 * The Space-Time Predictor (STP) is the element-local part of a linear
 * ADER-DG step (Gallard et al., arXiv 2003.12787, Sec. II-A and II-B): for
 * every hexahedral element it evolves the nodal state q(t_n) in time with the
 * Cauchy-Kowalewsky (CK) recurrence p_o = V p_{o-1} (the recurrence under
 * Eq. (exahypeTimeAverage)), sums the Taylor series of Eq.
 * (exahypeTimeAverage) on the fly, and projects the result onto the six faces
 * of the element (Sec. II-B: the STP must hand the time-averaged degrees of
 * freedom and their face projections to the corrector).
 *
 * Physics: the 3-D linear elastic wave equation in velocity-stress form
 * (Sec. VI: 3 velocities + 6 stresses, 3 material parameters per node),
 * written q_t + sum_d B_d(x) dq/dx_d = 0, so that one CK step is
 *     q^(k+1) = - sum_d B_d(x) (D_d q^(k)) / dx
 * with D the N x N Lagrange derivative matrix on N Gauss-Legendre nodes per
 * dimension (Sec. II-A) applied along dimension d. Gauss-Lobatto nodes are
 * available through stp_create_nodes; curvilinear elements (Sec. VI: 9 more
 * geometry parameters per node) through stp_predict_curvilinear and its
 * companions, with D along the reference directions and the chain rule
 * through the per-node inverse Jacobian.
 *
 * Outputs per element:
 *     avg  = sum_{k=0..N} dt^k/(k+1)! q^(k)          (time average over [t_n, t_n+dt])
 *     face[d,side] = phi(side)^T applied along d to avg,  side 0 -> reference 0, 1 -> 1
 *
 * All arrays are FP64, row-major, last index fastest:
 *     q, out_avg   [E][N][N][N][9]  element, z, y, x, quantity
 *                  quantities (v1, v2, v3, s11, s22, s33, s12, s13, s23)
 *     params       [E][N][N][N][3]  (rho, cp, cs): density, P and S wave speed
 *     out_faces    [E][6][N][N][9]  faces x-, x+, y-, y+, z-, z+; the two in-plane
 *                  indices are the remaining dimensions in (slower, faster) order:
 *                  x faces [z][y], y faces [z][x], z faces [y][x]
 *
 * Error behaviour: every entry point returns a stp_status. Argument errors are
 * detected before anything is enqueued and leave every buffer untouched.
 * CUDA launch/runtime errors are reported as STP_ERR_CUDA; the message of the
 * last failure on the calling thread is available from stp_last_error().
 */
#ifndef STP_GB300_H
#define STP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stp_handle_s* stp_handle; /* opaque, owned by the library */

typedef enum {
  STP_OK = 0,
  STP_ERR_INVALID_ARG = -1, /* null/misaligned/overlapping/host pointer, bad size */
  STP_ERR_UNSUPPORTED = -2, /* order or number of quantities not implemented */
  STP_ERR_OOM = -3,         /* device or pinned allocation failed */
  STP_ERR_CUDA = -4,        /* a CUDA call failed (see stp_last_error) */
  STP_ERR_TIMEOUT = -5      /* a bounded device-side wait gave up */
} stp_status;

/*
 * Create a predictor for one (order, dx, dt).
 *   order  polynomial degree p; N = p + 1 nodes per dimension, 1 <= N <= 12
 *          ("order N" in the paper's wording is this N, Sec. II-A)
 *   m      number of quantities; must be 9 (elastic system)
 *   dx     element side (the same in x, y and z), > 0 and finite
 *   dt     time step, > 0 and finite
 *   out    receives the handle
 * Computes the Gauss-Legendre nodes, the derivative matrix D (scaled per CK
 * step by dt/((k+2) dx)) and the face interpolation vectors phi(0), phi(1) in
 * extended precision on the host and uploads them to the current CUDA device,
 * which the handle is bound to. Returns STP_ERR_UNSUPPORTED for m != 9 or N
 * out of range, STP_ERR_INVALID_ARG for a bad dx, dt or a NULL out.
 */
stp_status stp_create(int order, int m, double dx, double dt, stp_handle* out);

/*
 * Enqueue the STP of `elements` elements on `stream` (a cudaStream_t; NULL =
 * the legacy default stream). Asynchronous: returns once the kernel is
 * enqueued, without a host synchronisation.
 *   q, params           device pointers (inputs, read only)
 *   out_avg, out_faces  device pointers (outputs, fully overwritten)
 * All four must be device (or managed) memory on the handle's device,
 * 16-byte aligned, and the outputs must not overlap the inputs or each other.
 * The caller owns the buffers and keeps them alive until the stream has
 * passed the kernel. elements == 0 returns STP_OK without a launch. The
 * handle is not modified, so several streams may use one handle at once.
 * The call may be captured into a CUDA graph (while `stream` is capturing,
 * the check that the pointers are device memory is skipped).
 */
stp_status stp_predict(stp_handle h, int64_t elements, const double* q,
                       const double* params, double* out_avg, double* out_faces,
                       void* stream);

/*
 * Face projection of the material, the input the corrector takes for it:
 *   face_params[e][f][a][b][c] = sum_i phi_i(side) params[e][line node i][c]
 * with faces and in-plane indices ordered as out_faces (f = x-,x+,y-,y+,z-,z+;
 * x-faces [z][y], y-faces [z][x], z-faces [y][x]) and c = (rho, cp, cs). In the
 * paper's code the material is stored inside the state vector and reaches the
 * faces through the same projection as the state (Sec. II-A, Sec. VI); it does
 * not change in time, so it is projected once per mesh here.
 *   params       device, [E][N][N][N][3] (input)
 *   face_params  device, [E][6][N][N][3] (output, must not overlap params)
 * Asynchronous on `stream`, capturable. elements == 0 is a no-op.
 */
stp_status stp_face_params(stp_handle h, int64_t elements, const double* params,
                           double* face_params, void* stream);

/*
 * Corrector step of the linear ADER-DG scheme (Sec. II-A, the update that
 * follows Eq. (exahypeTimeAverage)): the predictor's time-averaged state and
 * face projections give the state at t_{n+1},
 *   q_out = q + dt * ( sum_d A_d (D_d avg)/dx  -  lift(F) ),
 * on a structured grid of gx * gy * gz cubes of side dx (the handle's), periodic
 * in every direction, element e = (ez * gy + ey) * gx + ex. The paper leaves
 * the numerical flux open (it only requires it to be linear); this library
 * takes the Rusanov fluctuation of a linear non-conservative system on face f
 * (direction d, side 0/1) at face point (a,b):
 *   F = 1/2 ( Bn (q+ - q-) - s (q+ - q-) ),
 *   Bn = +-1/2 (B_d(m-) + B_d(m+))  (+ on the side-1 face, - on the side-0 face),
 *   s = max(|cp-|, |cp+|),
 * with q- = faces[e][f][a][b], q+ = the neighbour's faces[e'][f^1][a][b],
 * m-/m+ = the two sides' face_params, B_d = -A_d of q_t + sum_d B_d dq/dx_d = 0,
 * and the strong-form lift onto node i of the line through (a,b) along d:
 * phi_i(side) / (w_i dx) F (w the quadrature weights on [0,1]: the diagonal
 * mass matrix of the nodal basis). FP64 whatever the handle's precision.
 *   q, avg     device, [E][N][N][N][9]: the state at t_n and its predictor
 *              average (stp_predict of q with this handle)
 *   faces      device, [E][6][N][N][9]: the predictor's face projections
 *   params     device, [E][N][N][N][3]; face_params from stp_face_params
 *   q_out      device, [E][N][N][N][9]: may be q itself (in place); must not
 *              overlap any other input
 * E = gx * gy * gz. Asynchronous on `stream`, capturable like stp_predict.
 * STP_ERR_INVALID_ARG for a grid dimension < 1, a NULL or misaligned buffer,
 * overlapping buffers, or pointers that are not device memory on the
 * handle's device.
 */
stp_status stp_correct(stp_handle h, int gx, int gy, int gz, const double* q,
                       const double* params, const double* face_params, const double* avg,
                       const double* faces, double* q_out, void* stream);

/*
 * `steps` full ADER-DG steps on the periodic grid of stp_correct: each is
 * stp_predict(q -> avg, faces) in the handle's precision followed by
 * stp_correct(q -> q) in place. avg and faces are the caller's work buffers
 * ([E][N][N][N][9] and [E][6][N][N][9]); after the call they hold the last
 * step's predictor outputs. Arguments and errors as stp_predict and
 * stp_correct; steps == 0 validates and returns. Asynchronous on `stream`,
 * capturable.
 */
stp_status stp_ader_step(stp_handle h, int gx, int gy, int gz, int steps, double* q,
                         const double* params, const double* face_params, double* avg,
                         double* faces, void* stream);

/*
 * Point sources (Sec. II-A: the source term of the linear PDE, projected onto
 * the nodal basis; in the STP the source's time derivatives enter every
 * Cauchy-Kowalewsky order). A source is a Dirac delta at `position` (reference
 * coordinates x, y, z in [0,1]) of element `element`, times `amplitude` over
 * the 9 quantities, times a time function f given by its derivatives
 * f^(k)(t_n), k = 0..N-1 (`derivatives`, entries from N on are ignored). With
 * the diagonal quadrature mass matrix it adds
 *   s^(k)_node = phi_node(position) / (w_node dx^3) * amplitude * f^(k)
 * to every term: q^(k+1) = L q^(k) + s^(k). The paper gives neither the time
 * function nor the placement; the caller supplies both.
 */
typedef struct {
  int64_t element;
  double position[3];
  double amplitude[9];
  double derivatives[12];
} stp_point_source;

/*
 * stp_predict with point sources: the STP of every element as stp_predict
 * (any precision), then, for the elements that hold sources, their response
 * to the sources added to out_avg and out_faces in FP64 (one more launch; the
 * STP is linear, so the two add up). `sources` is a HOST array of nsources
 * entries; several sources may share an element. Asynchronous on `stream`
 * (a small stream-ordered device allocation holds the sources' data; it is
 * copied from host memory, so the call cannot be captured in a CUDA graph).
 * STP_ERR_INVALID_ARG for an element outside [0, elements), a position
 * outside [0,1]^3, a non-finite value or nsources < 0.
 */
stp_status stp_predict_sources(stp_handle h, int64_t elements, const double* q,
                               const double* params, double* out_avg, double* out_faces,
                               int nsources, const stp_point_source* sources, void* stream);

/*
 * stp_predict_sources on curvilinear elements (the LOH1-type setting: a point
 * source in a boundary-fitted mesh): the STP as stp_predict_curvilinear (its
 * precisions), then the sources' response in FP64 with the curvilinear
 * operator, the node volume of the mass matrix being w_node |det J_node| =
 * w_node / |det G_node| from the metric (position in reference coordinates of
 * the element, as before). Errors as stp_predict_sources and
 * stp_predict_curvilinear.
 */
stp_status stp_predict_sources_curvilinear(stp_handle h, int64_t elements, const double* q,
                                           const double* params, const double* metric,
                                           double* out_avg, double* out_faces, int nsources,
                                           const stp_point_source* sources, void* stream);

/*
 * The STP on curvilinear elements. The paper's benchmark meshes are
 * curvilinear and boundary-fitted and store 9 geometry parameters per node
 * beside the 3 material parameters (Sec. VI). Here those 9 are the inverse
 * Jacobian of each element's map from the reference cube [0,1]^3 to physical
 * space:
 *   metric: device, [E][N][N][N][9] float64, (z,y,x) nodes as q, entry 3d + j
 *           = G[d][j] = dxi_d/dx_j, where xi_1, xi_2, xi_3 run along the x, y,
 *           z node indices.
 * By the chain rule d/dx_j = sum_d G[d][j] d/dxi_d, so one Cauchy-Kowalewsky
 * step is q^(k+1) = sum_d (sum_j G[d][j] A_j) (D_d q^(k)) with D along the
 * reference direction d; a cube of side dx has G = I/dx and gives stp_predict's
 * result up to rounding. The handle's dx only scales internal tables (the
 * metric carries the geometry). Faces are the reference faces xi_d = 0, 1 in
 * stp_predict's order; other buffers and their layouts as stp_predict.
 * Asynchronous on `stream`, capturable like stp_predict.
 * The handle's precision selects FP64 (STP_PRECISION_FP64), float-float
 * (STP_PRECISION_FF, the FP64 error bar on the FP32 pipes) or FP32 with a
 * float-float first step (STP_PRECISION_FP32, about 1e-9 on resolved fields);
 * order 0 runs in FP64; STP_ERR_UNSUPPORTED for the tensor-core precisions;
 * STP_ERR_INVALID_ARG for a NULL or unaligned metric, or one that overlaps an
 * output. The library does not check that the metric is invertible.
 */
stp_status stp_predict_curvilinear(stp_handle h, int64_t elements, const double* q,
                                   const double* params, const double* metric,
                                   double* out_avg, double* out_faces, void* stream);

/*
 * stp_predict_curvilinear on HOST buffers (q, params, metric in; out_avg,
 * out_faces out), with the chunked copy/kernel pipeline and the synchronous
 * completion of stp_predict_host. Errors as stp_predict_curvilinear.
 */
stp_status stp_predict_curvilinear_host(stp_handle h, int64_t elements, const double* q,
                                        const double* params, const double* metric,
                                        double* out_avg, double* out_faces, void* stream);

/*
 * Same computation on HOST buffers (pinned host memory gives full copy
 * bandwidth; pageable memory works but copies slower). Synchronous: returns
 * once out_avg and out_faces hold the results. Elements are processed in
 * chunks: the host-to-device copy of one chunk, the kernel of the previous
 * chunk and the device-to-host copy of the one before run concurrently on
 * library-owned streams and device buffers (allocated on first use and kept
 * by the handle, so concurrent calls on ONE handle must be serialised by the
 * caller). `stream` orders the call after work already on that stream.
 */
stp_status stp_predict_host(stp_handle h, int64_t elements, const double* q,
                            const double* params, double* out_avg, double* out_faces,
                            void* stream);

/*
 * Arithmetic of the derivative contractions.
 *   STP_PRECISION_FP64    every step in FP64 (default)
 *   STP_PRECISION_BF16X2 / _BF16X3 / _FP16X2 / _FP16X3
 *       derivative contractions on the tensor cores (2 <= N <= 10): the
 *       first CK term r_1 = dt/2 L q, and every later term while it is above
 *       1e-3 of the state, runs in float-float on the CUDA cores; each later
 *       term is written per quantity in fixed point and cut into up to three
 *       (x3) or two (x2) integer digits of 10 bits (FP16) or 8 bits (BF16),
 *       contracted exactly against the equally cut D on the tensor cores
 *       (leading digit products exact in FP32, the rest accumulated in
 *       FP32), and updated pointwise in FP32. The Taylor average and the face
 *       projections are float-float. Stated bars (resolved and coarse
 *       fields): FP16X3 1e-9, FP16X2 5e-8, BF16X3 5e-9, BF16X2 5e-7 relative.
 *       For N = 11, 12 an earlier kernel runs (first term FP64, later terms
 *       split into 2 or 3 BF16/FP16 slices with FP32 accumulation).
 *   STP_PRECISION_FP32
 *       the same split on the CUDA cores without FP64 instructions: r_1,
 *       r_0 + r_1, the Taylor average and the faces in float-float (pairs of
 *       floats, about 48 significant bits, on the FP32 pipes), every later
 *       term in FP32 (state, step matrices and coefficients rounded to FP32).
 *   STP_PRECISION_FF
 *       every step in float-float on the FP32 pipes (about 48 significant
 *       bits): results agree with the FP64 kernel to about 1e-13 relative,
 *       several times faster on a GPU whose FP64 rate is low.
 * FP32 reaches about 1e-9 relative on well-resolved fields; its error grows
 * with the size of the higher Taylor terms (coarse elements: several 1e-9).
 * FF holds about 1e-13 on any data.
 * FP32 and FF scale each element's state by a power of two (exact) so that
 * its largest magnitude is about 1; within an element, values more than
 * 2^126 below that largest magnitude contribute as zero.
 * The paper's kernels are FP64 throughout; these variants are additions.
 * Reduced-precision variants need 2 <= N; for N = 1 the FP64 kernel runs.
 */
typedef enum {
  STP_PRECISION_FP64 = 0,
  STP_PRECISION_BF16X2 = 1,
  STP_PRECISION_BF16X3 = 2,
  STP_PRECISION_FP16X2 = 3,
  STP_PRECISION_FP16X3 = 4,
  STP_PRECISION_FP32 = 5,
  STP_PRECISION_FF = 6
} stp_precision;

/* Select the precision used by later stp_predict / stp_predict_host calls on
 * this handle (not synchronised with launches already enqueued: set it before
 * sharing the handle between streams). STP_ERR_INVALID_ARG for an unknown value. */
stp_status stp_set_precision(stp_handle h, stp_precision p);

/* Current precision of the handle (STP_PRECISION_FP64 for NULL). */
stp_precision stp_get_precision(stp_handle h);

/*
 * Synchronise `stream`, then read and clear the handle's device status word.
 * *flags receives its bits (bit 0: a bounded device-side wait exceeded its
 * iteration limit - a tensor-core completion wait of the tensor-core
 * precisions, or the wait for a bulk copy of an element into shared memory
 * in the FP32 and tensor-core precisions; the outputs of that launch are
 * invalid;
 * bit 1: set by stp_selftest_bounded_wait; bit 2: after such a timeout the
 * kernel's last bounded wait for the tensor cores to drain gave up too, so an
 * MMA may still have been writing tensor memory when the CTA released it -
 * discard every result computed on this CUDA context from then on and
 * recreate the context).
 * Returns STP_ERR_TIMEOUT if any bit was set, else STP_OK.
 */
stp_status stp_device_status(stp_handle h, void* stream, unsigned int* flags);

/*
 * Self-test of the bounded device-side wait: enqueues on `stream` one CTA that
 * waits on an mbarrier nothing arrives at, polling at most `polls` times (the
 * poll loop of the tensor-core kernel's MMA completion wait), then sets bit 1
 * of the handle's status word and returns. A following stp_device_status
 * reports STP_ERR_TIMEOUT with that bit, and the context stays usable: the
 * failure path is exercised without a fault, a trap or a hang.
 * STP_ERR_INVALID_ARG for polls outside [1, 2^22].
 */
stp_status stp_selftest_bounded_wait(stp_handle h, int polls, void* stream);

/*
 * Batched persistent launches: the STPs of several element sets, of
 * different orders and sizes, replayed from one CUDA graph. Each set is
 * described by a handle (order, dx, dt, precision) and its own device buffers
 * in the layouts above. The paper generates one kernel per order (Sec. II-D,
 * Sec. III); here, for FP64 sets, every shape (order and layout) has one
 * persistent kernel whose CTAs, one per SM, consume its sets' (set, element
 * range) units; a plan launches one such kernel per shape present (128 sets
 * at most per launch), over parallel graph branches so that shapes share the
 * SMs as their work runs out. Curvilinear FP64 sets
 * (stp_batch_create_curvilinear) are one-element units of the curvilinear
 * shape of their order. Batches with other precisions replay a graph of
 * per-set launches instead.
 */
typedef struct {
  stp_handle handle;   /* predictor of this set (FP64 for the allocation-free path) */
  int64_t elements;    /* E >= 0 */
  const double* q;     /* device [E][N][N][N][9] */
  const double* params;/* device [E][N][N][N][3] */
  double* out_avg;     /* device [E][N][N][N][9] */
  double* out_faces;   /* device [E][6][N][N][9] */
} stp_batch_set;

typedef struct stp_batch_s* stp_batch; /* opaque plan, owned by the library */

/*
 * Plan a batch. When every handle is FP64: autotunes (on first use of each
 * order on the device, then cached) the per-order shape, builds and uploads
 * the work list, and captures the counters' reset and the per-shape
 * persistent launches into a CUDA graph. When some handle has another precision: captures
 * one launch per set (each set's own kernel, in its handle's precision at
 * planning time) into a CUDA graph, largest sets first, over up to 8 parallel
 * branches; results equal stp_predict's for every set. The buffers are baked
 * into the plan: they must stay valid, unmoved, until stp_batch_destroy.
 * Outputs must not overlap any input or any other output. Synchronous
 * (allocates, copies, times). Errors: STP_ERR_INVALID_ARG for bad pointers or
 * sizes, STP_ERR_UNSUPPORTED for sets on different devices, STP_ERR_CUDA /
 * STP_ERR_OOM from CUDA.
 */
stp_status stp_batch_create(int nsets, const stp_batch_set* sets, stp_batch* out);

/* As stp_batch_create, with the shape of every set chosen by the caller:
 * shapes[i] = index of one of its order's candidate shapes (0, 1: see
 * stp_autotune), or -1 for the autotuner's choice. STP_ERR_INVALID_ARG for a
 * shape the order does not have, or for any shape >= 0 in a batch that is not
 * all FP64. */
stp_status stp_batch_create_ex(int nsets, const stp_batch_set* sets, const int* shapes,
                               stp_batch* out);

/* As stp_batch_create, with curvilinear sets: metrics is a HOST array of
 * nsets device pointers, metrics[i] the inverse Jacobians of set i in the
 * layout of stp_predict_curvilinear, or NULL for a Cartesian set. When every
 * handle is FP64 the curvilinear sets join the Cartesian ones in the one
 * persistent launch (a unit is one curvilinear element, run by the
 * curvilinear FP64 body with the same arithmetic as stp_predict_curvilinear);
 * otherwise the batch is the CUDA graph of per-set launches. Either way every
 * set's results equal those of its own stp_predict_curvilinear (or
 * stp_predict), bit for bit. Metrics must not overlap any output.
 * STP_ERR_INVALID_ARG for metrics == NULL with nsets > 0, otherwise the errors
 * of stp_batch_create and stp_predict_curvilinear. */
stp_status stp_batch_create_curvilinear(int nsets, const stp_batch_set* sets,
                                        const double* const* metrics, stp_batch* out);

/*
 * A batch plan whose sets may carry point sources (the source term of
 * Sec. II-A, as in stp_predict_sources): nsources[i] sources at sources[i]
 * (host arrays) for set i (0 = none); metrics as stp_batch_create_curvilinear
 * or NULL for a Cartesian batch. The sources' data are prepared and copied to
 * the device once, here; every stp_batch_launch then runs the plan and, on the
 * same stream after it, the sources' FP64 response of each set that has any,
 * added to that set's outputs. Each set's result equals its own
 * stp_predict_sources. Errors as stp_batch_create and stp_predict_sources.
 */
stp_status stp_batch_create_sources(int nsets, const stp_batch_set* sets,
                                    const double* const* metrics, const int* nsources,
                                    const stp_point_source* const* sources, stp_batch* out);

/* Enqueue one replay of the plan's graph on `stream` (async). */
stp_status stp_batch_launch(stp_batch b, void* stream);

/* Work units, CTAs over the plan's persistent launches and the largest
 * dynamic shared memory per CTA among them (for a batch of per-set launches:
 * the number of sets, 0, 0). */
stp_status stp_batch_info(stp_batch b, int* units, int* ctas, int64_t* smem_bytes);

/* Free the plan (after the work it enqueued has finished). NULL is a no-op. */
stp_status stp_batch_destroy(stp_batch b);

/*
 * The autotuner's choice for the handle's order on the current device:
 * *variant = index of the fastest candidate shape (nodes per thread, elements
 * per CTA), *us_per_element its measured time per element, us_variants[0..1]
 * the time of every candidate (0 where a candidate does not exist). Any
 * output may be NULL. The first call per (device, order) measures.
 */
stp_status stp_autotune(stp_handle h, int* variant, double* us_per_element,
                        double* us_variants);

/*
 * Batched FP64 launch that allocates nothing. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc where they
 * run the predictor (a host that owns all device memory through its own pool,
 * a thread that must not take the device-wide synchronisation an allocation
 * can cause, a device already handed out in full). stp_batch_create allocates
 * a work list, a work counter and scratch buffers; this call instead keeps its
 * scratch - the work counter and one parking area per CTA for the new Taylor
 * terms of order 11 (N = 12) - in one 24 MiB array that is part of
 * the library's device image (every GPU that loads the library holds it until
 * the process exits), and passes the set descriptors as kernel parameters.
 *
 *   nsets <= 128 sets, each as in stp_batch_set (FP64 handles, device
 *   buffers, outputs not overlapping any input or other output); results
 *   equal stp_predict's for every set (bit for bit up to order 10, N <= 11; to
 *   rounding at N = 12, where this path keeps a per-node body that parks its
 *   new Taylor terms in the scratch array). Enqueued on `stream`, asynchronous.
 *   Returns STP_ERR_INVALID_ARG when nsets exceeds 128 or the call would
 *   need more than the 24 MiB scratch (a device with more than about 190 SMs
 *   running order 11), STP_ERR_UNSUPPORTED for non-FP64 handles.
 *
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it together with the identity of the device's
 * current CUDA context; make that first call before any stream capture. After
 * cudaDeviceReset (or any new context on the device) the module can load at
 * another address: the first call in the new context sees the changed
 * identity and looks the address up again, so make that call before any
 * capture as well. Every call uses the same array and it keeps the last call's
 * contents; the call clears the work counter itself. Calls whose work overlaps
 * on the GPU (other streams, or host threads racing) race on the array: order
 * them on one stream. No cudaMalloc, cudaFree or other allocating routine is
 * called; only an argument error records its message in a host string.
 */
stp_status stp_batch_run_static(int nsets, const stp_batch_set* sets, void* stream);

/* stp_batch_run_static with curvilinear sets: metrics is a HOST array of
 * nsets device pointers (the inverse Jacobians of set i in the layout of
 * stp_predict_curvilinear, or NULL for a Cartesian set). The Cartesian sets
 * run in the persistent launch as above; each curvilinear set is one FP64
 * curvilinear launch after it on the same stream, with results equal to its
 * stp_predict_curvilinear. Still no allocating call. STP_ERR_INVALID_ARG for
 * metrics == NULL with nsets > 0, otherwise as stp_batch_run_static and
 * stp_predict_curvilinear. */
stp_status stp_batch_run_static_curvilinear(int nsets, const stp_batch_set* sets,
                                            const double* const* metrics, void* stream);

/* stp_batch_run_static with point sources per set (nsources[i] entries at
 * sources[i], host arrays; metrics as in stp_batch_run_static_curvilinear or
 * NULL). The sources' prepared data are copied into the top of the same
 * static array (no allocation), below which the persistent launch keeps its
 * own scratch; their FP64 response follows the launches on `stream`. The copy
 * is from pageable host memory: the call returns once the data are staged.
 * STP_ERR_INVALID_ARG when the data and the launch's scratch together exceed
 * the 24 MiB array, otherwise as stp_batch_run_static and stp_predict_sources.
 * The paper has no counterpart to the allocation-free form. */
stp_status stp_batch_run_static_sources(int nsets, const stp_batch_set* sets,
                                        const double* const* metrics, const int* nsources,
                                        const stp_point_source* const* sources, void* stream);

/*
 * Served predictor: a continuously batched request loop over many independent
 * simulations (each an element set with its own order, size and material),
 * whose state stays on the device. A request advances one simulation by one
 * STP step; q_{n+1} := avg_n stands in for the corrector (outside the STP),
 * implemented as a swap of two state buffers. Requests of one simulation are
 * served in order, one at a time.
 *
 * The server owns one device pool of hbm_budget_bytes (the HBM budget) and
 * `slots` in-flight batches (each a stream, an event and 24 MiB of scratch).
 * Its scheduler retires finished batches, admits ready simulations into the
 * pool (first fit; when full, idle simulations are evicted least recently
 * used first and their state copied back to pinned host memory), and launches
 * up to 128 ready resident simulations per free slot, whose footprints add up
 * to at most half the budget when slots > 1 (one simulation at least), so the
 * next batch is admitted while one runs. The FP64 ones, Cartesian and
 * curvilinear, run as one persistent launch when the batch is small, or as
 * one persistent launch per shape when it is large; simulations of another
 * precision each run with their own kernel on the same stream. Requests that
 * arrive while others run join the next batch, and batches on different
 * slots overlap on the GPU. The scheduler
 * runs on the calling thread (stp_server_progress / _drain / _run_trace);
 * a server is not thread-safe.
 */
typedef struct stp_server_s* stp_server;

/* Create a server on the current device: hbm_budget_bytes (> 0) is the size
 * of its device pool, allocated here; slots in [1, 8] is the number of
 * batches in flight. *out receives the server (NULL on failure), released
 * with stp_server_destroy. STP_ERR_INVALID_ARG for a NULL out, a budget <= 0
 * or slots outside [1, 8] (checked before any CUDA call); STP_ERR_OOM or
 * STP_ERR_CUDA when the pool or a stream cannot be made. */
stp_status stp_server_create(int64_t hbm_budget_bytes, int slots, stp_server* out);

/* Register a simulation: the handle gives its order, dx, dt and precision;
 * q0 and params ([E][N][N][N][9], [E][N][N][N][3], both host or both device)
 * are copied into the server, which keeps no reference to them. Device
 * buffers whose simulation fits the pool as it is are copied straight into the
 * pool (the simulation starts resident, and its pinned host copies are made
 * only when it is first evicted, so the pinned footprint follows what is
 * evicted); otherwise, and for host buffers, they are copied into
 * server-owned pinned host memory and admitted on the first request. The call
 * is synchronous. *sim_id = 0, 1, ... in
 * order. FP64 simulations share the persistent batched launch; a simulation
 * whose handle runs another precision (read at each launch) gets a launch of
 * its own with the handle's kernel, on the same slot stream. STP_ERR_INVALID_ARG
 * if its footprint (2 states + params + faces) exceeds the budget. The handle
 * must outlive the server. */
stp_status stp_server_add_sim(stp_server s, stp_handle h, int64_t elements, const double* q0,
                              const double* params, int* sim_id);

/* A curvilinear simulation: as stp_server_add_sim, plus its per-node inverse
 * Jacobians (layout of stp_predict_curvilinear; host or device like q0),
 * which stay resident beside the material while the simulation is admitted
 * (its footprint grows by 9N^3 doubles per element). Its steps run as
 * stp_predict_curvilinear (the handle's precision: FP64, float-float or
 * FP32), in a launch of their own on the slot's stream. STP_ERR_INVALID_ARG
 * for a NULL metric, STP_ERR_UNSUPPORTED for a tensor-core precision,
 * otherwise as stp_server_add_sim. */
stp_status stp_server_add_sim_curvilinear(stp_server s, stp_handle h, int64_t elements,
                                          const double* q0, const double* params,
                                          const double* metric, int* sim_id);

/* A simulation with point sources (Sec. II-A: the source term, whose time
 * derivatives enter every Cauchy-Kowalewsky order; the stp_point_source
 * fields as for stp_predict_sources). Cartesian when metric is NULL, else
 * curvilinear as stp_server_add_sim_curvilinear. The sources are validated,
 * projected onto the nodes and uploaded once, by this call, into a small
 * device block the server owns outside its HBM budget (freed by
 * stp_server_destroy); after every step of the simulation their response is
 * added in FP64 to the new average and faces, on the slot's stream and before
 * the step counts as complete. Each step uses the same source derivatives.
 * Errors as stp_server_add_sim and stp_predict_sources (an element outside
 * [0, elements), a position outside [0,1]^3, a non-finite value or
 * nsources < 0: STP_ERR_INVALID_ARG); STP_ERR_OOM when the device block
 * cannot be allocated. nsources = 0 registers a simulation without sources. */
stp_status stp_server_add_sim_sources(stp_server s, stp_handle h, int64_t elements,
                                      const double* q0, const double* params, const double* metric,
                                      int nsources, const stp_point_source* sources, int* sim_id);

/*
 * Order in which the scheduler offers ready simulations to a launch.
 *   policy 0  FIFO: in the order their requests became ready.
 *   policy 1  resident first (the default, age bound 0.05 s): first every
 *             simulation whose oldest request has waited at least age_bound_s
 *             seconds, then those already resident in the pool, then the
 *             rest, each group in FIFO order. A resident simulation needs no
 *             admission copy and evicts nothing; the age bound keeps the
 *             others from waiting without limit.
 * Takes effect at the next scheduler pass. STP_ERR_INVALID_ARG for another
 * policy or a negative or non-finite bound.
 */
stp_status stp_server_set_policy(stp_server s, int policy, double age_bound_s);

/* Queue one step of a simulation (arrival time = now). */
stp_status stp_server_submit(stp_server s, int sim_id);

/* One scheduler pass (non-blocking); *completed = requests retired in it. */
stp_status stp_server_progress(stp_server s, int* completed);

/* Run the scheduler until every queued request has completed. */
stp_status stp_server_drain(stp_server s);

/* Replay a trace in real time: request i of simulation sim_ids[i] arrives
 * t_arrival[i] seconds (sorted) after the call starts. latency[i] receives
 * completion - arrival in seconds (completion = when the scheduler saw the
 * launch finish), *wall_seconds the duration of the replay. */
stp_status stp_server_run_trace(stp_server s, int64_t n, const double* t_arrival, const int* sim_ids,
                                double* latency, double* wall_seconds);

/* Current state q_n and the faces of the last completed step of a simulation
 * (host buffers, may be NULL), and its number of completed steps. Drains. */
stp_status stp_server_read(stp_server s, int sim_id, double* q_host, double* faces_host,
                           int64_t* steps);

/* stats[0..8]: completed requests, launches, admissions, evictions, largest
 * launch (simulations), requests launched, pool bytes in use, peak bytes,
 * summed device time of the launches in microseconds (each from an event
 * before the launch to its completion event; launches on different slots
 * overlap, so the sum can exceed the wall time). */
stp_status stp_server_stats(stp_server s, int64_t* stats);

/* Finish outstanding work and free the server. NULL is a no-op. */
stp_status stp_server_destroy(stp_server s);

/* Interpolation points of the nodal basis (Sec. II-A: Gauss-Legendre or
 * Gauss-Lobatto points). Gauss-Lobatto points include the element's end
 * points, so the face projections phi(0), phi(1) are unit vectors. */
typedef enum {
  STP_NODES_GAUSS_LEGENDRE = 0,
  STP_NODES_GAUSS_LOBATTO = 1
} stp_node_family;

/* As stp_create, on the given node family (stp_create = Gauss-Legendre).
 * Gauss-Lobatto needs N >= 2 (order >= 1): STP_ERR_UNSUPPORTED otherwise, and
 * for an unknown family. Every precision, the batched, allocation-free and
 * served paths take handles of either family. */
stp_status stp_create_nodes(int order, int m, double dx, double dt, stp_node_family nodes,
                            stp_handle* out);

/* Node family of the handle (STP_NODES_GAUSS_LEGENDRE for NULL). */
stp_node_family stp_get_nodes(stp_handle h);

/* Release the handle's device tables and buffers. NULL is a no-op (STP_OK). */
stp_status stp_destroy(stp_handle h);

/*
 * The reference-element tables the library computes for `order` (N = order+1
 * nodes), on the host, without touching a GPU (any output may be NULL):
 *   nodes[N]   Gauss-Legendre nodes on [0,1], ascending (Sec. II-A)
 *   D[N*N]     D[i*N+j] = phi_j'(xi_i), the collocation derivative matrix
 *   phi0[N], phi1[N]   phi_j(0), phi_j(1), the face interpolation vectors
 * Returns STP_ERR_UNSUPPORTED for N outside [1, 12].
 */
stp_status stp_reference_tables(int order, double* nodes, double* D, double* phi0,
                                double* phi1);

/* The same tables on the given node family (STP_ERR_UNSUPPORTED for
 * Gauss-Lobatto with order 0 or an unknown family). */
stp_status stp_reference_tables_nodes(int order, stp_node_family family, double* nodes,
                                      double* D, double* phi0, double* phi1);

/* Nodes per dimension N of the handle, or -1 for an invalid handle. */
int stp_nodes(stp_handle h);

/* Static description of a status code. */
const char* stp_status_string(stp_status s);

/* Message of the last error on the calling thread ("" if none). */
const char* stp_last_error(void);

/*
 * Measure the device's FP64 fused multiply-add throughput (GFLOP/s, 2 flops
 * per FMA) with a dependent-chain-free DFMA loop over all SMs, timed with
 * CUDA events on `stream`. Synchronous. Used as the roofline denominator of
 * the FP64 path.
 */
stp_status stp_measure_fp64_peak(double* gflops, void* stream);

/*
 * The FP64 throughput probe with a choice of instruction: kind 0 = DFMA (as
 * stp_measure_fp64_peak), kind 1 = the warp-level FP64 MMA m8n8k4 (DMMA,
 * 512 flop per warp instruction), the tensor-core alternative for FP64
 * contractions. *gflops receives the best of five launches on `stream`.
 * STP_ERR_INVALID_ARG for another kind or a NULL gflops.
 */
stp_status stp_measure_fp64_peak_kind(int kind, double* gflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* STP_GB300_H */
