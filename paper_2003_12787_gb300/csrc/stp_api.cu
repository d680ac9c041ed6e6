// C ABI of the Space-Time Predictor library (declared in include/stp.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "stp_internal.h"

struct stp_handle_s {
  int N = 0;
  int device = -1;
  double dx = 0.0, dt = 0.0;
  stp::HostTables host;
  double* d_tables = nullptr;  // step matrices, phi0, phi1, D (device)
  unsigned int* d_status = nullptr;  // device-side status word (bounded-wait timeouts)
  int eD = 0;                        // binary exponent of max |D| (mixed-precision scaling)
  stp_precision precision = STP_PRECISION_FP64;
  // host-buffer path: chunked pipeline state, created on first use
  static constexpr int kStages = 3;
  cudaStream_t streams[kStages] = {nullptr, nullptr, nullptr};
  cudaEvent_t done[kStages] = {nullptr, nullptr, nullptr};
  double* stage_buf[kStages] = {nullptr, nullptr, nullptr};
  size_t stage_bytes = 0;  // bytes of each stage buffer
};

namespace {

thread_local std::string g_last_error;

stp_status fail(stp_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

stp_status cuda_fail(cudaError_t e, const char* what) {
  return fail(STP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
  return pa < pb + nb && pb < pa + na;
}

// Checks that p is device (or managed) memory reachable from `device`.
stp_status check_device_ptr(const void* p, int device, const char* name) {
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(STP_ERR_INVALID_ARG, std::string(name) + ": not a CUDA pointer");
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return fail(STP_ERR_INVALID_ARG, std::string(name) + ": not device memory");
  if (attr.type == cudaMemoryTypeDevice && attr.device != device)
    return fail(STP_ERR_INVALID_ARG, std::string(name) + ": on another device than the handle");
  return STP_OK;
}

struct Sizes {
  size_t q, params, avg, faces;  // bytes per element
};

Sizes sizes_per_element(int N) {
  const size_t n3 = (size_t)N * N * N;
  return {n3 * stp::kQuantities * 8, n3 * stp::kParams * 8, n3 * stp::kQuantities * 8,
          (size_t)6 * N * N * stp::kQuantities * 8};
}

stp_status validate_common(stp_handle h, int64_t E, const void* q, const void* params,
                           const void* avg, const void* faces) {
  if (!h || h->N < 1) return fail(STP_ERR_INVALID_ARG, "invalid handle");
  if (E < 0) return fail(STP_ERR_INVALID_ARG, "elements < 0");
  if (E == 0) return STP_OK;
  if (!q || !params || !avg || !faces) return fail(STP_ERR_INVALID_ARG, "null buffer");
  if (!aligned16(q) || !aligned16(params) || !aligned16(avg) || !aligned16(faces))
    return fail(STP_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  const Sizes s = sizes_per_element(h->N);
  const size_t E_ = (size_t)E;
  if (E_ > ((size_t)1 << 40) / s.q) return fail(STP_ERR_INVALID_ARG, "elements too large");
  const void* outs[2] = {avg, faces};
  const size_t nout[2] = {s.avg * E_, s.faces * E_};
  const void* ins[2] = {q, params};
  const size_t nin[2] = {s.q * E_, s.params * E_};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      if (overlap(outs[i], nout[i], ins[j], nin[j]))
        return fail(STP_ERR_INVALID_ARG, "an output overlaps an input");
  if (overlap(avg, nout[0], faces, nout[1])) return fail(STP_ERR_INVALID_ARG, "outputs overlap");
  return STP_OK;
}

// One launch of the handle's configured kernel.
cudaError_t launch_configured(stp_handle h, int64_t E, const double* q, const double* params,
                              double* avg, double* faces, cudaStream_t stream) {
  if (h->precision == STP_PRECISION_FP64 || h->N < 2)
    return stp::launch_fp64(h->N, E, q, params, avg, faces, h->d_tables, stream);
  if (h->precision == STP_PRECISION_FP32)
    return stp::launch_fp32(h->N, E, q, params, avg, faces, h->d_tables, h->d_status, stream);
  if (h->precision == STP_PRECISION_FF)
    return stp::launch_ff(h->N, E, q, params, avg, faces, h->d_tables, stream);
  return stp::launch_mixed(h->N, (int)h->precision, E, q, params, avg, faces, h->d_tables,
                           h->d_tables + stp::table_offset_D(h->N), h->dt / h->dx, h->eD,
                           h->d_status, stream);
}

// Checks of stp_predict_curvilinear's arguments beyond validate_common's;
// STP_OK for elements == 0.
stp_status validate_curvilinear(stp_handle h, int64_t E, const double* q, const double* params,
                                const double* metric, const double* avg, const double* faces) {
  stp_status s = validate_common(h, E, q, params, avg, faces);
  if (s != STP_OK || E == 0) return s;
  if (!metric) return fail(STP_ERR_INVALID_ARG, "null metric");
  if (!aligned16(metric)) return fail(STP_ERR_INVALID_ARG, "metric must be 16-byte aligned");
  const Sizes sz = sizes_per_element(h->N);
  const size_t E_ = (size_t)E, nmetric = sz.q * E_;  // 9 doubles per node, like q
  if (overlap(metric, nmetric, avg, sz.avg * E_) || overlap(metric, nmetric, faces, sz.faces * E_))
    return fail(STP_ERR_INVALID_ARG, "an output overlaps the metric");
  const bool other = h->N >= 2 && (h->precision == STP_PRECISION_FF ||
                                   h->precision == STP_PRECISION_FP32);
  if (h->precision != STP_PRECISION_FP64 && !other)
    return fail(STP_ERR_UNSUPPORTED, "curvilinear elements run in FP64, float-float or FP32 only");
  return STP_OK;
}

// One launch of the handle's curvilinear kernel (precision checked above).
cudaError_t launch_curvilinear_configured(stp_handle h, int64_t E, const double* q,
                                          const double* params, const double* metric, double* avg,
                                          double* faces, cudaStream_t st) {
  if (h->N >= 2 && h->precision == STP_PRECISION_FF)
    return stp::launch_ff_curvilinear(h->N, E, q, params, metric, avg, faces, h->d_tables, h->dx, st);
  if (h->N >= 2 && h->precision == STP_PRECISION_FP32)
    return stp::launch_fp32_curvilinear(h->N, E, q, params, metric, avg, faces, h->d_tables, h->dx,
                                        st);
  return stp::launch_curvilinear(h->N, E, q, params, metric, avg, faces, h->d_tables, h->dx, st);
}

}  // namespace

extern "C" {

const char* stp_status_string(stp_status s) {
  switch (s) {
    case STP_OK: return "ok";
    case STP_ERR_INVALID_ARG: return "invalid argument";
    case STP_ERR_UNSUPPORTED: return "unsupported configuration";
    case STP_ERR_OOM: return "out of memory";
    case STP_ERR_CUDA: return "CUDA error";
    case STP_ERR_TIMEOUT: return "device-side wait timed out";
  }
  return "unknown status";
}

const char* stp_last_error(void) { return g_last_error.c_str(); }

stp_status stp_create(int order, int m, double dx, double dt, stp_handle* out) {
  return stp_create_nodes(order, m, dx, dt, STP_NODES_GAUSS_LEGENDRE, out);
}

stp_status stp_create_nodes(int order, int m, double dx, double dt, stp_node_family nodes,
                            stp_handle* out) {
  if (!out) return fail(STP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  const int N = order + 1;
  if (m != stp::kQuantities) return fail(STP_ERR_UNSUPPORTED, "only m = 9 (elastic) is implemented");
  if (N < 1 || N > stp::kMaxNodes) return fail(STP_ERR_UNSUPPORTED, "order must be in [0, 11]");
  if (!(dx > 0.0) || !std::isfinite(dx)) return fail(STP_ERR_INVALID_ARG, "dx must be > 0 and finite");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(STP_ERR_INVALID_ARG, "dt must be > 0 and finite");
  stp_handle h = new (std::nothrow) stp_handle_s;
  if (!h) return fail(STP_ERR_OOM, "host allocation failed");
  h->N = N;
  h->dx = dx;
  h->dt = dt;
  if (nodes != STP_NODES_GAUSS_LEGENDRE && nodes != STP_NODES_GAUSS_LOBATTO) {
    delete h;
    return fail(STP_ERR_UNSUPPORTED, "unknown node family");
  }
  if (nodes == STP_NODES_GAUSS_LOBATTO && N < 2) {
    delete h;
    return fail(STP_ERR_UNSUPPORTED, "Gauss-Lobatto nodes need order >= 1");
  }
  if (!stp::make_tables(N, &h->host, nodes)) {
    delete h;
    return fail(STP_ERR_UNSUPPORTED, "node computation did not converge");
  }
  {
    double dmax = 0.0;
    for (int i = 0; i < N * N; ++i) dmax = std::fmax(dmax, std::fabs(h->host.D[i]));
    std::frexp(dmax, &h->eD);
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
  const int nt = stp::table_doubles(N);
  double buf[stp::kMaxNodes * stp::kMaxNodes * stp::kMaxNodes + 2 * stp::kMaxNodes +
             stp::kMaxNodes * stp::kMaxNodes + stp::kTcRegionBytes / 8];
  stp::make_step_matrices(h->host, dx, dt, buf);
  std::memcpy(buf + N * N * N, h->host.phi0, sizeof(double) * N);
  std::memcpy(buf + N * N * N + N, h->host.phi1, sizeof(double) * N);
  std::memcpy(buf + stp::table_offset_D(N), h->host.D, sizeof(double) * N * N);
  if (!stp::make_tc_tiles(h->host, h->eD, reinterpret_cast<unsigned char*>(buf + stp::table_offset_tc(N)))) {
    delete h;
    return fail(STP_ERR_UNSUPPORTED, "tensor-core tiles of D are not exactly representable");
  }
  e = cudaMalloc(&h->d_tables, sizeof(double) * nt);
  if (e != cudaSuccess) { cudaGetLastError(); delete h; return fail(STP_ERR_OOM, "cudaMalloc of tables failed"); }
  e = cudaMalloc(&h->d_status, 16);
  if (e != cudaSuccess) {
    cudaGetLastError(); cudaFree(h->d_tables); delete h;
    return fail(STP_ERR_OOM, "cudaMalloc of the status word failed");
  }
  e = cudaMemcpy(h->d_tables, buf, sizeof(double) * nt, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, 16);
  if (e != cudaSuccess) { cudaFree(h->d_tables); cudaFree(h->d_status); delete h; return cuda_fail(e, "table upload"); }
  *out = h;
  return STP_OK;
}

stp_status stp_destroy(stp_handle h) {
  if (!h) return STP_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (h->device >= 0) cudaSetDevice(h->device);
  for (int i = 0; i < stp_handle_s::kStages; ++i) {
    if (h->streams[i]) cudaStreamSynchronize(h->streams[i]);
    if (h->stage_buf[i]) cudaFree(h->stage_buf[i]);
    if (h->done[i]) cudaEventDestroy(h->done[i]);
    if (h->streams[i]) cudaStreamDestroy(h->streams[i]);
  }
  if (h->d_tables) cudaFree(h->d_tables);
  if (h->d_status) cudaFree(h->d_status);
  if (prev >= 0) cudaSetDevice(prev);
  delete h;
  return STP_OK;
}

int stp_nodes(stp_handle h) { return h ? h->N : -1; }

stp_node_family stp_get_nodes(stp_handle h) {
  return h ? (stp_node_family)h->host.family : STP_NODES_GAUSS_LEGENDRE;
}

stp_status stp_reference_tables(int order, double* nodes, double* D, double* phi0, double* phi1) {
  return stp_reference_tables_nodes(order, STP_NODES_GAUSS_LEGENDRE, nodes, D, phi0, phi1);
}

stp_status stp_reference_tables_nodes(int order, stp_node_family family, double* nodes, double* D,
                                      double* phi0, double* phi1) {
  const int N = order + 1;
  stp::HostTables t;
  if (N < 1 || N > stp::kMaxNodes || !stp::make_tables(N, &t, family))
    return fail(STP_ERR_UNSUPPORTED, "order out of range or unknown node family");
  if (nodes) std::memcpy(nodes, t.nodes, sizeof(double) * N);
  if (D) std::memcpy(D, t.D, sizeof(double) * N * N);
  if (phi0) std::memcpy(phi0, t.phi0, sizeof(double) * N);
  if (phi1) std::memcpy(phi1, t.phi1, sizeof(double) * N);
  return STP_OK;
}

stp_status stp_predict(stp_handle h, int64_t elements, const double* q, const double* params,
                       double* out_avg, double* out_faces, void* stream) {
  stp_status s = validate_common(h, elements, q, params, out_avg, out_faces);
  if (s != STP_OK || elements == 0) return s;
  // The memory-kind check queries the driver, which stream capture may forbid;
  // while the stream is being captured it is skipped (the other checks hold).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusNone;
  }
  if (cap == cudaStreamCaptureStatusNone) {
    const char* names[4] = {"q", "params", "out_avg", "out_faces"};
    const void* ptrs[4] = {q, params, out_avg, out_faces};
    for (int i = 0; i < 4; ++i)
      if ((s = check_device_ptr(ptrs[i], h->device, names[i])) != STP_OK) return s;
  }
  cudaError_t e = launch_configured(h, elements, q, params, out_avg, out_faces,
                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "STP kernel launch");
  return STP_OK;
}

stp_status stp_predict_curvilinear(stp_handle h, int64_t elements, const double* q,
                                   const double* params, const double* metric, double* out_avg,
                                   double* out_faces, void* stream) {
  stp_status s = validate_curvilinear(h, elements, q, params, metric, out_avg, out_faces);
  if (s != STP_OK || elements == 0) return s;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusNone;
  }
  if (cap == cudaStreamCaptureStatusNone) {
    const char* names[5] = {"q", "params", "metric", "out_avg", "out_faces"};
    const void* ptrs[5] = {q, params, metric, out_avg, out_faces};
    for (int i = 0; i < 5; ++i)
      if ((s = check_device_ptr(ptrs[i], h->device, names[i])) != STP_OK) return s;
  }
  cudaError_t e = launch_curvilinear_configured(h, elements, q, params, metric, out_avg, out_faces,
                                                static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "curvilinear STP kernel launch");
  return STP_OK;
}

}  // extern "C"

namespace {

// phi_j(a) for the handle's nodes (barycentric form, long double; a unit
// vector where a is a node).
void lagrange_at(const stp::HostTables& t, long double a, long double* phi) {
  const int N = t.N;
  long double bw[stp::kMaxNodes];
  for (int j = 0; j < N; ++j) {
    long double prod = 1.0L;
    for (int k = 0; k < N; ++k)
      if (k != j) prod *= ((long double)t.nodes[j] - (long double)t.nodes[k]);
    bw[j] = 1.0L / prod;
  }
  for (int j = 0; j < N; ++j)
    if ((long double)t.nodes[j] == a) {
      for (int i = 0; i < N; ++i) phi[i] = i == j ? 1.0L : 0.0L;
      return;
    }
  long double den = 0.0L;
  for (int k = 0; k < N; ++k) den += bw[k] / (a - (long double)t.nodes[k]);
  for (int j = 0; j < N; ++j) phi[j] = (bw[j] / (a - (long double)t.nodes[j])) / den;
}

}  // namespace

namespace {

// Point sources after the STP of the set (Cartesian when metric is NULL).
// Point-source data of one set, prepared on the host: sources grouped by
// element; per source the nodal projection phi_node(pos) / (w_node dx^3)
// (curvilinear: phi_node(pos) / w_node, the kernel supplies the node volume),
// the amplitude and dt^(k+1)/(k+2)! f^(k).
struct SourceData {
  int N = 0;
  std::vector<stp::SourceGroup> groups;
  std::vector<double> proj, amp, cf;
  // device block layout: groups | proj | amp | cf | scratch (9 N^3 per group)
  static size_t up(size_t b) { return (b + 255) & ~(size_t)255; }
  size_t b_groups() const { return sizeof(stp::SourceGroup) * groups.size(); }
  size_t b_proj() const { return sizeof(double) * proj.size(); }
  size_t b_amp() const { return sizeof(double) * amp.size(); }
  size_t b_cf() const { return sizeof(double) * cf.size(); }
  size_t b_scr() const { return sizeof(double) * groups.size() * 9 * (size_t)N * N * N; }
  size_t bytes() const { return up(b_groups()) + up(b_proj()) + up(b_amp()) + up(b_cf()) + up(b_scr()); }
};

stp_status validate_sources(stp_handle h, int64_t elements, int nsources,
                            const stp_point_source* sources) {
  if (nsources < 0 || (nsources > 0 && !sources))
    return fail(STP_ERR_INVALID_ARG, "bad source list");
  for (int i = 0; i < nsources; ++i) {
    const stp_point_source& src = sources[i];
    if (src.element < 0 || src.element >= elements)
      return fail(STP_ERR_INVALID_ARG, "source " + std::to_string(i) + ": element out of range");
    for (int d = 0; d < 3; ++d)
      if (!(src.position[d] >= 0.0 && src.position[d] <= 1.0))
        return fail(STP_ERR_INVALID_ARG, "source " + std::to_string(i) + ": position outside [0,1]");
    for (int k = 0; k < 9; ++k)
      if (!std::isfinite(src.amplitude[k]))
        return fail(STP_ERR_INVALID_ARG, "source " + std::to_string(i) + ": non-finite amplitude");
    for (int k = 0; k < h->N; ++k)
      if (!std::isfinite(src.derivatives[k]))
        return fail(STP_ERR_INVALID_ARG, "source " + std::to_string(i) + ": non-finite derivative");
  }
  return STP_OK;
}

void prepare_sources(stp_handle h, bool curvilinear, int nsources, const stp_point_source* sources,
                     SourceData* out) {
  const int N = h->N, N3 = N * N * N;
  out->N = N;
  out->groups.clear();
  std::vector<int> order(nsources);
  for (int i = 0; i < nsources; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return sources[a].element < sources[b].element; });
  out->proj.assign((size_t)nsources * N3, 0.0);
  out->amp.assign((size_t)nsources * 9, 0.0);
  out->cf.assign((size_t)nsources * N, 0.0);
  const long double h3 = curvilinear ? 1.0L : (long double)h->dx * h->dx * h->dx;
  for (int r = 0; r < nsources; ++r) {
    const stp_point_source& src = sources[order[r]];
    if (out->groups.empty() || out->groups.back().element != src.element)
      out->groups.push_back(stp::SourceGroup{src.element, r, 0});
    ++out->groups.back().count;
    long double px[stp::kMaxNodes], py[stp::kMaxNodes], pz[stp::kMaxNodes];
    lagrange_at(h->host, src.position[0], px);
    lagrange_at(h->host, src.position[1], py);
    lagrange_at(h->host, src.position[2], pz);
    const double* w = h->host.weights;
    for (int z = 0; z < N; ++z)
      for (int y = 0; y < N; ++y)
        for (int x = 0; x < N; ++x)
          out->proj[(size_t)r * N3 + (z * N + y) * N + x] =
              (double)(pz[z] * py[y] * px[x] / ((long double)w[z] * w[y] * w[x] * h3));
    for (int k = 0; k < 9; ++k) out->amp[(size_t)r * 9 + k] = src.amplitude[k];
    long double c = 1.0L;  // dt^(k+1) / (k+2)!
    for (int k = 0; k < N; ++k) {
      c = c * (long double)h->dt / (long double)(k + 2);
      out->cf[(size_t)r * N + k] = (double)(c * (long double)src.derivatives[k]);
    }
  }
}

// Copies the prepared data into a device block of sd.bytes() bytes on `st`.
cudaError_t upload_sources(const SourceData& sd, char* d, cudaStream_t st) {
  char* d_proj = d + SourceData::up(sd.b_groups());
  char* d_amp = d_proj + SourceData::up(sd.b_proj());
  char* d_cf = d_amp + SourceData::up(sd.b_amp());
  cudaError_t e = cudaMemcpyAsync(d, sd.groups.data(), sd.b_groups(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_proj, sd.proj.data(), sd.b_proj(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_amp, sd.amp.data(), sd.b_amp(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cf, sd.cf.data(), sd.b_cf(), cudaMemcpyHostToDevice, st);
  return e;
}

// The sources' response of one set from an uploaded block, added to its outputs.
cudaError_t launch_source_block(stp_handle h, const SourceData& sd, const char* d,
                                const double* params, const double* metric, double* avg,
                                double* faces, cudaStream_t st) {
  const char* d_proj = d + SourceData::up(sd.b_groups());
  const char* d_amp = d_proj + SourceData::up(sd.b_proj());
  const char* d_cf = d_amp + SourceData::up(sd.b_amp());
  char* d_scr = const_cast<char*>(d_cf + SourceData::up(sd.b_cf()));
  return stp::launch_sources(sd.N, (int)sd.groups.size(), reinterpret_cast<const stp::SourceGroup*>(d),
                             reinterpret_cast<const double*>(d_proj), reinterpret_cast<const double*>(d_amp),
                             reinterpret_cast<const double*>(d_cf), h->d_tables, params, metric, h->dx,
                             avg, faces, reinterpret_cast<double*>(d_scr), st);
}

}  // namespace

namespace stp {

// Point sources of a served simulation: the prepared data and its device block.
struct ServedSources {
  stp_handle handle = nullptr;
  SourceData sd;
  char* d = nullptr;
};

cudaError_t served_sources_launch(const ServedSources* src, const double* params,
                                  const double* metric, double* avg, double* faces, cudaStream_t st) {
  return launch_source_block(src->handle, src->sd, src->d, params, metric, avg, faces, st);
}

void served_sources_free(ServedSources* src) {
  if (!src) return;
  cudaFree(src->d);
  delete src;
}

}  // namespace stp

namespace {

stp_status predict_sources_impl(stp_handle h, int64_t elements, const double* q,
                                const double* params, const double* metric, double* out_avg,
                                double* out_faces, int nsources, const stp_point_source* sources,
                                void* stream) {
  stp_status s = metric ? validate_curvilinear(h, elements, q, params, metric, out_avg, out_faces)
                        : validate_common(h, elements, q, params, out_avg, out_faces);
  if (s != STP_OK) return s;
  if ((s = validate_sources(h, elements, nsources, sources)) != STP_OK) return s;
  s = metric ? stp_predict_curvilinear(h, elements, q, params, metric, out_avg, out_faces, stream)
             : stp_predict(h, elements, q, params, out_avg, out_faces, stream);
  if (s != STP_OK) return s;
  if (nsources == 0 || elements == 0) return STP_OK;
  SourceData sd;
  prepare_sources(h, metric != nullptr, nsources, sources, &sd);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* d = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), sd.bytes(), st);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(STP_ERR_OOM, "source buffer allocation failed"); }
  e = upload_sources(sd, d, st);
  if (e == cudaSuccess) e = launch_source_block(h, sd, d, params, metric, out_avg, out_faces, st);
  const cudaError_t fe = cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = fe;
  if (e != cudaSuccess) return cuda_fail(e, "point-source launch");
  return STP_OK;
}

}  // namespace

extern "C" {

stp_status stp_predict_sources(stp_handle h, int64_t elements, const double* q, const double* params,
                               double* out_avg, double* out_faces, int nsources,
                               const stp_point_source* sources, void* stream) {
  return predict_sources_impl(h, elements, q, params, nullptr, out_avg, out_faces, nsources, sources,
                              stream);
}

stp_status stp_predict_sources_curvilinear(stp_handle h, int64_t elements, const double* q,
                                           const double* params, const double* metric,
                                           double* out_avg, double* out_faces, int nsources,
                                           const stp_point_source* sources, void* stream) {
  if (!metric && elements > 0) return fail(STP_ERR_INVALID_ARG, "null metric");
  return predict_sources_impl(h, elements, q, params, metric, out_avg, out_faces, nsources, sources,
                              stream);
}

}  // extern "C"

namespace {

// Host-buffer pipeline: chunks of elements cycle through kStages library-owned
// streams, each doing H2D of the chunk's inputs, the kernel, D2H of its
// outputs, so copies of one chunk overlap the kernel of another. metric
// (host, may be NULL) selects the curvilinear kernels.
stp_status predict_host_impl(stp_handle h, int64_t elements, const double* q, const double* params,
                             const double* metric, double* out_avg, double* out_faces,
                             void* stream) {
  const Sizes sz = sizes_per_element(h->N);
  const size_t szm = metric ? sz.q : 0;  // 9 doubles per node, like q
  const size_t per_elem = sz.q + sz.params + szm + sz.avg + sz.faces;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  struct Restore {
    int dev;
    ~Restore() { if (dev >= 0) cudaSetDevice(dev); }
  } restore{prev};
  cudaError_t e;
  // Chunk: ~64 MiB of inputs+outputs per stage, a multiple of the CTA width.
  const int epc = stp::fp64_elements_per_cta(h->N);
  int64_t chunk = (int64_t)((64u << 20) / per_elem);
  chunk = chunk < epc ? epc : (chunk / epc) * epc;
  if (chunk > elements) chunk = elements;
  if (h->stage_bytes < per_elem * (size_t)chunk) {
    for (int i = 0; i < stp_handle_s::kStages; ++i) {
      if (h->streams[i]) cudaStreamSynchronize(h->streams[i]);
      if (h->stage_buf[i]) { cudaFree(h->stage_buf[i]); h->stage_buf[i] = nullptr; }
    }
    h->stage_bytes = 0;
    for (int i = 0; i < stp_handle_s::kStages; ++i) {
      if (!h->streams[i]) {
        if ((e = cudaStreamCreateWithFlags(&h->streams[i], cudaStreamNonBlocking)) != cudaSuccess)
          return cuda_fail(e, "cudaStreamCreate");
        if ((e = cudaEventCreateWithFlags(&h->done[i], cudaEventDisableTiming)) != cudaSuccess)
          return cuda_fail(e, "cudaEventCreate");
      }
      if (cudaMalloc(&h->stage_buf[i], per_elem * (size_t)chunk) != cudaSuccess) {
        cudaGetLastError();
        return fail(STP_ERR_OOM, "cudaMalloc of staging buffers failed");
      }
    }
    h->stage_bytes = per_elem * (size_t)chunk;
  }
  // order after the caller's stream
  cudaEvent_t start;
  if ((e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreate");
  cudaEventRecord(start, static_cast<cudaStream_t>(stream));
  for (int i = 0; i < stp_handle_s::kStages; ++i) cudaStreamWaitEvent(h->streams[i], start, 0);
  cudaEventDestroy(start);

  const char* hq = reinterpret_cast<const char*>(q);
  const char* hp = reinterpret_cast<const char*>(params);
  const char* hm = reinterpret_cast<const char*>(metric);
  char* ha = reinterpret_cast<char*>(out_avg);
  char* hf = reinterpret_cast<char*>(out_faces);
  int stage = 0;
  for (int64_t base = 0; base < elements; base += chunk, stage = (stage + 1) % stp_handle_s::kStages) {
    const int64_t n = (elements - base < chunk) ? elements - base : chunk;
    cudaStream_t st = h->streams[stage];
    char* b = reinterpret_cast<char*>(h->stage_buf[stage]);
    double* dq = reinterpret_cast<double*>(b);
    double* dp = reinterpret_cast<double*>(b + sz.q * chunk);
    double* dm = reinterpret_cast<double*>(b + (sz.q + sz.params) * chunk);
    double* da = reinterpret_cast<double*>(b + (sz.q + sz.params + szm) * chunk);
    double* df = reinterpret_cast<double*>(b + (sz.q + sz.params + szm + sz.avg) * chunk);
    // one stream per stage: its previous chunk's copies and kernel finish first
    if ((e = cudaMemcpyAsync(dq, hq + base * sz.q, n * sz.q, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dp, hp + base * sz.params, n * sz.params, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (metric && (e = cudaMemcpyAsync(dm, hm + base * szm, n * szm, cudaMemcpyHostToDevice, st)) != cudaSuccess))
      return cuda_fail(e, "host-to-device copy");
    e = metric ? launch_curvilinear_configured(h, n, dq, dp, dm, da, df, st)
               : launch_configured(h, n, dq, dp, da, df, st);
    if (e != cudaSuccess) return cuda_fail(e, "STP kernel launch");
    if ((e = cudaMemcpyAsync(ha + base * sz.avg, da, n * sz.avg, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(hf + base * sz.faces, df, n * sz.faces, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "device-to-host copy");
  }
  for (int i = 0; i < stp_handle_s::kStages; ++i) {
    if ((e = cudaStreamSynchronize(h->streams[i])) != cudaSuccess)
      return cuda_fail(e, "host-path synchronisation");
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "host-path copy");
  return STP_OK;
}

}  // namespace

extern "C" {

stp_status stp_predict_host(stp_handle h, int64_t elements, const double* q, const double* params,
                            double* out_avg, double* out_faces, void* stream) {
  stp_status s = validate_common(h, elements, q, params, out_avg, out_faces);
  if (s != STP_OK || elements == 0) return s;
  return predict_host_impl(h, elements, q, params, nullptr, out_avg, out_faces, stream);
}

stp_status stp_predict_curvilinear_host(stp_handle h, int64_t elements, const double* q,
                                        const double* params, const double* metric,
                                        double* out_avg, double* out_faces, void* stream) {
  stp_status s = validate_curvilinear(h, elements, q, params, metric, out_avg, out_faces);
  if (s != STP_OK || elements == 0) return s;
  return predict_host_impl(h, elements, q, params, metric, out_avg, out_faces, stream);
}

stp_status stp_set_precision(stp_handle h, stp_precision p) {
  if (!h) return fail(STP_ERR_INVALID_ARG, "invalid handle");
  if (p < STP_PRECISION_FP64 || p > STP_PRECISION_FF)
    return fail(STP_ERR_INVALID_ARG, "unknown precision");
  if (p == STP_PRECISION_FF && h->N >= 2 && !stp::ff_supported(h->N))
    return fail(STP_ERR_UNSUPPORTED, "no float-float kernel for this order");
  h->precision = p;
  return STP_OK;
}

stp_precision stp_get_precision(stp_handle h) { return h ? h->precision : STP_PRECISION_FP64; }

stp_status stp_selftest_bounded_wait(stp_handle h, int polls, void* stream) {
  if (!h) return fail(STP_ERR_INVALID_ARG, "invalid handle");
  if (polls < 1 || polls > (1 << 22)) return fail(STP_ERR_INVALID_ARG, "polls outside [1, 2^22]");
  cudaError_t e = stp::launch_wait_selftest(h->d_status, polls, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test launch");
  return STP_OK;
}

stp_status stp_device_status(stp_handle h, void* stream, unsigned int* flags) {
  if (!h || !flags) return fail(STP_ERR_INVALID_ARG, "invalid handle or flags pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronisation");
  unsigned int v = 0;
  if ((e = cudaMemcpy(&v, h->d_status, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "status read");
  if ((e = cudaMemset(h->d_status, 0, sizeof(v))) != cudaSuccess) return cuda_fail(e, "status reset");
  *flags = v;
  if (v & 4u)
    return fail(STP_ERR_TIMEOUT, "a bounded device-side wait gave up and the tensor cores were "
                                 "not drained: discard results of this context and recreate it");
  return v ? fail(STP_ERR_TIMEOUT, "a bounded device-side wait gave up") : STP_OK;
}

}  // extern "C"

namespace stp {
const double* stp_handle_tables(stp_handle h) { return h->d_tables; }
double stp_handle_dx(stp_handle h) { return h->dx; }
bool stp_handle_is_fp64(stp_handle h) { return h->precision == STP_PRECISION_FP64 || h->N < 2; }
cudaError_t stp_launch_handle(stp_handle h, int64_t E, const double* q, const double* params,
                              const double* metric, double* avg, double* faces, cudaStream_t st) {
  return metric ? launch_curvilinear_configured(h, E, q, params, metric, avg, faces, st)
                : launch_configured(h, E, q, params, avg, faces, st);
}
}  // namespace stp

struct stp_server_s {
  stp::Server* impl = nullptr;
};

// Point sources of one set of a batch: prepared data, its offset in the
// batch's device block, and the set's buffers the response is added to.
struct BatchSetSources {
  stp_handle h = nullptr;
  SourceData sd;
  size_t off = 0;
  const double* params = nullptr;
  const double* metric = nullptr;
  double* avg = nullptr;
  double* faces = nullptr;
};

struct stp_batch_s {
  stp::BatchPlan* plan = nullptr;   // all sets FP64: per-shape persistent launches
  cudaGraph_t graph = nullptr;      // otherwise: one launch per set, parallel branches
  cudaGraphExec_t exec = nullptr;
  int nsets = 0;
  int device = -1;
  std::vector<BatchSetSources> sources;  // sets with point sources
  char* d_sources = nullptr;             // their data, one device block
};

namespace {

// A graph holding one launch per set (the set's own kernel and precision),
// largest estimated work first, spread round-robin over up to 8 parallel
// branches so that small sets run beside large ones.
cudaError_t capture_set_launches(int nsets, const stp_batch_set* sets, const double* const* metrics,
                                 cudaGraph_t* graph) {
  constexpr int kBranches = 8;
  const int nb = std::max(1, std::min(kBranches, nsets));
  std::vector<int> order(nsets);
  std::vector<double> work(nsets);
  for (int i = 0; i < nsets; ++i) {
    const double n = sets[i].handle->N;
    order[i] = i;
    work[i] = (double)sets[i].elements * (36.0 * std::pow(n, 5) + 66.0 * std::pow(n, 4) + 108.0 * std::pow(n, 3));
    if (metrics && metrics[i]) work[i] *= 1.7;  // curvilinear: every quantity along every direction
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> br(nb, nullptr);
  std::vector<cudaEvent_t> ev(nb + 1, nullptr);
  cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
  for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking);
  for (int b = 0; b <= nb && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming);
  bool capturing = false;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    capturing = true;
    e = cudaEventRecord(ev[nb], origin);  // fork
    for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(br[b], ev[nb], 0);
    for (int k = 0; k < nsets && e == cudaSuccess; ++k) {
      const stp_batch_set& st = sets[order[k]];
      const double* m = metrics ? metrics[order[k]] : nullptr;
      if (st.elements > 0)
        e = m ? launch_curvilinear_configured(st.handle, st.elements, st.q, st.params, m,
                                              st.out_avg, st.out_faces, br[k % nb])
              : launch_configured(st.handle, st.elements, st.q, st.params, st.out_avg,
                                  st.out_faces, br[k % nb]);
    }
    for (int b = 0; b < nb && e == cudaSuccess; ++b) {  // join
      e = cudaEventRecord(ev[b], br[b]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, ev[b], 0);
    }
  }
  if (capturing) {
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(origin, &g);
    if (e == cudaSuccess) e = ce;
    if (e == cudaSuccess) *graph = g;
    else if (g) cudaGraphDestroy(g);
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  for (cudaStream_t x : br)
    if (x) cudaStreamDestroy(x);
  if (origin) cudaStreamDestroy(origin);
  return e;
}

}  // namespace

namespace {

// Plans a batch: the persistent FP64 plan when every set is FP64 (metrics[i],
// when given and not NULL, makes set i curvilinear: one element per unit),
// else a CUDA graph of per-set launches.
stp_status batch_create_impl(int nsets, const stp_batch_set* sets, const int* shapes,
                             const double* const* metrics, stp_batch* out) {
  if (!out) return fail(STP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nsets < 0 || (nsets > 0 && !sets)) return fail(STP_ERR_INVALID_ARG, "bad set list");
  int dev = -1;
  cudaGetDevice(&dev);
  std::vector<int> N(nsets);
  std::vector<int64_t> E(nsets);
  std::vector<const double*> q(nsets), p(nsets), tb(nsets);
  std::vector<double*> a(nsets), f(nsets);
  std::vector<const double*> mt(nsets, nullptr);
  bool any_metric = false;
  for (int i = 0; i < nsets; ++i) {
    const stp_batch_set& st = sets[i];
    const double* m = metrics ? metrics[i] : nullptr;
    stp_status s = m ? validate_curvilinear(st.handle, st.elements, st.q, st.params, m, st.out_avg,
                                            st.out_faces)
                     : validate_common(st.handle, st.elements, st.q, st.params, st.out_avg,
                                       st.out_faces);
    if (s != STP_OK) return fail(s, "set " + std::to_string(i) + ": " + g_last_error);
    if (st.handle->device != dev)
      return fail(STP_ERR_UNSUPPORTED, "set " + std::to_string(i) + ": handle on another device");
    if (st.elements > 0) {
      const char* names[5] = {"q", "params", "out_avg", "out_faces", "metric"};
      const void* ptrs[5] = {st.q, st.params, st.out_avg, st.out_faces, m};
      for (int k = 0; k < (m ? 5 : 4); ++k)
        if ((s = check_device_ptr(ptrs[k], dev, names[k])) != STP_OK)
          return fail(s, "set " + std::to_string(i) + ": " + g_last_error);
    }
    mt[i] = m;
    any_metric = any_metric || (m && st.elements > 0);
    N[i] = st.handle->N;
    E[i] = st.elements;
    q[i] = st.q;
    p[i] = st.params;
    a[i] = st.out_avg;
    f[i] = st.out_faces;
    tb[i] = st.handle->d_tables;
  }
  // outputs of different sets must not overlap each other or any set's inputs
  for (int i = 0; i < nsets; ++i) {
    const Sizes si = sizes_per_element(N[i]);
    const void* oi[2] = {a[i], f[i]};
    const size_t ni[2] = {si.avg * (size_t)E[i], si.faces * (size_t)E[i]};
    for (int j = 0; j < nsets; ++j) {
      if (j == i) continue;
      const Sizes sj = sizes_per_element(N[j]);
      const void* bj[5] = {q[j], p[j], a[j], f[j], mt[j]};
      const size_t nj[5] = {sj.q * (size_t)E[j], sj.params * (size_t)E[j], sj.avg * (size_t)E[j],
                            sj.faces * (size_t)E[j], mt[j] ? sj.q * (size_t)E[j] : 0};
      for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 5; ++y)
          if (ni[x] && nj[y] && overlap(oi[x], ni[x], bj[y], nj[y]))
            return fail(STP_ERR_INVALID_ARG, "outputs of set " + std::to_string(i) +
                                                 " overlap buffers of set " + std::to_string(j));
    }
  }
  // the persistent kernels hold the FP64 bodies, Cartesian and curvilinear
  bool all_fp64 = true;
  for (int i = 0; i < nsets; ++i)
    if (sets[i].handle->precision != STP_PRECISION_FP64) all_fp64 = false;
  stp_batch b = new (std::nothrow) stp_batch_s;
  if (!b) return fail(STP_ERR_OOM, "host allocation failed");
  b->device = dev;
  b->nsets = nsets;
  if (!all_fp64) {
    for (int i = 0; shapes && i < nsets; ++i)
      if (shapes[i] >= 0) {
        delete b;
        return fail(STP_ERR_INVALID_ARG, "shapes apply to all-FP64 batches only");
      }
    cudaError_t e = capture_set_launches(nsets, sets, any_metric ? mt.data() : nullptr, &b->graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (b->graph) cudaGraphDestroy(b->graph);
      delete b;
      return cuda_fail(e, "batch graph");
    }
    *out = b;
    return STP_OK;
  }
  std::vector<int> forced;
  if (shapes) {
    forced.assign(shapes, shapes + nsets);
    for (int i = 0; i < nsets; ++i) {
      if (mt[i] && forced[i] >= 0) {
        delete b;
        return fail(STP_ERR_INVALID_ARG, "set " + std::to_string(i) + ": shapes apply to Cartesian sets");
      }
      int epc[4];
      const int nv = stp::batch_variants_mask(N[i], epc);
      if (forced[i] >= 0 && (forced[i] >= 8 || !((nv >> forced[i]) & 1))) {
        delete b;
        return fail(STP_ERR_INVALID_ARG, "set " + std::to_string(i) + ": no such shape for its order");
      }
    }
  }
  std::vector<double> dxs(nsets);
  for (int i = 0; i < nsets; ++i) dxs[i] = sets[i].handle->dx;
  cudaError_t e = stp::create_plan(nsets, N.data(), E.data(), q.data(), p.data(), a.data(), f.data(),
                                   tb.data(), shapes ? forced.data() : nullptr, &b->plan,
                                   any_metric ? mt.data() : nullptr, dxs.data());
  if (e != cudaSuccess) {
    delete b;
    if (e == cudaErrorMemoryAllocation) return fail(STP_ERR_OOM, "batch plan allocation failed");
    return cuda_fail(e, "batch plan");
  }
  *out = b;
  return STP_OK;
}

}  // namespace

extern "C" {

stp_status stp_batch_create(int nsets, const stp_batch_set* sets, stp_batch* out) {
  return batch_create_impl(nsets, sets, nullptr, nullptr, out);
}

stp_status stp_batch_create_ex(int nsets, const stp_batch_set* sets, const int* shapes,
                               stp_batch* out) {
  return batch_create_impl(nsets, sets, shapes, nullptr, out);
}

stp_status stp_batch_create_curvilinear(int nsets, const stp_batch_set* sets,
                                        const double* const* metrics, stp_batch* out) {
  if (nsets > 0 && !metrics) return fail(STP_ERR_INVALID_ARG, "metrics is NULL");
  return batch_create_impl(nsets, sets, nullptr, metrics, out);
}

stp_status stp_batch_create_sources(int nsets, const stp_batch_set* sets,
                                    const double* const* metrics, const int* nsources,
                                    const stp_point_source* const* sources, stp_batch* out) {
  if (!out) return fail(STP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nsets > 0 && (!sets || !nsources || !sources))
    return fail(STP_ERR_INVALID_ARG, "sets, nsources and sources must not be NULL");
  for (int i = 0; i < nsets; ++i) {
    if (!sets[i].handle || sets[i].handle->N < 1)
      return fail(STP_ERR_INVALID_ARG, "set " + std::to_string(i) + ": invalid handle");
    stp_status s = validate_sources(sets[i].handle, sets[i].elements, nsources[i], sources[i]);
    if (s != STP_OK) return fail(s, "set " + std::to_string(i) + ": " + g_last_error);
  }
  stp_status s = batch_create_impl(nsets, sets, nullptr, metrics, out);
  if (s != STP_OK) return s;
  stp_batch b = *out;
  size_t total = 0;
  for (int i = 0; i < nsets; ++i) {
    if (nsources[i] == 0 || sets[i].elements == 0) continue;
    BatchSetSources bs;
    bs.h = sets[i].handle;
    const double* m = metrics ? metrics[i] : nullptr;
    prepare_sources(bs.h, m != nullptr, nsources[i], sources[i], &bs.sd);
    bs.off = total;
    bs.params = sets[i].params;
    bs.metric = m;
    bs.avg = sets[i].out_avg;
    bs.faces = sets[i].out_faces;
    total += bs.sd.bytes();
    b->sources.push_back(std::move(bs));
  }
  if (total == 0) return STP_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->d_sources), total);
  for (size_t k = 0; e == cudaSuccess && k < b->sources.size(); ++k)
    e = upload_sources(b->sources[k].sd, b->d_sources + b->sources[k].off, nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    stp_batch_destroy(b);
    *out = nullptr;
    return e == cudaErrorMemoryAllocation ? fail(STP_ERR_OOM, "source buffer allocation failed")
                                          : cuda_fail(e, "source upload");
  }
  return STP_OK;
}

stp_status stp_batch_launch(stp_batch b, void* stream) {
  if (!b || (!b->plan && !b->exec)) return fail(STP_ERR_INVALID_ARG, "invalid batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = b->plan ? stp::launch_plan(b->plan, st) : cudaGraphLaunch(b->exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
  // the sets' point-source responses, after the STP of every set on the same stream
  for (const BatchSetSources& bs : b->sources) {
    e = launch_source_block(bs.h, bs.sd, b->d_sources + bs.off, bs.params, bs.metric, bs.avg,
                            bs.faces, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch point-source launch");
  }
  return STP_OK;
}

stp_status stp_batch_info(stp_batch b, int* units, int* ctas, int64_t* smem_bytes) {
  if (!b || (!b->plan && !b->exec)) return fail(STP_ERR_INVALID_ARG, "invalid batch");
  if (!b->plan) {  // one launch per set
    if (units) *units = b->nsets;
    if (ctas) *ctas = 0;
    if (smem_bytes) *smem_bytes = 0;
    return STP_OK;
  }
  size_t sm = 0;
  stp::plan_info(b->plan, units, ctas, &sm);
  if (smem_bytes) *smem_bytes = (int64_t)sm;
  return STP_OK;
}

stp_status stp_batch_destroy(stp_batch b) {
  if (!b) return STP_OK;
  stp::destroy_plan(b->plan);
  cudaFree(b->d_sources);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
  return STP_OK;
}

stp_status stp_autotune(stp_handle h, int* variant, double* us_per_element, double* us_variants) {
  if (!h) return fail(STP_ERR_INVALID_ARG, "invalid handle");
  cudaError_t e = stp::autotune(h->N, h->d_tables, variant, us_per_element, us_variants);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  return STP_OK;
}

}  // extern "C"

namespace {

// The allocation-free batched launch; metrics (host array, may be NULL or hold
// NULLs) marks curvilinear sets, which run in the same persistent launch as
// the Cartesian ones (one element per work unit).
stp_status run_static_impl(int nsets, const stp_batch_set* sets, const double* const* metrics,
                           void* stream, const int* nsources = nullptr,
                           const stp_point_source* const* sources = nullptr) {
  constexpr int kMax = 128;  // the static path's set limit (kernel-parameter descriptors)
  if (nsets < 0 || (nsets > 0 && !sets)) return fail(STP_ERR_INVALID_ARG, "bad set list");
  if (nsets > kMax) return fail(STP_ERR_INVALID_ARG, "more than 128 sets for the static path");
  int dev = -1;
  cudaGetDevice(&dev);
  int N[kMax];
  int64_t E[kMax];
  const double* q[kMax];
  const double* p[kMax];
  const double* tb[kMax];
  const double* mt[kMax];
  double* a[kMax];
  double* f[kMax];
  for (int i = 0; i < nsets; ++i) {
    const stp_batch_set& st = sets[i];
    const double* m = metrics ? metrics[i] : nullptr;
    stp_status s = m ? validate_curvilinear(st.handle, st.elements, st.q, st.params, m, st.out_avg,
                                            st.out_faces)
                     : validate_common(st.handle, st.elements, st.q, st.params, st.out_avg,
                                       st.out_faces);
    if (s != STP_OK) return s;
    if (st.handle->precision != STP_PRECISION_FP64)
      return fail(STP_ERR_UNSUPPORTED, "static batched launches are FP64");
    if (st.handle->device != dev) return fail(STP_ERR_UNSUPPORTED, "handle on another device");
    if (st.elements > 0) {
      const void* ptrs[5] = {st.q, st.params, st.out_avg, st.out_faces, m};
      for (int k = 0; k < (m ? 5 : 4); ++k)
        if ((s = check_device_ptr(ptrs[k], dev, "buffer")) != STP_OK) return s;
    }
    N[i] = st.handle->N;
    E[i] = st.elements;
    q[i] = st.q;
    p[i] = st.params;
    a[i] = st.out_avg;
    f[i] = st.out_faces;
    tb[i] = st.handle->d_tables;
    mt[i] = m;
  }
  for (int i = 0; i < nsets; ++i) {
    const Sizes si = sizes_per_element(N[i]);
    const void* oi[2] = {a[i], f[i]};
    const size_t ni[2] = {si.avg * (size_t)E[i], si.faces * (size_t)E[i]};
    for (int j = 0; j < nsets; ++j) {
      if (j == i) continue;
      const Sizes sj = sizes_per_element(N[j]);
      const void* bj[5] = {q[j], p[j], a[j], f[j], mt[j]};
      const size_t nj[5] = {sj.q * (size_t)E[j], sj.params * (size_t)E[j], sj.avg * (size_t)E[j],
                            sj.faces * (size_t)E[j], mt[j] ? sj.q * (size_t)E[j] : 0};
      for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 5; ++y)
          if (ni[x] && nj[y] && overlap(oi[x], ni[x], bj[y], nj[y]))
            return fail(STP_ERR_INVALID_ARG, "outputs overlap another set's buffers");
    }
  }
  // point sources: prepared on the host, copied into the top of the static
  // array before the launches (the persistent launch keeps below them)
  std::vector<SourceData> sds;
  std::vector<int> src_set;
  size_t reserve = 0;
  if (nsources) {
    for (int i = 0; i < nsets; ++i) {
      stp_status s = validate_sources(sets[i].handle, sets[i].elements, nsources[i],
                                      sources ? sources[i] : nullptr);
      if (s != STP_OK) return fail(s, "set " + std::to_string(i) + ": " + g_last_error);
      if (nsources[i] == 0 || sets[i].elements == 0) continue;
      sds.emplace_back();
      prepare_sources(sets[i].handle, mt[i] != nullptr, nsources[i], sources[i], &sds.back());
      src_set.push_back(i);
      reserve += sds.back().bytes();
    }
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* top = nullptr;
  if (reserve > 0) {
    cudaError_t e = stp::static_scratch_top(reserve, &top);
    if (e == cudaErrorInvalidValue)
      return fail(STP_ERR_INVALID_ARG, "point-source data exceed the 24 MiB static scratch");
    if (e != cudaSuccess) return cuda_fail(e, "static scratch address");
    size_t off = 0;
    for (const SourceData& sd : sds) {
      if ((e = upload_sources(sd, reinterpret_cast<char*>(top) + off, st)) != cudaSuccess)
        return cuda_fail(e, "point-source copy");
      off += sd.bytes();
    }
  }
  // every set, Cartesian and curvilinear, in one persistent launch
  double dxs[kMax];
  for (int i = 0; i < nsets; ++i) dxs[i] = sets[i].handle->dx;
  cudaError_t e = cudaSuccess;
  if (nsets > 0) {
    int too_big = 0;
    e = stp::run_static_batch(nsets, N, E, q, p, a, f, tb, st, &too_big, reserve, mt, dxs);
    if (too_big) return fail(STP_ERR_INVALID_ARG, "the call needs more than the 24 MiB static scratch");
    if (e != cudaSuccess) return cuda_fail(e, "static batched launch");
  }
  size_t off = 0;
  for (size_t k = 0; k < sds.size(); ++k) {
    const stp_batch_set& s = sets[src_set[k]];
    e = launch_source_block(s.handle, sds[k], reinterpret_cast<const char*>(top) + off, s.params,
                            mt[src_set[k]], s.out_avg, s.out_faces, st);
    if (e != cudaSuccess) return cuda_fail(e, "static point-source launch");
    off += sds[k].bytes();
  }
  return STP_OK;
}

}  // namespace

extern "C" {

stp_status stp_batch_run_static_sources(int nsets, const stp_batch_set* sets,
                                        const double* const* metrics, const int* nsources,
                                        const stp_point_source* const* sources, void* stream) {
  if (nsets > 0 && (!nsources || !sources))
    return fail(STP_ERR_INVALID_ARG, "nsources and sources must not be NULL");
  return run_static_impl(nsets, sets, metrics, stream, nsources, sources);
}

stp_status stp_batch_run_static(int nsets, const stp_batch_set* sets, void* stream) {
  return run_static_impl(nsets, sets, nullptr, stream);
}

stp_status stp_batch_run_static_curvilinear(int nsets, const stp_batch_set* sets,
                                            const double* const* metrics, void* stream) {
  if (nsets > 0 && !metrics) return fail(STP_ERR_INVALID_ARG, "metrics is NULL");
  return run_static_impl(nsets, sets, metrics, stream);
}

stp_status stp_server_create(int64_t hbm_budget_bytes, int slots, stp_server* out) {
  if (!out) return fail(STP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes <= 0) return fail(STP_ERR_INVALID_ARG, "budget must be > 0");
  if (slots < 1 || slots > 8) return fail(STP_ERR_INVALID_ARG, "slots must be in [1, 8]");
  stp_server s = new (std::nothrow) stp_server_s;
  if (!s) return fail(STP_ERR_OOM, "host allocation failed");
  cudaError_t e = stp::server_create(hbm_budget_bytes, slots, &s->impl);
  if (e != cudaSuccess) {
    delete s;
    if (e == cudaErrorMemoryAllocation) return fail(STP_ERR_OOM, "server pool allocation failed");
    return cuda_fail(e, "server create");
  }
  *out = s;
  return STP_OK;
}

}  // extern "C"

namespace {

bool is_device_memory(const void* p) {
  cudaPointerAttributes a;
  bool d = false;
  if (cudaPointerGetAttributes(&a, p) == cudaSuccess)
    d = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
  cudaGetLastError();
  return d;
}

stp_status server_add_sim_impl(stp_server s, stp_handle h, int64_t elements, const double* q0,
                               const double* params, const double* metric, int* sim_id,
                               int nsources = 0, const stp_point_source* sources = nullptr) {
  if (!s || !s->impl || !h || !sim_id) return fail(STP_ERR_INVALID_ARG, "null argument");
  if (elements <= 0 || !q0 || !params) return fail(STP_ERR_INVALID_ARG, "bad simulation buffers");
  if (metric && h->N >= 2 && h->precision != STP_PRECISION_FP64 &&
      h->precision != STP_PRECISION_FF && h->precision != STP_PRECISION_FP32)
    return fail(STP_ERR_UNSUPPORTED, "curvilinear elements run in FP64, float-float or FP32 only");
  const bool dq = is_device_memory(q0), dp = is_device_memory(params);
  if (dq != dp || (metric && is_device_memory(metric) != dq))
    return fail(STP_ERR_INVALID_ARG, "q0, params (and metric) must be all host or all device");
  stp::ServedSources* src = nullptr;
  if (nsources > 0) {
    stp_status st = validate_sources(h, elements, nsources, sources);
    if (st != STP_OK) return st;
    src = new (std::nothrow) stp::ServedSources;
    if (!src) return fail(STP_ERR_OOM, "host allocation failed");
    src->handle = h;
    prepare_sources(h, metric != nullptr, nsources, sources, &src->sd);
    cudaError_t e = cudaMalloc(&src->d, src->sd.bytes());
    if (e != cudaSuccess) {
      cudaGetLastError();
      src->d = nullptr;
      stp::served_sources_free(src);
      return fail(STP_ERR_OOM, "cudaMalloc of the point-source data failed");
    }
    e = upload_sources(src->sd, src->d, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
      stp::served_sources_free(src);
      return cuda_fail(e, "point-source upload");
    }
  }
  bool too_big = false;
  cudaError_t e = stp::server_add_sim(s->impl, h, h->N, elements, q0, params, metric, dq, sim_id,
                                      &too_big, src);
  if (e != cudaSuccess || too_big) stp::served_sources_free(src);
  if (too_big) return fail(STP_ERR_INVALID_ARG, "simulation does not fit the HBM budget");
  if (e == cudaErrorMemoryAllocation) return fail(STP_ERR_OOM, "pinned host allocation failed");
  if (e != cudaSuccess) return cuda_fail(e, "add simulation");
  return STP_OK;
}

}  // namespace

extern "C" {

stp_status stp_server_add_sim(stp_server s, stp_handle h, int64_t elements, const double* q0,
                              const double* params, int* sim_id) {
  return server_add_sim_impl(s, h, elements, q0, params, nullptr, sim_id);
}

stp_status stp_server_add_sim_curvilinear(stp_server s, stp_handle h, int64_t elements,
                                          const double* q0, const double* params,
                                          const double* metric, int* sim_id) {
  if (!metric) return fail(STP_ERR_INVALID_ARG, "null metric");
  return server_add_sim_impl(s, h, elements, q0, params, metric, sim_id);
}

stp_status stp_server_add_sim_sources(stp_server s, stp_handle h, int64_t elements,
                                      const double* q0, const double* params, const double* metric,
                                      int nsources, const stp_point_source* sources, int* sim_id) {
  if (nsources < 0 || (nsources > 0 && !sources)) return fail(STP_ERR_INVALID_ARG, "bad source list");
  return server_add_sim_impl(s, h, elements, q0, params, metric, sim_id, nsources, sources);
}

stp_status stp_server_set_policy(stp_server s, int policy, double age_bound_s) {
  if (!s || !s->impl) return fail(STP_ERR_INVALID_ARG, "invalid server");
  if (policy != 0 && policy != 1) return fail(STP_ERR_INVALID_ARG, "policy must be 0 or 1");
  if (!(age_bound_s >= 0.0) || !std::isfinite(age_bound_s))
    return fail(STP_ERR_INVALID_ARG, "age bound must be finite and >= 0");
  stp::server_set_policy(s->impl, policy, age_bound_s);
  return STP_OK;
}

stp_status stp_server_submit(stp_server s, int sim_id) {
  if (!s || !s->impl || sim_id < 0 || sim_id >= stp::server_sims(s->impl))
    return fail(STP_ERR_INVALID_ARG, "bad server or simulation id");
  stp::server_submit(s->impl, sim_id);
  return STP_OK;
}

stp_status stp_server_progress(stp_server s, int* completed) {
  if (!s || !s->impl) return fail(STP_ERR_INVALID_ARG, "invalid server");
  cudaError_t e = stp::server_progress(s->impl, completed);
  if (e != cudaSuccess) return cuda_fail(e, "server progress");
  return STP_OK;
}

stp_status stp_server_drain(stp_server s) {
  if (!s || !s->impl) return fail(STP_ERR_INVALID_ARG, "invalid server");
  cudaError_t e = stp::server_drain(s->impl);
  if (e != cudaSuccess) return cuda_fail(e, "server drain");
  return STP_OK;
}

stp_status stp_server_run_trace(stp_server s, int64_t n, const double* t_arrival, const int* sim_ids,
                                double* latency, double* wall_seconds) {
  if (!s || !s->impl || n < 0 || (n > 0 && (!t_arrival || !sim_ids || !latency)))
    return fail(STP_ERR_INVALID_ARG, "bad trace");
  const int nsims = stp::server_sims(s->impl);
  for (int64_t i = 0; i < n; ++i) {
    if (sim_ids[i] < 0 || sim_ids[i] >= nsims) return fail(STP_ERR_INVALID_ARG, "bad simulation id in trace");
    if (i > 0 && t_arrival[i] < t_arrival[i - 1]) return fail(STP_ERR_INVALID_ARG, "arrivals must be sorted");
  }
  cudaError_t e = stp::server_run_trace(s->impl, n, t_arrival, sim_ids, latency, wall_seconds);
  if (e != cudaSuccess) return cuda_fail(e, "server trace");
  return STP_OK;
}

stp_status stp_server_read(stp_server s, int sim_id, double* q_host, double* faces_host, int64_t* steps) {
  if (!s || !s->impl || sim_id < 0 || sim_id >= stp::server_sims(s->impl))
    return fail(STP_ERR_INVALID_ARG, "bad server or simulation id");
  cudaError_t e = stp::server_read(s->impl, sim_id, q_host, faces_host, steps);
  if (e != cudaSuccess) return cuda_fail(e, "server read");
  return STP_OK;
}

stp_status stp_server_stats(stp_server s, int64_t* stats) {
  if (!s || !s->impl || !stats) return fail(STP_ERR_INVALID_ARG, "invalid server or stats");
  stp::server_stats(s->impl, stats);
  return STP_OK;
}

stp_status stp_server_destroy(stp_server s) {
  if (!s) return STP_OK;
  stp::server_destroy(s->impl);
  delete s;
  return STP_OK;
}

stp_status stp_measure_fp64_peak(double* gflops, void* stream) {
  return stp_measure_fp64_peak_kind(0, gflops, stream);
}

stp_status stp_measure_fp64_peak_kind(int kind, double* gflops, void* stream) {
  if (!gflops) return fail(STP_ERR_INVALID_ARG, "gflops is NULL");
  if (kind != 0 && kind != 1) return fail(STP_ERR_INVALID_ARG, "kind must be 0 (DFMA) or 1 (DMMA)");
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double* sink = nullptr;
  if (cudaMalloc(&sink, 64) != cudaSuccess) { cudaGetLastError(); return fail(STP_ERR_OOM, "cudaMalloc"); }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int threads = 256, blocks = sms * 4, iters = 4096;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  // warm-up long enough (~100 ms) for the SM clock to leave its idle state
  auto launch = [&]() {
    return kind == 0 ? stp::launch_fp64_peak(sink, blocks, threads, iters, st)
                     : stp::launch_dmma_peak(sink, blocks, threads, iters / 4, st);
  };
  for (int rep = 0; rep < 6; ++rep) launch();
  double best = 0.0;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(a, st);
    e = launch();
    cudaEventRecord(b, st);
    if (e != cudaSuccess) break;
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    // DFMA: 8 chains x 2 flop per thread and iteration; DMMA: 4 fragments x
    // 512 flop per warp and iteration
    const double flops = kind == 0 ? 2.0 * 8.0 * iters * (double)blocks * threads
                                   : 4.0 * 512.0 * (iters / 4) * (double)blocks * (threads / 32);
    const double g = flops / (ms * 1e-3) / 1e9;
    if (g > best) best = g;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "fp64 peak probe");
  *gflops = best;
  return STP_OK;
}

}  // extern "C"

// ---- corrector (Sec. II-A) ---------------------------------------------------

namespace {

// Checks of stp_correct's arguments; E receives gx * gy * gz.
stp_status validate_correct(stp_handle h, int gx, int gy, int gz, const double* q,
                            const double* params, const double* face_params, const double* avg,
                            const double* faces, const double* q_out, int64_t* E) {
  if (!h || h->N < 1) return fail(STP_ERR_INVALID_ARG, "invalid handle");
  if (gx < 1 || gy < 1 || gz < 1) return fail(STP_ERR_INVALID_ARG, "grid dimensions must be >= 1");
  const int64_t n = (int64_t)gx * gy * gz;
  if (n > ((int64_t)1 << 31) - 1) return fail(STP_ERR_INVALID_ARG, "grid too large");
  *E = n;
  if (!q || !params || !face_params || !avg || !faces || !q_out)
    return fail(STP_ERR_INVALID_ARG, "null buffer");
  const void* all[6] = {q, params, face_params, avg, faces, q_out};
  for (const void* p : all)
    if (!aligned16(p)) return fail(STP_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  const Sizes s = sizes_per_element(h->N);
  const size_t E_ = (size_t)n, nfp = (size_t)6 * h->N * h->N * 3 * 8 * E_;
  if (E_ > ((size_t)1 << 40) / s.q) return fail(STP_ERR_INVALID_ARG, "elements too large");
  const void* ins[4] = {params, face_params, avg, faces};
  const size_t nin[4] = {s.params * E_, nfp, s.avg * E_, s.faces * E_};
  for (int i = 0; i < 4; ++i)
    if (overlap(q_out, s.q * E_, ins[i], nin[i]))
      return fail(STP_ERR_INVALID_ARG, "q_out overlaps an input other than q");
  if (q_out != q && overlap(q_out, s.q * E_, q, s.q * E_))
    return fail(STP_ERR_INVALID_ARG, "q_out overlaps q without being q");
  return STP_OK;
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cap != cudaStreamCaptureStatusNone;
}

}  // namespace

extern "C" {

stp_status stp_face_params(stp_handle h, int64_t elements, const double* params,
                           double* face_params, void* stream) {
  if (!h || h->N < 1) return fail(STP_ERR_INVALID_ARG, "invalid handle");
  if (elements < 0) return fail(STP_ERR_INVALID_ARG, "elements < 0");
  if (elements == 0) return STP_OK;
  if (!params || !face_params) return fail(STP_ERR_INVALID_ARG, "null buffer");
  if (!aligned16(params) || !aligned16(face_params))
    return fail(STP_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  const Sizes s = sizes_per_element(h->N);
  const size_t E_ = (size_t)elements;
  if (E_ > ((size_t)1 << 40) / s.q) return fail(STP_ERR_INVALID_ARG, "elements too large");
  if (overlap(params, s.params * E_, face_params, (size_t)6 * h->N * h->N * 3 * 8 * E_))
    return fail(STP_ERR_INVALID_ARG, "face_params overlaps params");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!capturing(st)) {
    stp_status r;
    if ((r = check_device_ptr(params, h->device, "params")) != STP_OK) return r;
    if ((r = check_device_ptr(face_params, h->device, "face_params")) != STP_OK) return r;
  }
  cudaError_t e = stp::launch_face_params(h->N, elements, h->d_tables, params, face_params, st);
  if (e != cudaSuccess) return cuda_fail(e, "face-parameter kernel launch");
  return STP_OK;
}

stp_status stp_correct(stp_handle h, int gx, int gy, int gz, const double* q,
                       const double* params, const double* face_params, const double* avg,
                       const double* faces, double* q_out, void* stream) {
  int64_t E = 0;
  stp_status s = validate_correct(h, gx, gy, gz, q, params, face_params, avg, faces, q_out, &E);
  if (s != STP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!capturing(st)) {
    const char* names[6] = {"q", "params", "face_params", "avg", "faces", "q_out"};
    const void* ptrs[6] = {q, params, face_params, avg, faces, q_out};
    for (int i = 0; i < 6; ++i)
      if ((s = check_device_ptr(ptrs[i], h->device, names[i])) != STP_OK) return s;
  }
  cudaError_t e = stp::launch_corrector(h->N, gx, gy, gz, h->host, h->dx, h->dt, h->d_tables, q,
                                        params, face_params, avg, faces, q_out, st);
  if (e != cudaSuccess) return cuda_fail(e, "corrector kernel launch");
  return STP_OK;
}

stp_status stp_ader_step(stp_handle h, int gx, int gy, int gz, int steps, double* q,
                         const double* params, const double* face_params, double* avg,
                         double* faces, void* stream) {
  if (steps < 0) return fail(STP_ERR_INVALID_ARG, "steps < 0");
  int64_t E = 0;
  stp_status s = validate_correct(h, gx, gy, gz, q, params, face_params, avg, faces, q, &E);
  if (s != STP_OK) return s;
  if ((s = validate_common(h, E, q, params, avg, faces)) != STP_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!capturing(st)) {
    const char* names[5] = {"q", "params", "face_params", "avg", "faces"};
    const void* ptrs[5] = {q, params, face_params, avg, faces};
    for (int i = 0; i < 5; ++i)
      if ((s = check_device_ptr(ptrs[i], h->device, names[i])) != STP_OK) return s;
  }
  for (int k = 0; k < steps; ++k) {
    cudaError_t e = launch_configured(h, E, q, params, avg, faces, st);
    if (e != cudaSuccess) return cuda_fail(e, "STP kernel launch");
    e = stp::launch_corrector(h->N, gx, gy, gz, h->host, h->dx, h->dt, h->d_tables, q, params,
                              face_params, avg, faces, q, st);
    if (e != cudaSuccess) return cuda_fail(e, "corrector kernel launch");
  }
  return STP_OK;
}

}  // extern "C"
