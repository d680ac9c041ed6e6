"""ctypes binding of the C ABI in include/stp.h (argument marshalling only).

Every step of the predictor runs in the CUDA library; this module converts
torch tensors / numpy arrays to pointers and status codes to exceptions. If
the library has not been built, loading fails loudly: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

STP_OK = 0
STP_ERR_INVALID_ARG = -1
STP_ERR_UNSUPPORTED = -2
STP_ERR_OOM = -3
STP_ERR_CUDA = -4
STP_ERR_TIMEOUT = -5

M = 9

_lock = threading.Lock()
_lib = None


class STPError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({detail})")


def library_path() -> str:
    return _build.LIB


def load():
    """Load libstp_gb300.so (build it first with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: build it with "
                               "paper_2003_12787_gb300.build.build() (no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        lib.stp_create.argtypes = [ctypes.c_int, ctypes.c_int, dbl, dbl, ctypes.POINTER(vp)]
        lib.stp_predict.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        lib.stp_predict_host.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        lib.stp_destroy.argtypes = [vp]
        lib.stp_reference_tables.argtypes = [ctypes.c_int, vp, vp, vp, vp]
        lib.stp_create_nodes.argtypes = [ctypes.c_int, ctypes.c_int, dbl, dbl, ctypes.c_int,
                                         ctypes.POINTER(vp)]
        lib.stp_reference_tables_nodes.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
        lib.stp_get_nodes.argtypes = [vp]
        lib.stp_get_nodes.restype = ctypes.c_int
        lib.stp_predict_sources.argtypes = [vp, i64, vp, vp, vp, vp, ctypes.c_int, vp, vp]
        lib.stp_predict_curvilinear.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
        lib.stp_predict_sources_curvilinear.argtypes = [vp, i64, vp, vp, vp, vp, vp,
                                                        ctypes.c_int, vp, vp]
        lib.stp_predict_curvilinear_host.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
        lib.stp_nodes.argtypes = [vp]
        lib.stp_nodes.restype = ctypes.c_int
        lib.stp_status_string.argtypes = [ctypes.c_int]
        lib.stp_status_string.restype = ctypes.c_char_p
        lib.stp_last_error.argtypes = []
        lib.stp_last_error.restype = ctypes.c_char_p
        lib.stp_measure_fp64_peak.argtypes = [ctypes.POINTER(dbl), vp]
        lib.stp_set_precision.argtypes = [vp, ctypes.c_int]
        lib.stp_get_precision.argtypes = [vp]
        lib.stp_get_precision.restype = ctypes.c_int
        lib.stp_device_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint)]
        lib.stp_selftest_bounded_wait.argtypes = [vp, ctypes.c_int, vp]
        lib.stp_selftest_bounded_wait.restype = ctypes.c_int
        lib.stp_batch_create.argtypes = [ctypes.c_int, vp, ctypes.POINTER(vp)]
        lib.stp_batch_launch.argtypes = [vp, vp]
        lib.stp_batch_create_ex.argtypes = [ctypes.c_int, vp, vp, ctypes.POINTER(vp)]
        lib.stp_batch_create_curvilinear.argtypes = [ctypes.c_int, vp, vp, ctypes.POINTER(vp)]
        lib.stp_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(i64)]
        lib.stp_batch_destroy.argtypes = [vp]
        lib.stp_autotune.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(dbl),
                                     ctypes.POINTER(dbl)]
        ci = ctypes.c_int
        lib.stp_face_params.argtypes = [vp, i64, vp, vp, vp]
        lib.stp_face_params.restype = ci
        lib.stp_correct.argtypes = [vp, ci, ci, ci, vp, vp, vp, vp, vp, vp, vp]
        lib.stp_correct.restype = ci
        lib.stp_ader_step.argtypes = [vp, ci, ci, ci, ci, vp, vp, vp, vp, vp, vp]
        lib.stp_ader_step.restype = ci
        lib.stp_batch_run_static.argtypes = [ctypes.c_int, vp, vp]
        lib.stp_batch_run_static.restype = ctypes.c_int
        lib.stp_batch_run_static_curvilinear.argtypes = [ctypes.c_int, vp, vp, vp]
        lib.stp_batch_run_static_curvilinear.restype = ctypes.c_int
        srv = {"stp_server_create": [i64, ctypes.c_int, ctypes.POINTER(vp)],
               "stp_server_add_sim": [vp, vp, i64, vp, vp, ctypes.POINTER(ctypes.c_int)],
               "stp_server_add_sim_curvilinear": [vp, vp, i64, vp, vp, vp,
                                                  ctypes.POINTER(ctypes.c_int)],
               "stp_server_add_sim_sources": [vp, vp, i64, vp, vp, vp, ctypes.c_int, vp,
                                              ctypes.POINTER(ctypes.c_int)],
               "stp_server_submit": [vp, ctypes.c_int],
               "stp_server_set_policy": [vp, ctypes.c_int, ctypes.c_double],
               "stp_server_progress": [vp, ctypes.POINTER(ctypes.c_int)],
               "stp_server_drain": [vp],
               "stp_server_run_trace": [vp, i64, vp, vp, vp, ctypes.POINTER(dbl)],
               "stp_server_read": [vp, ctypes.c_int, vp, vp, ctypes.POINTER(i64)],
               "stp_server_stats": [vp, vp],
               "stp_server_destroy": [vp]}
        for name, args in srv.items():
            getattr(lib, name).argtypes = args
            getattr(lib, name).restype = ctypes.c_int
        for name in ("stp_create", "stp_predict", "stp_predict_host", "stp_destroy",
                     "stp_reference_tables", "stp_measure_fp64_peak", "stp_set_precision",
                     "stp_device_status", "stp_batch_create", "stp_batch_create_ex",
                     "stp_batch_launch",
                     "stp_batch_info", "stp_batch_destroy", "stp_autotune"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != STP_OK:
        lib = load()
        detail = lib.stp_last_error().decode() or lib.stp_status_string(status).decode()
        raise STPError(status, where, detail)


def _ptr(x) -> int | None:
    """Address of a torch tensor, numpy array or raw integer pointer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


NODE_FAMILIES = {"gl": 0, "gll": 1}


def stp_create(order: int, m: int, dx: float, dt: float, nodes="gl") -> int:
    h = ctypes.c_void_p()
    if nodes == "gl":
        _check(load().stp_create(order, m, dx, dt, ctypes.byref(h)), "stp_create")
    else:
        fam = NODE_FAMILIES[nodes] if isinstance(nodes, str) else int(nodes)
        _check(load().stp_create_nodes(order, m, dx, dt, fam, ctypes.byref(h)), "stp_create_nodes")
    return h.value


def stp_get_nodes(h: int) -> int:
    return int(load().stp_get_nodes(h))


def stp_predict(h: int, elements: int, q, params, out_avg, out_faces, stream=None) -> None:
    _check(load().stp_predict(h, elements, _ptr(q), _ptr(params), _ptr(out_avg),
                              _ptr(out_faces), _stream(stream)), "stp_predict")


def stp_predict_host(h: int, elements: int, q, params, out_avg, out_faces, stream=None) -> None:
    _check(load().stp_predict_host(h, elements, _ptr(q), _ptr(params), _ptr(out_avg),
                                   _ptr(out_faces), _stream(stream)), "stp_predict_host")


def stp_face_params(h: int, elements: int, params, face_params, stream=None) -> None:
    _check(load().stp_face_params(h, elements, _ptr(params), _ptr(face_params), _stream(stream)),
           "stp_face_params")


def stp_correct(h: int, grid, q, params, face_params, avg, faces, q_out, stream=None) -> None:
    gx, gy, gz = (int(g) for g in grid)
    _check(load().stp_correct(h, gx, gy, gz, _ptr(q), _ptr(params), _ptr(face_params), _ptr(avg),
                              _ptr(faces), _ptr(q_out), _stream(stream)), "stp_correct")


def stp_ader_step(h: int, grid, steps: int, q, params, face_params, avg, faces,
                  stream=None) -> None:
    gx, gy, gz = (int(g) for g in grid)
    _check(load().stp_ader_step(h, gx, gy, gz, int(steps), _ptr(q), _ptr(params),
                                _ptr(face_params), _ptr(avg), _ptr(faces), _stream(stream)),
           "stp_ader_step")


def stp_destroy(h: int | None) -> None:
    _check(load().stp_destroy(h), "stp_destroy")


def _host_buf(x, n: int, name: str, dtype: str = "float64"):
    """A host buffer the library reads or writes n elements of: the given
    dtype, C-contiguous, at least n elements (None passes through)."""
    if x is None:
        return None
    got = str(getattr(x, "dtype", None)).replace("torch.", "")
    contiguous = x.is_contiguous() if hasattr(x, "is_contiguous") else x.flags["C_CONTIGUOUS"]
    size = x.numel() if hasattr(x, "numel") else x.size
    if getattr(x, "is_cuda", False):
        raise ValueError(f"{name} must be a host buffer")
    if got != dtype or not contiguous or size < n:
        raise ValueError(f"{name} must be a C-contiguous {dtype} buffer of at least {n} "
                         f"elements (got {got}, {size} elements, contiguous={contiguous})")
    return x


def stp_reference_tables(order: int, nodes=None, D=None, phi0=None, phi1=None,
                         family="gl") -> None:
    fam = NODE_FAMILIES[family] if isinstance(family, str) else int(family)
    N = int(order) + 1
    if N >= 1:
        nodes, D = _host_buf(nodes, N, "nodes"), _host_buf(D, N * N, "D")
        phi0, phi1 = _host_buf(phi0, N, "phi0"), _host_buf(phi1, N, "phi1")
    _check(load().stp_reference_tables_nodes(order, fam, _ptr(nodes), _ptr(D), _ptr(phi0),
                                             _ptr(phi1)), "stp_reference_tables_nodes")


def stp_nodes(h: int) -> int:
    return int(load().stp_nodes(h))


def stp_status_string(status: int) -> str:
    return load().stp_status_string(status).decode()


def stp_last_error() -> str:
    return load().stp_last_error().decode()


PRECISIONS = {"fp64": 0, "bf16x2": 1, "bf16x3": 2, "fp16x2": 3, "fp16x3": 4, "fp32": 5, "ff": 6}


def stp_set_precision(h: int, precision) -> None:
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(load().stp_set_precision(h, p), "stp_set_precision")


def stp_get_precision(h: int) -> int:
    return int(load().stp_get_precision(h))


def stp_selftest_bounded_wait(h: int, polls: int, stream=None) -> None:
    _check(load().stp_selftest_bounded_wait(h, int(polls), _stream(stream)),
           "stp_selftest_bounded_wait")


def stp_device_status(h: int, stream=None) -> int:
    """Synchronise `stream`, read and clear the device status word; raises on a timeout bit."""
    flags = ctypes.c_uint()
    _check(load().stp_device_status(h, _stream(stream), ctypes.byref(flags)), "stp_device_status")
    return flags.value


def stp_measure_fp64_peak(stream=None) -> float:
    g = ctypes.c_double()
    _check(load().stp_measure_fp64_peak(ctypes.byref(g), _stream(stream)), "stp_measure_fp64_peak")
    return g.value


def stp_measure_fp64_peak_kind(kind: str, stream=None) -> float:
    """FP64 probe in GFLOP/s with kind "dfma" or "dmma" (warp-level FP64 MMA)."""
    g = ctypes.c_double()
    lib = load()
    lib.stp_measure_fp64_peak_kind.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                               ctypes.c_void_p]
    lib.stp_measure_fp64_peak_kind.restype = ctypes.c_int
    _check(lib.stp_measure_fp64_peak_kind({"dfma": 0, "dmma": 1}[kind], ctypes.byref(g),
                                          _stream(stream)), "stp_measure_fp64_peak_kind")
    return g.value


class PointSource(ctypes.Structure):
    """Mirror of stp_point_source."""
    _fields_ = [("element", ctypes.c_int64), ("position", ctypes.c_double * 3),
                ("amplitude", ctypes.c_double * 9), ("derivatives", ctypes.c_double * 12)]


def _source_array(sources):
    arr = (PointSource * max(1, len(sources)))()
    for i, src in enumerate(sources):
        der = list(src["derivatives"])[:12]
        arr[i] = PointSource(int(src["element"]), (ctypes.c_double * 3)(*src["position"]),
                             (ctypes.c_double * 9)(*src["amplitude"]),
                             (ctypes.c_double * 12)(*(der + [0.0] * (12 - len(der)))))
    return arr


def stp_predict_sources(h: int, elements: int, q, params, out_avg, out_faces, sources,
                        stream=None) -> None:
    """sources: sequence of dicts with "element", "position" (3), "amplitude"
    (9) and "derivatives" (f^(k)(t_n), k = 0..N-1; at most 12 are used)."""
    arr = _source_array(sources)
    _check(load().stp_predict_sources(h, elements, _ptr(q), _ptr(params), _ptr(out_avg),
                                      _ptr(out_faces), len(sources),
                                      ctypes.cast(arr, ctypes.c_void_p), _stream(stream)),
           "stp_predict_sources")


def stp_predict_sources_curvilinear(h: int, elements: int, q, params, metric, out_avg, out_faces,
                                    sources, stream=None) -> None:
    """stp_predict_sources on curvilinear elements (metric: device inverse Jacobians)."""
    arr = _source_array(sources)
    _check(load().stp_predict_sources_curvilinear(h, elements, _ptr(q), _ptr(params), _ptr(metric),
                                                  _ptr(out_avg), _ptr(out_faces), len(sources),
                                                  ctypes.cast(arr, ctypes.c_void_p),
                                                  _stream(stream)),
           "stp_predict_sources_curvilinear")


def stp_predict_curvilinear(h: int, elements: int, q, params, metric, out_avg, out_faces,
                            stream=None) -> None:
    """metric: device [E][N][N][N][9] (or [..][3][3]) float64, dxi_d/dx_j at 3d + j."""
    _check(load().stp_predict_curvilinear(h, elements, _ptr(q), _ptr(params), _ptr(metric),
                                          _ptr(out_avg), _ptr(out_faces), _stream(stream)),
           "stp_predict_curvilinear")


def stp_predict_curvilinear_host(h: int, elements: int, q, params, metric, out_avg, out_faces,
                                 stream=None) -> None:
    """Host tensors in and out (synchronous), as stp_predict_host."""
    _check(load().stp_predict_curvilinear_host(h, elements, _ptr(q), _ptr(params), _ptr(metric),
                                               _ptr(out_avg), _ptr(out_faces), _stream(stream)),
           "stp_predict_curvilinear_host")


class BatchSet(ctypes.Structure):
    """Mirror of stp_batch_set."""
    _fields_ = [("handle", ctypes.c_void_p), ("elements", ctypes.c_int64),
                ("q", ctypes.c_void_p), ("params", ctypes.c_void_p),
                ("out_avg", ctypes.c_void_p), ("out_faces", ctypes.c_void_p)]


def stp_batch_create(sets, shapes=None, metrics=None) -> int:
    """sets: sequence of (handle, elements, q, params, out_avg, out_faces);
    shapes: optional per-set candidate shape index (-1 = autotuned);
    metrics: optional per-set device metric (None for a Cartesian set)."""
    arr = (BatchSet * max(1, len(sets)))()
    for i, (h, E, q, p, a, f) in enumerate(sets):
        arr[i] = BatchSet(h, E, _ptr(q), _ptr(p), _ptr(a), _ptr(f))
    b = ctypes.c_void_p()
    if metrics is not None:
        if shapes is not None:
            raise ValueError("shapes apply to Cartesian FP64 batches only")
        mt = (ctypes.c_void_p * max(1, len(sets)))(*[_ptr(m) for m in metrics])
        _check(load().stp_batch_create_curvilinear(len(sets), ctypes.cast(arr, ctypes.c_void_p),
                                                   ctypes.cast(mt, ctypes.c_void_p),
                                                   ctypes.byref(b)),
               "stp_batch_create_curvilinear")
    elif shapes is None:
        _check(load().stp_batch_create(len(sets), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(b)),
               "stp_batch_create")
    else:
        sh = (ctypes.c_int * max(1, len(sets)))(*[int(x) for x in shapes])
        _check(load().stp_batch_create_ex(len(sets), ctypes.cast(arr, ctypes.c_void_p),
                                          ctypes.cast(sh, ctypes.c_void_p), ctypes.byref(b)),
               "stp_batch_create_ex")
    return b.value


def stp_batch_launch(b: int, stream=None) -> None:
    _check(load().stp_batch_launch(b, _stream(stream)), "stp_batch_launch")


def stp_batch_info(b: int):
    u, c, sm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check(load().stp_batch_info(b, ctypes.byref(u), ctypes.byref(c), ctypes.byref(sm)),
           "stp_batch_info")
    return {"units": u.value, "ctas": c.value, "smem_bytes": sm.value}


def stp_batch_destroy(b: int | None) -> None:
    _check(load().stp_batch_destroy(b), "stp_batch_destroy")


def stp_autotune(h: int):
    v, us = ctypes.c_int(), ctypes.c_double()
    allv = (ctypes.c_double * 2)()
    _check(load().stp_autotune(h, ctypes.byref(v), ctypes.byref(us), allv), "stp_autotune")
    return {"variant": v.value, "us_per_element": us.value, "us_variants": list(allv)}


def _source_lists(sources_per_set, N_of_set=None):
    """Per-set ctypes arrays of PointSource (None or [] for a set without)."""
    n = len(sources_per_set)
    counts = (ctypes.c_int * max(1, n))()
    arrays = []
    ptrs = (ctypes.c_void_p * max(1, n))()
    for i, lst in enumerate(sources_per_set):
        lst = lst or []
        counts[i] = len(lst)
        arr = _source_array(lst) if lst else None
        arrays.append(arr)
        ptrs[i] = ctypes.cast(arr, ctypes.c_void_p).value if arr is not None else None
    return counts, ptrs, arrays


def stp_batch_create_sources(sets, sources_per_set, N_of_set, metrics=None) -> int:
    """A batch plan with per-set point sources (lists of source dicts)."""
    arr = (BatchSet * max(1, len(sets)))()
    for i, (h, E, q, p, a, f) in enumerate(sets):
        arr[i] = BatchSet(h, E, _ptr(q), _ptr(p), _ptr(a), _ptr(f))
    counts, ptrs, keep = _source_lists(sources_per_set, N_of_set)
    mt = None
    if metrics is not None:
        mt = (ctypes.c_void_p * max(1, len(sets)))(*[_ptr(m) for m in metrics])
    out = ctypes.c_void_p()
    lib = load()
    lib.stp_batch_create_sources.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_void_p)]
    lib.stp_batch_create_sources.restype = ctypes.c_int
    _check(lib.stp_batch_create_sources(len(sets), ctypes.cast(arr, ctypes.c_void_p),
                                        ctypes.cast(mt, ctypes.c_void_p) if mt is not None else None,
                                        ctypes.cast(counts, ctypes.c_void_p),
                                        ctypes.cast(ptrs, ctypes.c_void_p), ctypes.byref(out)),
           "stp_batch_create_sources")
    del keep
    return out.value


def stp_batch_run_static_sources(sets, sources_per_set, N_of_set, stream=None, metrics=None) -> None:
    """The allocation-free batched launch with per-set point sources."""
    arr = (BatchSet * max(1, len(sets)))()
    for i, (h, E, q, p, a, f) in enumerate(sets):
        arr[i] = BatchSet(h, E, _ptr(q), _ptr(p), _ptr(a), _ptr(f))
    counts, ptrs, keep = _source_lists(sources_per_set, N_of_set)
    mt = None
    if metrics is not None:
        mt = (ctypes.c_void_p * max(1, len(sets)))(*[_ptr(m) for m in metrics])
    lib = load()
    lib.stp_batch_run_static_sources.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.stp_batch_run_static_sources.restype = ctypes.c_int
    _check(lib.stp_batch_run_static_sources(len(sets), ctypes.cast(arr, ctypes.c_void_p),
                                            ctypes.cast(mt, ctypes.c_void_p) if mt is not None else None,
                                            ctypes.cast(counts, ctypes.c_void_p),
                                            ctypes.cast(ptrs, ctypes.c_void_p), _stream(stream)),
           "stp_batch_run_static_sources")
    del keep


def stp_batch_run_static(sets, stream=None, metrics=None) -> None:
    """The allocation-free batched launch; sets as for stp_batch_create;
    metrics: optional per-set device metric (None for a Cartesian set)."""
    arr = (BatchSet * max(1, len(sets)))()
    for i, (h, E, q, p, a, f) in enumerate(sets):
        arr[i] = BatchSet(h, E, _ptr(q), _ptr(p), _ptr(a), _ptr(f))
    if metrics is None:
        _check(load().stp_batch_run_static(len(sets), ctypes.cast(arr, ctypes.c_void_p),
                                           _stream(stream)), "stp_batch_run_static")
    else:
        mt = (ctypes.c_void_p * max(1, len(sets)))(*[_ptr(m) for m in metrics])
        _check(load().stp_batch_run_static_curvilinear(len(sets), ctypes.cast(arr, ctypes.c_void_p),
                                                       ctypes.cast(mt, ctypes.c_void_p),
                                                       _stream(stream)),
               "stp_batch_run_static_curvilinear")


def stp_server_create(hbm_budget_bytes: int, slots: int = 3) -> int:
    h = ctypes.c_void_p()
    _check(load().stp_server_create(int(hbm_budget_bytes), int(slots), ctypes.byref(h)),
           "stp_server_create")
    return h.value


def stp_server_add_sim(srv: int, handle: int, elements: int, q0, params, metric=None,
                       sources=None) -> int:
    """metric: optional inverse Jacobians of a curvilinear simulation;
    sources: optional point sources (dicts as for stp_predict_sources), added
    after every step of the simulation."""
    i = ctypes.c_int()
    if sources:
        arr = _source_array(sources)
        _check(load().stp_server_add_sim_sources(srv, handle, elements, _ptr(q0), _ptr(params),
                                                 None if metric is None else _ptr(metric),
                                                 len(sources), ctypes.cast(arr, ctypes.c_void_p),
                                                 ctypes.byref(i)), "stp_server_add_sim_sources")
    elif metric is None:
        _check(load().stp_server_add_sim(srv, handle, elements, _ptr(q0), _ptr(params),
                                         ctypes.byref(i)), "stp_server_add_sim")
    else:
        _check(load().stp_server_add_sim_curvilinear(srv, handle, elements, _ptr(q0), _ptr(params),
                                                     _ptr(metric), ctypes.byref(i)),
               "stp_server_add_sim_curvilinear")
    return i.value


def stp_server_set_policy(srv: int, policy: int, age_bound_s: float = 0.05) -> None:
    """Ready order of the scheduler: 0 FIFO, 1 resident first with an age bound."""
    _check(load().stp_server_set_policy(srv, int(policy), float(age_bound_s)),
           "stp_server_set_policy")


def stp_server_submit(srv: int, sim_id: int) -> None:
    _check(load().stp_server_submit(srv, sim_id), "stp_server_submit")


def stp_server_progress(srv: int) -> int:
    n = ctypes.c_int()
    _check(load().stp_server_progress(srv, ctypes.byref(n)), "stp_server_progress")
    return n.value


def stp_server_drain(srv: int) -> None:
    _check(load().stp_server_drain(srv), "stp_server_drain")


def stp_server_run_trace(srv: int, t_arrival, sim_ids, latency) -> float:
    """t_arrival float64[n] (sorted, seconds), sim_ids int32[n], latency float64[n] out."""
    n = len(t_arrival)
    _host_buf(t_arrival, n, "t_arrival")
    _host_buf(sim_ids, n, "sim_ids", "int32")
    _host_buf(latency, n, "latency")
    wall = ctypes.c_double()
    _check(load().stp_server_run_trace(srv, len(t_arrival), _ptr(t_arrival), _ptr(sim_ids),
                                       _ptr(latency), ctypes.byref(wall)), "stp_server_run_trace")
    return wall.value


def stp_server_read(srv: int, sim_id: int, q_host=None, faces_host=None) -> int:
    steps = ctypes.c_int64()
    _check(load().stp_server_read(srv, sim_id, _ptr(q_host), _ptr(faces_host), ctypes.byref(steps)),
           "stp_server_read")
    return steps.value


def stp_server_stats(srv: int) -> dict:
    arr = (ctypes.c_int64 * 9)()
    _check(load().stp_server_stats(srv, ctypes.cast(arr, ctypes.c_void_p)), "stp_server_stats")
    keys = ["completed", "launches", "admissions", "evictions", "max_batch", "requests_launched",
            "pool_bytes_in_use", "pool_bytes_peak", "kernel_us"]
    return dict(zip(keys, list(arr)))


def stp_server_destroy(srv: int | None) -> None:
    _check(load().stp_server_destroy(srv), "stp_server_destroy")
