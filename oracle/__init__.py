"""Plain FP64 CPU oracle of the linear ADER-DG Space-Time Predictor.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers. The product path (the CUDA library and
its binding) never imports this package, and this package imports nothing from
the product.

The arithmetic lives in ``stp_oracle.c`` (plain C, one element at a time,
dense 9x9 operators, no blocking or fusion); this module compiles it with gcc
and marshals numpy arrays into it. See the header of ``stp_oracle.c`` for the
paper's equations it follows and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stp_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "corrector_oracle.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_stp.so")
_lock = threading.Lock()
_lib = None

M = 9  # quantities of the elastic system


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle_stp.so`` with gcc.

    -O3 with -ffp-contract=off keeps plain IEEE binary64 arithmetic (no fused
    multiply-add contraction), so x86 and Arm hosts round identically.
    OpenMP only spreads independent elements over threads.
    """
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-fopenmp"] + _SRCS + ["-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_gl_nodes.argtypes = [ctypes.c_int, dp, dp]
            lib.oracle_gl_nodes.restype = ctypes.c_int
            lib.oracle_tables.argtypes = [ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_tables.restype = ctypes.c_int
            lib.oracle_stp.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                       ctypes.c_double, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
            lib.oracle_stp.restype = ctypes.c_int
            lib.oracle_gll_nodes.argtypes = [ctypes.c_int, dp, dp]
            lib.oracle_gll_nodes.restype = ctypes.c_int
            lib.oracle_tables_nodes.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_tables_nodes.restype = ctypes.c_int
            lib.oracle_stp_nodes.argtypes = [ctypes.c_int] + lib.oracle_stp.argtypes
            lib.oracle_stp_nodes.restype = ctypes.c_int
            lib.oracle_stp_sources.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]
            lib.oracle_stp_sources.restype = ctypes.c_int
            lib.oracle_stp_curvilinear.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int64, ctypes.c_double,
                                                   ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_stp_curvilinear.restype = ctypes.c_int
            lib.oracle_stp_sources_curvilinear.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_stp_sources_curvilinear.restype = ctypes.c_int
            lib.oracle_face_params.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                               ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_face_params.restype = ctypes.c_int
            lib.oracle_correct.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_correct.restype = ctypes.c_int
            lib.oracle_elastic_B.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_void_p]
            lib.oracle_elastic_B.restype = None
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gl_nodes(N: int):
    """Gauss-Legendre nodes and weights on [0,1] (ascending)."""
    xi = np.zeros(N)
    w = np.zeros(N)
    if _load().oracle_gl_nodes(N, _dptr(xi), _dptr(w)) != 0:
        raise ValueError(f"oracle_gl_nodes failed for N={N}")
    return xi, w


def gll_nodes(N: int):
    """Gauss-Lobatto nodes and weights on [0,1] (ascending, N >= 2)."""
    xi = np.zeros(N)
    w = np.zeros(N)
    if _load().oracle_gll_nodes(N, _dptr(xi), _dptr(w)) != 0:
        raise ValueError(f"oracle_gll_nodes failed for N={N}")
    return xi, w


NODE_FAMILIES = {"gl": 0, "gll": 1}


def tables(N: int, nodes: str = "gl"):
    """(xi, D, phi0, phi1): nodes, D[i,j] = phi_j'(xi_i), phi_j(0), phi_j(1).
    nodes: "gl" (Gauss-Legendre) or "gll" (Gauss-Lobatto)."""
    xi = np.zeros(N)
    D = np.zeros((N, N))
    p0 = np.zeros(N)
    p1 = np.zeros(N)
    if _load().oracle_tables_nodes(NODE_FAMILIES[nodes], N, _dptr(xi), _dptr(D), _dptr(p0),
                                   _dptr(p1)) != 0:
        raise ValueError(f"oracle_tables failed for N={N}, nodes={nodes}")
    return xi, D, p0, p1


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().oracle_num_threads())


def _source_arrays(sources, K):
    """(n, elem, pos, amp, der) arrays of a list of point-source dicts."""
    n = len(sources)
    elem = np.array([int(x["element"]) for x in sources], dtype=np.int64)
    pos = np.ascontiguousarray([x["position"] for x in sources], dtype=np.float64).reshape(n, 3)
    amp = np.ascontiguousarray([x["amplitude"] for x in sources], dtype=np.float64).reshape(n, 9)
    der = np.ascontiguousarray([list(x["derivatives"])[:K - 1] for x in sources],
                               dtype=np.float64).reshape(n, max(K - 1, 0))
    if der.shape[1] != K - 1:
        raise ValueError(f"each source needs {K - 1} derivatives")
    return n, elem, pos, amp, der


def stp(q: np.ndarray, params: np.ndarray, h: float, dt: float, K: int | None = None,
        return_terms: bool = False, nodes: str = "gl", sources=None):
    """Run the oracle STP.

    q: [E][N][N][N][9] float64 (z,y,x,quantity); params: [E][N][N][N][3]
    (rho, cp, cs). K = number of Taylor terms q^(0..K-1), default N+1.
    nodes: "gl" (Gauss-Legendre) or "gll" (Gauss-Lobatto).
    sources: optional list of point sources, each a dict with "element",
    "position" (x, y, z in [0,1]), "amplitude" (9 values) and "derivatives"
    (f^(k)(t_n) for k = 0..K-2); see oracle_stp_sources in stp_oracle.c.
    Returns (avg [E][N][N][N][9], faces [E][6][N][N][9]) and, with
    return_terms, every q^(k) as [E][K][N][N][N][9].
    """
    q = np.ascontiguousarray(q, dtype=np.float64)
    params = np.ascontiguousarray(params, dtype=np.float64)
    if q.ndim != 5 or q.shape[4] != M or not (q.shape[1] == q.shape[2] == q.shape[3]):
        raise ValueError(f"q must be [E][N][N][N][9], got {q.shape}")
    E, N = q.shape[0], q.shape[1]
    if params.shape != (E, N, N, N, 3):
        raise ValueError(f"params must be {(E, N, N, N, 3)}, got {params.shape}")
    K = N + 1 if K is None else int(K)
    avg = np.empty_like(q)
    faces = np.empty((E, 6, N, N, M))
    terms = np.empty((E, K, N, N, N, M)) if return_terms else None
    if sources:
        n, elem, pos, amp, der = _source_arrays(sources, K)
        rc = _load().oracle_stp_sources(NODE_FAMILIES[nodes], N, K, E, float(h), float(dt),
                                        q.ctypes.data, params.ctypes.data, n, elem.ctypes.data,
                                        pos.ctypes.data, amp.ctypes.data,
                                        der.ctypes.data if der.size else None, avg.ctypes.data,
                                        faces.ctypes.data,
                                        terms.ctypes.data if terms is not None else None)
    else:
        rc = _load().oracle_stp_nodes(NODE_FAMILIES[nodes], N, K, E, float(h), float(dt),
                                      q.ctypes.data, params.ctypes.data, avg.ctypes.data,
                                      faces.ctypes.data,
                                      terms.ctypes.data if terms is not None else None)
    if rc != 0:
        raise RuntimeError(f"oracle_stp returned {rc}")
    if return_terms:
        return avg, faces, terms
    return avg, faces


def stp_curvilinear(q: np.ndarray, params: np.ndarray, metric: np.ndarray, dt: float,
                    K: int | None = None, return_terms: bool = False, nodes: str = "gl",
                    sources=None):
    """Run the oracle STP on curvilinear elements.

    metric: [E][N][N][N][3][3] (or [..][9]) float64, the inverse Jacobian
    G[d][j] = dxi_d/dx_j of the map from the reference cube [0,1]^3 to
    physical space at every node (xi_1, xi_2, xi_3 along the x, y, z node
    indices); see oracle_stp_curvilinear in stp_oracle.c. Other arguments and
    the outputs as in ``stp`` (no element side: the metric carries the scale);
    point sources project with the node volumes w_node |det J_node|.
    """
    q = np.ascontiguousarray(q, dtype=np.float64)
    params = np.ascontiguousarray(params, dtype=np.float64)
    if q.ndim != 5 or q.shape[4] != M or not (q.shape[1] == q.shape[2] == q.shape[3]):
        raise ValueError(f"q must be [E][N][N][N][9], got {q.shape}")
    E, N = q.shape[0], q.shape[1]
    if params.shape != (E, N, N, N, 3):
        raise ValueError(f"params must be {(E, N, N, N, 3)}, got {params.shape}")
    metric = np.ascontiguousarray(metric, dtype=np.float64).reshape(E, N, N, N, 9)
    K = N + 1 if K is None else int(K)
    avg = np.empty_like(q)
    faces = np.empty((E, 6, N, N, M))
    terms = np.empty((E, K, N, N, N, M)) if return_terms else None
    if sources:
        n, elem, pos, amp, der = _source_arrays(sources, K)
        rc = _load().oracle_stp_sources_curvilinear(
            NODE_FAMILIES[nodes], N, K, E, float(dt), q.ctypes.data, params.ctypes.data,
            metric.ctypes.data, n, elem.ctypes.data, pos.ctypes.data, amp.ctypes.data,
            der.ctypes.data if der.size else None, avg.ctypes.data, faces.ctypes.data,
            terms.ctypes.data if terms is not None else None)
    else:
        rc = _load().oracle_stp_curvilinear(NODE_FAMILIES[nodes], N, K, E, float(dt),
                                            q.ctypes.data, params.ctypes.data, metric.ctypes.data,
                                            avg.ctypes.data, faces.ctypes.data,
                                            terms.ctypes.data if terms is not None else None)
    if rc != 0:
        raise RuntimeError(f"oracle_stp_curvilinear returned {rc}")
    if return_terms:
        return avg, faces, terms
    return avg, faces


def elastic_B(d: int, rho: float, cp: float, cs: float) -> np.ndarray:
    """B_d (9x9) of q_t + sum_d B_d dq/dx_d = 0 for one material point."""
    B = np.zeros((M, M))
    _load().oracle_elastic_B(int(d), float(rho), float(cp), float(cs), B.ctypes.data)
    return B


def face_params(params: np.ndarray, nodes: str = "gl") -> np.ndarray:
    """Face projection of the material: [E][N][N][N][3] -> [E][6][N][N][3]."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    E, N = params.shape[0], params.shape[1]
    out = np.empty((E, 6, N, N, 3))
    if _load().oracle_face_params(NODE_FAMILIES[nodes], N, E, params.ctypes.data,
                                  out.ctypes.data) != 0:
        raise RuntimeError("oracle_face_params failed")
    return out


def correct(q: np.ndarray, params: np.ndarray, avg: np.ndarray, faces: np.ndarray, grid,
            h: float, dt: float, nodes: str = "gl") -> np.ndarray:
    """One corrector step on a periodic grid of gx*gy*gz elements (element
    e = (ez*gy + ey)*gx + ex); see corrector_oracle.c for the flux and the
    readings. avg, faces: the predictor's outputs for q. Returns q(t_n + dt)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    params = np.ascontiguousarray(params, dtype=np.float64)
    avg = np.ascontiguousarray(avg, dtype=np.float64)
    faces = np.ascontiguousarray(faces, dtype=np.float64)
    gx, gy, gz = (int(g) for g in grid)
    E, N = q.shape[0], q.shape[1]
    if E != gx * gy * gz:
        raise ValueError(f"grid {grid} holds {gx * gy * gz} elements, q has {E}")
    if avg.shape != q.shape or faces.shape != (E, 6, N, N, M) or params.shape != (E, N, N, N, 3):
        raise ValueError("avg, faces or params of the wrong shape")
    out = np.empty_like(q)
    rc = _load().oracle_correct(NODE_FAMILIES[nodes], N, gx, gy, gz, float(h), float(dt),
                                q.ctypes.data, params.ctypes.data, avg.ctypes.data,
                                faces.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_correct returned {rc}")
    return out


def ader_steps(q: np.ndarray, params: np.ndarray, grid, h: float, dt: float, steps: int,
               nodes: str = "gl") -> np.ndarray:
    """`steps` full ADER-DG steps (predictor, then corrector) on the periodic
    grid; returns q after the last one."""
    for _ in range(int(steps)):
        avg, faces = stp(q, params, h, dt, nodes=nodes)
        q = correct(q, params, avg, faces, grid, h, dt, nodes=nodes)
    return q
