"""Pins of the oracle's curvilinear STP (CPU only).

On curvilinear elements (the paper's benchmark meshes, Sec. VI) the
directional derivative (1/h) D_d of the Cartesian step becomes the chain rule
through the per-node inverse Jacobian G[d][j] = dxi_d/dx_j. These pins fix
that step by facts other than the oracle's own code:

* a cube (G = I/h) reduces to the Cartesian oracle, pinned on its own;
* on an affine element with a general (non-symmetric, non-orthogonal) G a
  polynomial plane wave in an arbitrary direction is carried exactly: the
  average is the closed form (F(s) - F(s - c dt)) / (c dt) times the wave's
  eigenvector, derived from the elastic wave equation (P and S waves);
* a rigid rotation R of physical space (G -> G R^T, v -> R v,
  sigma -> R sigma R^T) rotates the outputs, as isotropic elasticity must;
* on tiny curved elements the dense operator assembled with Kronecker
  products, physical derivative first, gives the same Taylor average.

Planted mistakes in a copy of the oracle (a transposed metric, the reference
direction's coefficient matrix in place of the physical one's) fail them.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests import _elastic as ref


def _params(E, N, rng, uniform=None):
    if uniform is not None:
        p = np.zeros((E, N, N, N, 3))
        p[...] = uniform
        return p
    rho = rng.uniform(2, 3, (E, N, N, N))
    cp = rng.uniform(4, 6, (E, N, N, N))
    cs = rng.uniform(1.0, 2.0, (E, N, N, N))  # lambda != mu
    return np.stack([rho, cp, cs], axis=-1)


def _random_metric(E, N, h, rng):
    """Per-node invertible G = (I + 0.3 U)/h, U ~ U[-1,1]^(3x3)."""
    return (np.eye(3) + 0.3 * rng.uniform(-1, 1, (E, N, N, N, 3, 3))) / h


def _rotation(rng):
    Q, R = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def _to_tensor(a):
    """state [..., 9] -> (v [..., 3], sigma [..., 3, 3])"""
    v = a[..., :3]
    sig = np.empty(a.shape[:-1] + (3, 3))
    for i in range(3):
        for j in range(3):
            sig[..., i, j] = a[..., ref.SIG[(i, j)]]
    return v, sig


def _from_tensor(v, sig):
    out = np.empty(v.shape[:-1] + (9,))
    out[..., :3] = v
    for (i, j), s in ref.SIG.items():
        out[..., s] = sig[..., i, j]
    return out


def _rotate(a, R):
    v, sig = _to_tensor(a)
    return _from_tensor(v @ R.T, R @ sig @ R.T)


@pytest.mark.parametrize("N,nodes", [(2, "gl"), (5, "gl"), (4, "gll")])
def test_cube_reduces_to_cartesian(N, nodes):
    E, h, dt = 3, 0.2, 0.004
    rng = np.random.default_rng(N)
    params = _params(E, N, rng)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    G = np.zeros((E, N, N, N, 3, 3))
    G[...] = np.eye(3) / h
    a_c, f_c = oracle.stp(q, params, h, dt, nodes=nodes)
    a, f = oracle.stp_curvilinear(q, params, G, dt, nodes=nodes)
    assert ref.rel_err(a, a_c) <= 1e-14 and ref.rel_err(f, f_c) <= 1e-14


def _wave(n, pol, rho, cp, cs):
    """Eigenvector r and speed c of q = r f(n.x - c t): v = a,
    sigma = -(lam (n.a) I + mu (a n^T + n a^T)) / c (P: a = n; S: a _|_ n)."""
    lam, mu = ref.lame(rho, cp, cs)
    if pol == "P":
        a, c = n, cp
    else:
        a = np.cross(n, [0.3, -0.5, 0.8])
        a /= np.linalg.norm(a)
        c = cs
    sig = -(lam * np.dot(n, a) * np.eye(3) + mu * (np.outer(a, n) + np.outer(n, a))) / c
    return _from_tensor(a, sig), c


@pytest.mark.parametrize("N,nodes", [(3, "gl"), (5, "gl"), (7, "gl"), (4, "gll"), (6, "gll")])
@pytest.mark.parametrize("pol", ["P", "S"])
def test_affine_element_plane_wave_exact(N, nodes, pol):
    rho, cp, cs = 2.3, 4.7, 2.1
    h, dt = 0.25, 0.015
    rng = np.random.default_rng(10 * N + (pol == "S"))
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    r, c = _wave(n, pol, rho, cp, cs)
    f = np.polynomial.Polynomial(rng.uniform(-1, 1, N))  # degree N-1
    F = f.integ()
    avg_of = lambda s: (F(s) - F(s - c * dt)) / (c * dt)
    xi, _ = ref.points(N, nodes)
    # affine elements x = x0 + Jm xi with general (non-symmetric) Jm
    Jms = [h * np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]]),
           h * np.array([[0.8, -0.4, 0.1], [0.35, 1.2, 0.0], [0.05, -0.3, 0.7]])]
    x0s = [np.zeros(3), np.array([0.3, -0.2, 0.5])]
    E = len(Jms)
    q = np.zeros((E, N, N, N, 9))
    avg_x = np.zeros_like(q)
    faces_x = np.zeros((E, 6, N, N, 9))
    G = np.zeros((E, N, N, N, 3, 3))
    Z, Y, X = np.meshgrid(xi, xi, xi, indexing="ij")
    ref_pts = np.stack([X, Y, Z], axis=-1)  # xi of node (z,y,x) = (xi_x, xi_y, xi_z)
    A2, B2 = np.meshgrid(xi, xi, indexing="ij")
    for e in range(E):
        s_node = (x0s[e] + ref_pts @ Jms[e].T) @ n
        q[e] = f(s_node)[..., None] * r
        avg_x[e] = avg_of(s_node)[..., None] * r
        G[e] = np.linalg.inv(Jms[e])
        for d in range(3):
            for side in range(2):
                pts = np.zeros((N, N, 3))
                const = np.full((N, N), float(side))
                if d == 0:
                    pts[..., 0], pts[..., 1], pts[..., 2] = const, B2, A2   # [z][y]
                elif d == 1:
                    pts[..., 0], pts[..., 1], pts[..., 2] = B2, const, A2   # [z][x]
                else:
                    pts[..., 0], pts[..., 1], pts[..., 2] = B2, A2, const   # [y][x]
                s_face = (x0s[e] + pts @ Jms[e].T) @ n
                faces_x[e, 2 * d + side] = avg_of(s_face)[..., None] * r
    params = _params(E, N, rng, uniform=(rho, cp, cs))
    avg, faces = oracle.stp_curvilinear(q, params, G, dt, nodes=nodes)
    assert ref.rel_err(avg, avg_x) <= 1e-12
    assert ref.rel_err(avg - q, avg_x - q) <= 1e-10
    # the face vectors extrapolate to the boundary (sum |phi_j(0)| grows with
    # N), so rounding in the average grows by a few times there
    assert ref.rel_err(faces, faces_x) <= 5e-12


@pytest.mark.parametrize("N", [3, 6])
def test_rotation_covariance(N):
    E, h, dt = 2, 0.2, 0.003
    rng = np.random.default_rng(40 + N)
    params = _params(E, N, rng)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    G = _random_metric(E, N, h, rng)
    R = _rotation(rng)
    avg, faces = oracle.stp_curvilinear(q, params, G, dt)
    avg_r, faces_r = oracle.stp_curvilinear(_rotate(q, R), params, G @ R.T, dt)
    assert ref.rel_err(avg_r, _rotate(avg, R)) <= 1e-13
    assert ref.rel_err(faces_r, _rotate(faces, R)) <= 1e-13
    # and the rotation is not trivial for this data
    assert ref.rel_err(avg_r, avg) > 1e-3


@pytest.mark.parametrize("N,nodes", [(2, "gl"), (3, "gl"), (3, "gll")])
def test_brute_force_dense_operator(N, nodes):
    E, h, dt = 2, 0.25, 0.004
    rng = np.random.default_rng(70 + N)
    params = _params(E, N, rng)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    G = _random_metric(E, N, h, rng)
    avg, faces, terms = oracle.stp_curvilinear(q, params, G, dt, return_terms=True, nodes=nodes)
    p0 = ref.lagrange_phi_numpy(N, 0.0, nodes)
    p1 = ref.lagrange_phi_numpy(N, 1.0, nodes)
    for e in range(E):
        L = ref.dense_operator_curvilinear(N, params[e], G[e], nodes)
        v = q[e].reshape(-1)
        avg_x = ref.dense_time_average(L, v, dt, N + 1).reshape(N, N, N, 9)
        assert ref.rel_err(avg[e], avg_x) <= 1e-13
        p = v.copy()
        for k in range(N + 1):
            assert ref.rel_err(terms[e, k].reshape(-1), p) <= 1e-12
            p = L @ p
        for d, axis in ((0, 2), (1, 1), (2, 0)):
            for side, phi in ((0, p0), (1, p1)):
                fx = np.tensordot(avg_x, phi, axes=([axis], [0]))
                assert ref.rel_err(faces[e, 2 * d + side], fx) <= 1e-13


# --- point sources on curvilinear elements (the node volume is w |det J|) ---

def _source(e, rng, K):
    return {"element": e, "position": tuple(rng.uniform(0, 1, 3)),
            "amplitude": rng.uniform(-1, 1, 9), "derivatives": rng.uniform(-2, 2, K - 1)}


def test_sources_on_a_cube_metric_match_the_cartesian_oracle():
    N, E, h, dt = 4, 3, 0.3, 0.004
    rng = np.random.default_rng(91)
    params = _params(E, N, rng)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    src = [_source(1, rng, N + 1), _source(1, rng, N + 1), _source(2, rng, N + 1)]
    G = np.zeros((E, N, N, N, 3, 3))
    G[...] = np.eye(3) / h
    a_c, f_c = oracle.stp(q, params, h, dt, sources=src)
    a, f = oracle.stp_curvilinear(q, params, G, dt, sources=src)
    assert ref.rel_err(a, a_c) <= 1e-14 and ref.rel_err(f, f_c) <= 1e-14


@pytest.mark.parametrize("N,nodes", [(2, "gl"), (3, "gl"), (3, "gll")])
def test_sources_brute_force_dense_operator(N, nodes):
    """Dense operator physical derivative first, and the source projected
    with numpy's Lagrange basis, quadrature weights and determinant:
    s_node = phi_node(pos) / (w_node |det G_node|^-1) amp f^(k)."""
    rng = np.random.default_rng(95 + N)
    E, K, h, dt = 2, N + 1, 0.3, 0.004
    params = _params(E, N, rng)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    G = _random_metric(E, N, h, rng)
    src = [_source(0, rng, K), _source(0, rng, K), _source(1, rng, K)]
    avg, _, terms = oracle.stp_curvilinear(q, params, G, dt, return_terms=True, nodes=nodes,
                                           sources=src)
    _, w = ref.points(N, nodes)
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    for e in range(E):
        L = ref.dense_operator_curvilinear(N, params[e], G[e], nodes)
        vol = W / np.abs(np.linalg.det(G[e]))  # w_node |det J_node|
        S = np.zeros((K - 1, N, N, N, 9))
        for x in src:
            if x["element"] != e:
                continue
            px = ref.lagrange_phi_numpy(N, x["position"][0], nodes)
            py = ref.lagrange_phi_numpy(N, x["position"][1], nodes)
            pz = ref.lagrange_phi_numpy(N, x["position"][2], nodes)
            P = pz[:, None, None] * py[None, :, None] * px[None, None, :] / vol
            for k in range(K - 1):
                S[k] += P[..., None] * np.asarray(x["amplitude"]) * x["derivatives"][k]
        p = q[e].reshape(-1)
        expect = p.copy()
        for k in range(K - 1):
            p = L @ p + S[k].reshape(-1)
            expect = expect + dt ** (k + 1) / math.factorial(k + 2) * p
            assert ref.rel_err(terms[e, k + 1].reshape(-1), p) <= 1e-12
        assert ref.rel_err(avg[e].reshape(-1), expect) <= 1e-13


def test_rejects_bad_arguments():
    q = np.zeros((1, 3, 3, 3, 9))
    with pytest.raises(ValueError):
        oracle.stp_curvilinear(q, np.zeros((1, 3, 3, 3, 2)), np.zeros((1, 3, 3, 3, 9)), 0.01)
    with pytest.raises(ValueError):
        oracle.stp_curvilinear(q, np.zeros((1, 3, 3, 3, 3)), np.zeros((1, 3, 3, 3, 8)), 0.01)


# --- the pins catch plausible mistakes (planted in copies of the oracle) -----

SRC = os.path.join(os.path.dirname(oracle.__file__), "stp_oracle.c")

MUTANTS = {
    "metric transposed": ("metric[n * 9 + 3 * d + j]", "metric[n * 9 + 3 * j + d]"),
    "reference direction's B": ("elastic_B(j, params[n * 3 + 0]", "elastic_B(d, params[n * 3 + 0]"),
    "diagonal of the metric only": ("const double gdj = metric[n * 9 + 3 * d + j];",
                                    "const double gdj = j == d ? metric[n * 9 + 3 * d + j] : 0.0;"),
}
SOURCE_MUTANTS = {
    "det G taken for det J": ("1.0 / fabs(det3(metric + ((size_t)e * n3 + NODE(z, y, x)) * 9))",
                              "fabs(det3(metric + ((size_t)e * n3 + NODE(z, y, x)) * 9))"),
    "cube volume on a curvilinear element": (
        "const double vol = metric ? 1.0 / fabs(det3(metric + ((size_t)e * n3 + NODE(z, y, x)) * 9))",
        "const double vol = metric ? 1.0"),
}


def _variant(tmp_path, name, text):
    c = tmp_path / f"{name.replace(' ', '_').replace(chr(39), '')}.c"
    so = c.with_suffix(".so")
    c.write_text(text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", str(c),
                    "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_stp_curvilinear.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int64, ctypes.c_double] + [ctypes.c_void_p] * 6
    lib.oracle_stp_curvilinear.restype = ctypes.c_int
    return lib


def _run(lib, q, params, G, dt):
    E, N = q.shape[0], q.shape[1]
    q, params = np.ascontiguousarray(q), np.ascontiguousarray(params)
    G = np.ascontiguousarray(G.reshape(E, N, N, N, 9))
    avg = np.empty_like(q)
    faces = np.empty((E, 6, N, N, 9))
    assert lib.oracle_stp_curvilinear(0, N, N + 1, E, dt, q.ctypes.data, params.ctypes.data,
                                      G.ctypes.data, avg.ctypes.data, faces.ctypes.data,
                                      None) == 0
    return avg, faces


def _pins_pass(lib):
    rng = np.random.default_rng(5)
    N, E, h, dt = 3, 2, 0.25, 0.004
    params = _params(E, N, rng)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    G = _random_metric(E, N, h, rng)
    avg, _ = _run(lib, q, params, G, dt)
    for e in range(E):
        L = ref.dense_operator_curvilinear(N, params[e], G[e])
        avg_x = ref.dense_time_average(L, q[e].reshape(-1), dt, N + 1).reshape(N, N, N, 9)
        if ref.rel_err(avg[e], avg_x) > 1e-13:
            return False
    R = _rotation(rng)
    avg_r, _ = _run(lib, _rotate(q, R), params, G @ R.T, dt)
    return ref.rel_err(avg_r, _rotate(avg, R)) <= 1e-13


def _source_pin_passes(lib):
    """The dense-operator source pin (N = 2) through a compiled variant."""
    rng = np.random.default_rng(7)
    N, E, K, h, dt = 2, 1, 3, 0.3, 0.004
    params = _params(E, N, rng)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    G = np.ascontiguousarray(_random_metric(E, N, h, rng))
    x = _source(0, rng, K)
    lib.oracle_stp_sources_curvilinear.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int64, ctypes.c_double] + \
        [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 7
    lib.oracle_stp_sources_curvilinear.restype = ctypes.c_int
    elem = np.zeros(1, dtype=np.int64)
    pos = np.asarray(x["position"], dtype=np.float64)
    amp = np.asarray(x["amplitude"], dtype=np.float64)
    der = np.asarray(x["derivatives"], dtype=np.float64)
    avg = np.empty_like(q)
    faces = np.empty((E, 6, N, N, 9))
    assert lib.oracle_stp_sources_curvilinear(0, N, K, E, dt, q.ctypes.data, params.ctypes.data,
                                              G.ctypes.data, 1, elem.ctypes.data, pos.ctypes.data,
                                              amp.ctypes.data, der.ctypes.data, avg.ctypes.data,
                                              faces.ctypes.data, None) == 0
    # the independent expectation: dense operator and numpy projection
    _, w = ref.points(N)
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    L = ref.dense_operator_curvilinear(N, params[0], G[0])
    px, py, pz = (ref.lagrange_phi_numpy(N, c) for c in x["position"])
    P = pz[:, None, None] * py[None, :, None] * px[None, None, :] / (W / np.abs(np.linalg.det(G[0])))
    p = q[0].reshape(-1)
    expect = p.copy()
    for k in range(K - 1):
        p = L @ p + (P[..., None] * amp * der[k]).reshape(-1)
        expect = expect + dt ** (k + 1) / math.factorial(k + 2) * p
    return ref.rel_err(avg[0].reshape(-1), expect) <= 1e-13


def test_pins_catch_planted_mistakes(tmp_path):
    text = open(SRC).read()
    assert _pins_pass(_variant(tmp_path, "unmutated", text))
    for name, (old, new) in MUTANTS.items():
        assert text.count(old) == 1, name
        assert not _pins_pass(_variant(tmp_path, name, text.replace(old, new))), name
    assert _source_pin_passes(_variant(tmp_path, "unmutated_sources", text))
    for name, (old, new) in SOURCE_MUTANTS.items():
        assert text.count(old) == 1, name
        assert not _source_pin_passes(_variant(tmp_path, name + "_src", text.replace(old, new))), name
