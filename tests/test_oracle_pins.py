"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each test checks the oracle against something other than itself: closed-form
quadrature nodes, exactness of the collocation derivative on polynomials,
a terminating Taylor series computed symbolically, the exact Taylor shift of
1-D plane waves through the elastic system, brute-force dense operators, and
invariants (linearity, element independence, axis rotation).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from tests import _elastic as ref

RNG = np.random.default_rng(12345)


# --- nodes and tables --------------------------------------------------------

def closed_form_nodes(N):
    """Gauss-Legendre points on [-1,1] with closed forms (N <= 5)."""
    if N == 1:
        t = [0.0]
    elif N == 2:
        t = [-1 / math.sqrt(3), 1 / math.sqrt(3)]
    elif N == 3:
        t = [-math.sqrt(3 / 5), 0.0, math.sqrt(3 / 5)]
    elif N == 4:
        a = math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5))
        b = math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))
        t = [-b, -a, a, b]
    elif N == 5:
        a = math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3
        b = math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3
        t = [-b, -a, 0.0, a, b]
    return (np.array(t) + 1) / 2


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_nodes_closed_form(N):
    xi, _ = oracle.gl_nodes(N)
    assert np.abs(xi - closed_form_nodes(N)).max() <= 2e-16


@pytest.mark.parametrize("N", range(1, 17))
def test_nodes_and_weights_match_numpy(N):
    xi, w = oracle.gl_nodes(N)
    t, wt = np.polynomial.legendre.leggauss(N)
    assert np.abs(xi - (t + 1) / 2).max() <= 4e-16
    assert np.abs(w - wt / 2).max() <= 4e-15


@pytest.mark.parametrize("N", range(1, 13))
def test_quadrature_exact_to_degree_2N_minus_1(N):
    xi, w = oracle.gl_nodes(N)
    for p in range(2 * N):
        assert abs(np.dot(w, xi ** p) - 1.0 / (p + 1)) <= 2e-15


@pytest.mark.parametrize("N", range(2, 13))
def test_D_exact_on_polynomials(N):
    xi, D, p0, p1 = oracle.tables(N)
    for p in range(N):
        f = xi ** p
        df = p * xi ** (p - 1) if p > 0 else np.zeros(N)
        err = np.abs(D @ f - df).max()
        assert err <= 1e-13 * max(1.0, np.abs(D).max())
        assert abs(p0 @ f - (1.0 if p == 0 else 0.0)) <= 1e-13
        assert abs(p1 @ f - 1.0) <= 1e-13
    assert np.abs(D.sum(axis=1)).max() <= 1e-13 * np.abs(D).max()
    assert abs(p0.sum() - 1) <= 1e-14 and abs(p1.sum() - 1) <= 1e-14


@pytest.mark.parametrize("N", range(2, 13))
def test_tables_match_vandermonde_construction(N):
    _, D, p0, p1 = oracle.tables(N)
    assert ref.rel_err(D, ref.lagrange_D_numpy(N)) <= 1e-12
    assert np.abs(p0 - ref.lagrange_phi_numpy(N, 0.0)).max() <= 1e-12
    assert np.abs(p1 - ref.lagrange_phi_numpy(N, 1.0)).max() <= 1e-12


@pytest.mark.parametrize("N", [2, 5, 8, 12])
def test_D_against_50_digit_barycentric(N):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    xi_d, D, _, _ = oracle.tables(N)
    nodes = [mp.findroot(lambda x: mpmath.legendre(N, 2 * x - 1), mp.mpf(x)) for x in xi_d]
    w = [1 / mpmath.fprod([nodes[j] - nodes[k] for k in range(N) if k != j]) for j in range(N)]
    Dm = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if i != j:
                Dm[i, j] = float((w[j] / w[i]) / (nodes[i] - nodes[j]))
        Dm[i, i] = -sum(Dm[i, j] for j in range(N) if j != i)
    assert np.abs(np.array([float(x) for x in nodes]) - xi_d).max() <= 2e-16
    assert ref.rel_err(D, Dm) <= 2e-14


# --- constant states ---------------------------------------------------------

def random_params(E, N, rng):
    rho = rng.uniform(2, 3, (E, N, N, N))
    cp = rng.uniform(4, 6, (E, N, N, N))
    cs = cp / math.sqrt(3)
    return np.stack([rho, cp, cs], axis=-1)


@pytest.mark.parametrize("N", [2, 4, 7])
def test_constant_state_is_steady(N):
    E = 3
    rng = np.random.default_rng(N)
    params = random_params(E, N, rng)
    q = np.broadcast_to(rng.uniform(-1, 1, (E, 1, 1, 1, 9)), (E, N, N, N, 9)).copy()
    avg, faces, terms = oracle.stp(q, params, h=0.1, dt=0.002, return_terms=True)
    assert ref.rel_err(avg, q) <= 1e-13
    for f in range(6):
        assert ref.rel_err(faces[:, f], q[:, 0]) <= 1e-13
    # q^(1) = L q vanishes up to rounding of the row sums of D (the higher
    # terms amplify that rounding noise, but enter avg scaled by dt^k/(k+1)!)
    _, D, _, _ = oracle.tables(N)
    scale = np.abs(q).max() * np.abs(D).max() / 0.1 * 3 * 6.0 ** 2 * 3.0
    assert np.abs(terms[:, 1]).max() <= 1e-14 * scale


# --- terminating series: polynomial data, uniform material ------------------

def _poly_case(N, rho, cp, cs, h, dt, origins, seed, nodes="gl"):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    rng = np.random.default_rng(seed)
    lam, mu = ref.lame(rho, cp, cs)
    lam_r, mu_r, rho_r = sp.Rational(lam), sp.Rational(mu), sp.Rational(rho)
    # total degree <= N-1 in (x,y,z): inside Q_{N-1} and annihilated by L^N
    monos = [(a, b, c) for a in range(N) for b in range(N) for c in range(N) if a + b + c <= N - 1]
    q0 = []
    for s in range(9):
        coeffs = rng.integers(-3, 4, len(monos))
        q0.append(sum(int(cf) * x ** a * y ** b * z ** c for cf, (a, b, c) in zip(coeffs, monos)))
    terms = [q0]
    while True:
        f = terms[-1]
        grad = [[sp.diff(f[s], v) for s in range(9)] for v in (x, y, z)]
        nxt = [sp.expand(e) for e in ref.elastic_rate(grad, rho_r, lam_r, mu_r)]
        if all(e == 0 for e in nxt):
            break
        terms.append(nxt)
    assert len(terms) <= N
    dt_r = sp.Rational(dt)
    avg_expr = [sp.expand(sum(dt_r ** k / sp.factorial(k + 1) * terms[k][s] for k in range(len(terms))))
                for s in range(9)]
    q0f = [sp.lambdify((x, y, z), e, "numpy") for e in q0]
    avgf = [sp.lambdify((x, y, z), e, "numpy") for e in avg_expr]
    xi, _ = ref.points(N, nodes)
    E = len(origins)
    q = np.zeros((E, N, N, N, 9))
    avg_x = np.zeros_like(q)
    faces_x = np.zeros((E, 6, N, N, 9))
    for e, (ox, oy, oz) in enumerate(origins):
        Z, Y, X = np.meshgrid(oz + xi * h, oy + xi * h, ox + xi * h, indexing="ij")
        for s in range(9):
            q[e, ..., s] = np.broadcast_to(q0f[s](X, Y, Z), (N, N, N))
            avg_x[e, ..., s] = np.broadcast_to(avgf[s](X, Y, Z), (N, N, N))
        P = xi * h
        for d in range(3):
            for side in range(2):
                c = (ox, oy, oz)[d] + side * h
                A, B = np.meshgrid(P, P, indexing="ij")
                if d == 0:   # [z][y]
                    pts = (c + 0 * A, oy + B, oz + A)
                elif d == 1:  # [z][x]
                    pts = (ox + B, c + 0 * A, oz + A)
                else:        # [y][x]
                    pts = (ox + B, oy + A, c + 0 * A)
                for s in range(9):
                    faces_x[e, 2 * d + side, ..., s] = np.broadcast_to(avgf[s](*pts), (N, N))
    params = np.zeros((E, N, N, N, 3))
    params[...] = (rho, cp, cs)
    return q, params, avg_x, faces_x


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_polynomial_data_matches_symbolic_series(N):
    h, dt = 0.5, 0.03
    origins = [(0.0, 0.0, 0.0), (0.5, -1.0, 1.5)]
    # cs != cp/sqrt(3): lambda != mu, so swapped Lame parameters are visible
    q, params, avg_x, faces_x = _poly_case(N, 2.0, 3.0, 1.0, h, dt, origins, seed=N)
    avg, faces = oracle.stp(q, params, h=h, dt=dt)
    assert ref.rel_err(avg, avg_x) <= 1e-12
    assert ref.rel_err(faces, faces_x) <= 1e-12
    # the time-dependent part alone must also agree (not drowned by q itself)
    assert ref.rel_err(avg - q, avg_x - q) <= 1e-10


# --- exact Taylor shift of 1-D plane waves ----------------------------------

def plane_wave_eigvec(axis, pol, rho, cp, cs):
    """Right eigenvector and speed of a wave along `axis` polarised along `pol`."""
    lam, mu = ref.lame(rho, cp, cs)
    r = np.zeros(9)
    r[pol] = 1.0
    if pol == axis:  # P wave
        c = cp
        for j in range(3):
            r[ref.SIG[(j, j)]] = -rho * cp if j == axis else -lam / cp
    else:            # S wave
        c = cs
        r[ref.SIG[(pol, axis)]] = -rho * cs
    return r, c


@pytest.mark.parametrize("N", [3, 5, 8])
@pytest.mark.parametrize("axis,pol", [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0)])
def test_plane_wave_exact_taylor_shift(N, axis, pol):
    rho, cp, cs = 2.3, 4.7, 2.1
    h, dt = 0.25, 0.02
    rng = np.random.default_rng(100 * N + 10 * axis + pol)
    f = np.polynomial.Polynomial(rng.uniform(-1, 1, N))  # degree N-1
    F = f.integ()
    r, c = plane_wave_eigvec(axis, pol, rho, cp, cs)
    xi, _ = ref.gl_points(N)
    origins = np.array([[0.0, 0.0, 0.0], [0.25, 0.5, -0.25]])
    E = len(origins)
    q = np.zeros((E, N, N, N, 9))
    avg_x = np.zeros_like(q)
    for e in range(E):
        coord = origins[e][axis] + xi * h
        shape = [1, 1, 1]
        shape[2 - axis] = N  # array axes are (z, y, x)
        s0 = f(coord).reshape(shape)
        s1 = ((F(coord) - F(coord - c * dt)) / (c * dt)).reshape(shape)
        q[e] = np.broadcast_to(s0[..., None] * r, (N, N, N, 9))
        avg_x[e] = np.broadcast_to(s1[..., None] * r, (N, N, N, 9))
    params = np.zeros((E, N, N, N, 3))
    params[...] = (rho, cp, cs)
    avg, _ = oracle.stp(q, params, h=h, dt=dt)
    assert ref.rel_err(avg, avg_x) <= 1e-12
    assert ref.rel_err(avg - q, avg_x - q) <= 1e-10


# --- brute force: dense operator, heterogeneous material ---------------------

@pytest.mark.parametrize("N", [2, 3])
def test_brute_force_dense_operator(N):
    E = 2
    rng = np.random.default_rng(7 + N)
    params = random_params(E, N, rng)
    params[..., 2] = rng.uniform(1.0, 2.0, (E, N, N, N))  # lambda != mu
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    h, dt = 0.2, 0.004
    avg, faces, terms = oracle.stp(q, params, h=h, dt=dt, return_terms=True)
    p0 = ref.lagrange_phi_numpy(N, 0.0)
    p1 = ref.lagrange_phi_numpy(N, 1.0)
    for e in range(E):
        L = ref.dense_operator(N, h, params[e])
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


@pytest.mark.parametrize("N", [2, 3])
def test_truncation_error_order(N):
    """The STP average is the degree-N Taylor truncation of the exact time
    average of the semi-discrete system, (1/dt) int_0^dt exp(t L) q dt =
    phi_1(dt L) q (matrix exponential of an augmented matrix, scipy). Its
    error is led by the first omitted term, dt^(N+1)/(N+2)! L^(N+1) q, so
    halving dt divides it by about 2^(N+1). A dropped or extra Taylor term,
    or a wrong weight, changes that exponent. Sanity check of the scheme,
    independent of the oracle's own series."""
    from scipy.linalg import expm
    rng = np.random.default_rng(31 + N)
    params = random_params(1, N, rng)
    q = rng.uniform(-1, 1, (1, N, N, N, 9))
    h = 0.5
    L = ref.dense_operator(N, h, params[0])
    v = q[0].reshape(-1)
    n = v.size
    rho = max(abs(np.linalg.eigvals(L)))

    def exact_average(dt):
        aug = np.zeros((n + 1, n + 1))
        aug[:n, :n] = dt * L
        aug[:n, n] = v
        return expm(aug)[:n, n]  # = phi_1(dt L) v

    errs = []
    for dt in (0.4 / rho, 0.2 / rho):
        avg, _ = oracle.stp(q, params, h=h, dt=dt)
        errs.append(np.abs(avg[0].reshape(-1) - exact_average(dt)).max() / np.abs(v).max())
    assert errs[1] > 1e-13  # above rounding, so the ratio measures truncation
    ratio = errs[0] / errs[1]
    assert 0.6 * 2 ** (N + 1) < ratio < 1.4 * 2 ** (N + 1), (errs, ratio)


@pytest.mark.parametrize("K", [1, 2, 4])
def test_term_count_parameter(K):
    N = 3
    rng = np.random.default_rng(K)
    params = random_params(1, N, rng)
    q = rng.uniform(-1, 1, (1, N, N, N, 9))
    avg, _ = oracle.stp(q, params, h=0.3, dt=0.01, K=K)
    L = ref.dense_operator(N, 0.3, params[0])
    avg_x = ref.dense_time_average(L, q[0].reshape(-1), 0.01, K)
    assert ref.rel_err(avg[0].reshape(-1), avg_x) <= 1e-13


# --- Gauss-Lobatto nodes (the paper's other node family, Sec. II-A) ---------

def closed_form_gll(N):
    """Gauss-Lobatto points on [-1,1] with closed forms (N <= 5)."""
    t = {2: [-1.0, 1.0], 3: [-1.0, 0.0, 1.0],
         4: [-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0],
         5: [-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0]}[N]
    return (np.array(t) + 1) / 2


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_gll_nodes_closed_form(N):
    xi, _ = oracle.gll_nodes(N)
    assert np.abs(xi - closed_form_gll(N)).max() <= 2e-16


@pytest.mark.parametrize("N", list(range(2, 13)))
def test_gll_nodes_weights_and_quadrature(N):
    xi, w = oracle.gll_nodes(N)
    xr, wr = ref.gll_points(N)
    assert np.abs(xi - xr).max() <= 1e-14 and np.abs(w - wr).max() <= 1e-14
    assert xi[0] == 0.0 and xi[-1] == 1.0
    for p in range(2 * N - 2):  # exact to degree 2N-3 on [0,1]
        assert abs(np.dot(w, xi ** p) - 1.0 / (p + 1)) <= 1e-14


@pytest.mark.parametrize("N", list(range(2, 13)))
def test_gll_tables_exact_on_polynomials(N):
    xi, D, p0, p1 = oracle.tables(N, "gll")
    assert np.abs(D - ref.lagrange_D_numpy(N, "gll")).max() <= 1e-11 * max(1.0, np.abs(D).max())
    e0 = np.zeros(N); e0[0] = 1.0
    eN = np.zeros(N); eN[-1] = 1.0
    assert np.array_equal(p0, e0) and np.array_equal(p1, eN)
    for p in range(N):
        assert np.abs(D @ xi ** p - (p * xi ** (p - 1) if p else 0 * xi)).max() <= 1e-11 * N ** 2


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_gll_polynomial_data_matches_symbolic_series(N):
    h, dt = 0.5, 0.03
    origins = [(0.0, 0.0, 0.0), (0.5, -1.0, 1.5)]
    q, params, avg_x, faces_x = _poly_case(N, 2.0, 3.0, 1.0, h, dt, origins, seed=40 + N,
                                           nodes="gll")
    avg, faces = oracle.stp(q, params, h=h, dt=dt, nodes="gll")
    assert ref.rel_err(avg, avg_x) <= 1e-12
    assert ref.rel_err(faces, faces_x) <= 1e-12
    assert ref.rel_err(avg - q, avg_x - q) <= 1e-10


@pytest.mark.parametrize("N", [2, 3])
def test_gll_brute_force_dense_operator(N):
    rng = np.random.default_rng(70 + N)
    params = random_params(1, N, rng)
    q = rng.uniform(-1, 1, (1, N, N, N, 9))
    h, dt = 0.2, 0.004
    avg, _ = oracle.stp(q, params, h=h, dt=dt, nodes="gll")
    L = ref.dense_operator(N, h, params[0], "gll")
    avg_x = ref.dense_time_average(L, q[0].reshape(-1), dt, N + 1).reshape(N, N, N, 9)
    assert ref.rel_err(avg[0], avg_x) <= 1e-13
    # the two families differ (so the family switch is not a no-op)
    avg_gl, _ = oracle.stp(q, params, h=h, dt=dt)
    assert ref.rel_err(avg_gl[0], avg_x) > 1e-8


# --- point sources ---------------------------------------------------------------

def _source(e, rng, K):
    return {"element": e, "position": tuple(rng.uniform(0, 1, 3)),
            "amplitude": rng.uniform(-1, 1, 9), "derivatives": rng.uniform(-2, 2, K - 1)}


@pytest.mark.parametrize("K", [2, 3, 5])
def test_source_single_node_closed_form(K):
    """N = 1: D = 0, so q^(k+1) = s^(k) = amp f^(k) / h^3 (one node of weight
    1, basis function 1) and avg = q + sum_k dt^(k+1)/(k+2)! amp f^(k) / h^3."""
    rng = np.random.default_rng(K)
    h, dt = 0.4, 0.03
    q = rng.uniform(-1, 1, (3, 1, 1, 1, 9))
    params = random_params(3, 1, rng)
    src = [_source(2, rng, K), _source(2, rng, K), _source(0, rng, K)]
    avg, faces = oracle.stp(q, params, h, dt, K=K, sources=src)
    expect = q.copy()
    for x in src:
        for k in range(K - 1):
            expect[x["element"], 0, 0, 0] += (dt ** (k + 1) / math.factorial(k + 2)
                                              * np.asarray(x["amplitude"]) * x["derivatives"][k] / h ** 3)
    assert np.abs(avg - expect).max() <= 1e-15 * np.abs(expect).max()
    assert np.abs(faces[:, 0, 0, 0] - avg[:, 0, 0, 0]).max() <= 1e-15


def _nodal_projection(N, pos, h, nodes):
    """phi_l(pos) / (w_l h^3) on the element's nodes [z][y][x] (numpy
    Lagrange basis and quadrature weights)."""
    _, w = ref.points(N, nodes)
    px = ref.lagrange_phi_numpy(N, pos[0], nodes)
    py = ref.lagrange_phi_numpy(N, pos[1], nodes)
    pz = ref.lagrange_phi_numpy(N, pos[2], nodes)
    P = pz[:, None, None] * py[None, :, None] * px[None, None, :]
    return P / (w[:, None, None] * w[None, :, None] * w[None, None, :] * h ** 3)


@pytest.mark.parametrize("N,nodes", [(2, "gl"), (3, "gl"), (3, "gll")])
def test_source_brute_force_dense_operator(N, nodes):
    rng = np.random.default_rng(55 + N)
    E, K = 2, N + 1
    params = random_params(E, N, rng)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    h, dt = 0.3, 0.004
    src = [_source(0, rng, K), _source(0, rng, K), _source(1, rng, K)]
    avg, _, terms = oracle.stp(q, params, h, dt, return_terms=True, nodes=nodes, sources=src)
    for e in range(E):
        L = ref.dense_operator(N, h, params[e], nodes)
        S = np.zeros((K - 1, N, N, N, 9))
        for x in src:
            if x["element"] != e:
                continue
            P = _nodal_projection(N, x["position"], h, nodes)
            for k in range(K - 1):
                S[k] += P[..., None] * np.asarray(x["amplitude"]) * x["derivatives"][k]
        p = q[e].reshape(-1)
        expect = p.copy()
        for k in range(K - 1):
            p = L @ p + S[k].reshape(-1)
            expect = expect + dt ** (k + 1) / math.factorial(k + 2) * p
            assert ref.rel_err(terms[e, k + 1].reshape(-1), p) <= 1e-12
        assert ref.rel_err(avg[e].reshape(-1), expect) <= 1e-13


def test_source_superposition_and_linearity():
    N, E = 4, 3
    rng = np.random.default_rng(77)
    params = random_params(E, N, rng)
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    h, dt = 0.25, 0.01
    s1 = [_source(1, rng, N + 1)]
    s2 = [_source(1, rng, N + 1), _source(2, rng, N + 1)]
    a12, f12 = oracle.stp(q, params, h, dt, sources=s1 + s2)
    a1, f1 = oracle.stp(q, params, h, dt, sources=s1)
    a2, f2 = oracle.stp(np.zeros_like(q), params, h, dt, sources=s2)
    assert ref.rel_err(a12, a1 + a2) <= 1e-14 and ref.rel_err(f12, f1 + f2) <= 1e-14
    a0, _ = oracle.stp(q, params, h, dt)
    assert np.array_equal(a1[0], a0[0]) and np.array_equal(a1[2], a0[2])  # other elements untouched
    assert ref.rel_err(a1[1], a0[1]) > 1e-6


# --- invariants ----------------------------------------------------------------

def test_linearity_and_element_independence():
    N, E = 4, 5
    rng = np.random.default_rng(99)
    params = random_params(E, N, rng)
    q1 = rng.uniform(-1, 1, (E, N, N, N, 9))
    q2 = rng.uniform(-1, 1, (E, N, N, N, 9))
    a1, f1 = oracle.stp(q1, params, 0.125, 0.003)
    a2, f2 = oracle.stp(q2, params, 0.125, 0.003)
    a3, f3 = oracle.stp(2.0 * q1 - 0.5 * q2, params, 0.125, 0.003)
    assert ref.rel_err(a3, 2.0 * a1 - 0.5 * a2) <= 1e-14
    assert ref.rel_err(f3, 2.0 * f1 - 0.5 * f2) <= 1e-14
    perm = rng.permutation(E)
    ap, fp = oracle.stp(q1[perm], params[perm], 0.125, 0.003)
    assert np.array_equal(ap, a1[perm]) and np.array_equal(fp, f1[perm])


# v'_{pi(i)} = v_i, sigma'_{pi(i) pi(j)} = sigma_ij for the cyclic axis map
# pi = (x->y, y->z, z->x)
_PI = (1, 2, 0)


def _rotate_state(a):
    out = np.empty_like(a)
    for i in range(3):
        out[..., _PI[i]] = a[..., i]
        for j in range(3):
            out[..., ref.SIG[(_PI[i], _PI[j])]] = a[..., ref.SIG[(i, j)]]
    return out


def test_axis_rotation_symmetry():
    N, E = 5, 2
    rng = np.random.default_rng(5)
    params = random_params(E, N, rng)
    params[..., 2] = rng.uniform(1.0, 2.0, (E, N, N, N))
    q = rng.uniform(-1, 1, (E, N, N, N, 9))
    avg, faces = oracle.stp(q, params, 0.1, 0.002)
    # new array B[z',y',x'] = A[z=x', y=z', x=y']  (old x axis becomes new y axis)
    tq = _rotate_state(q.transpose(0, 2, 3, 1, 4))
    tp = params.transpose(0, 2, 3, 1, 4)
    avg_r, faces_r = oracle.stp(tq, tp, 0.1, 0.002)
    assert ref.rel_err(avg_r, _rotate_state(avg.transpose(0, 2, 3, 1, 4))) <= 1e-13
    # old x faces ([z][y]) become new y faces ([z'][x'] = [y][z]); old y faces
    # ([z][x]) become new z faces ([y'][x'] = [x][z]); old z faces ([y][x])
    # become new x faces ([z'][y'] = [y][x])
    for d in range(3):
        for side in range(2):
            old = faces[:, 2 * d + side]
            if d in (0, 1):
                old = old.transpose(0, 2, 1, 3)
            new = faces_r[:, 2 * _PI[d] + side]
            assert ref.rel_err(new, _rotate_state(old)) <= 1e-13


def test_rejects_bad_arguments():
    q = np.zeros((1, 3, 3, 3, 9))
    with pytest.raises(ValueError):
        oracle.stp(q, np.zeros((1, 3, 3, 3, 2)), 0.1, 0.01)
    with pytest.raises(RuntimeError):
        oracle.stp(q, np.ones((1, 3, 3, 3, 3)), -0.1, 0.01)
