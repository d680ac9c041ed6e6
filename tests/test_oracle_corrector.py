"""Pins of the corrector oracle (CPU only): what the method and the
mathematics fix, independently of the oracle's own loops.

* a constant state is steady on any material (no derivative, no jump);
* on uniform material, data that is one global polynomial of total degree
  below N leaves no jump at the faces of an interior element, the predictor is
  exact there, and the corrected state is the exact solution at t + dt (a
  symbolic Taylor series of the continuous operator);
* with the Rusanov flux on uniform material the semi-discrete energy obeys
  dE/dt = -(s/2) * sum over faces of the face quadrature of [[q]]^T H [[q]]
  (H the energy matrix of elasticity) exactly: the central part of the flux
  cancels against the volume term by summation by parts;
* with one node per element (N = 1) the scheme is the first-order Rusanov
  finite-volume scheme, written here in its textbook form;
* a dense brute force (global operator assembled with Kronecker products
  from numpy's quadrature and Lagrange tables) on 2-element grids with
  per-node material agrees with the oracle;
* mirroring the grid along x (with the matching sign changes of v1, s12 and
  s13) mirrors the result.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from tests import _elastic as ref

SIGN_X = np.array([-1, 1, 1, 1, 1, 1, -1, -1, 1], dtype=float)  # x -> -x


def periodic_field(N, grid, h, seed, amplitude=1.0):
    """A random state and per-node material on the grid (no smoothness)."""
    rng = np.random.default_rng(seed)
    E = int(np.prod(grid))
    q = rng.uniform(-1, 1, (E, N, N, N, 9)) * amplitude
    params = np.empty((E, N, N, N, 3))
    params[..., 0] = rng.uniform(2, 3, (E, N, N, N))
    params[..., 1] = rng.uniform(4, 6, (E, N, N, N))
    params[..., 2] = params[..., 1] / math.sqrt(3) * rng.uniform(0.9, 1.0, (E, N, N, N))
    return q, params


def uniform_params(E, N, rho=2.4, cp=5.1, cs=2.2):
    p = np.empty((E, N, N, N, 3))
    p[...] = (rho, cp, cs)
    return p


def one_step(q, params, grid, h, dt, nodes="gl"):
    avg, faces = oracle.stp(q, params, h, dt, nodes=nodes)
    return oracle.correct(q, params, avg, faces, grid, h, dt, nodes=nodes)


# --------------------------------------------------------------------------
# constant state
@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_constant_state_is_steady(N):
    grid = (3, 2, 2)
    _, params = periodic_field(N, grid, 0.25, seed=N)
    q = np.empty((12, N, N, N, 9))
    q[...] = np.arange(1.0, 10.0)
    out = one_step(q, params, grid, 0.25, 0.01)
    # rounding only: the rows of D sum to zero up to a few ulp of max|D|, then
    # scaled by dt/h and the material (|B| ~ 70); a structural mistake is O(1)
    assert ref.rel_err(out, q) <= 1e-11


# --------------------------------------------------------------------------
# global polynomial, interior element, exact solution at t + dt
def _exact_poly_step(N, rho, cp, cs, h, dt, seed):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    rng = np.random.default_rng(seed)
    lam, mu = ref.lame(rho, cp, cs)
    lam_r, mu_r, rho_r = sp.Rational(lam), sp.Rational(mu), sp.Rational(rho)
    monos = [(a, b, c) for a in range(N) for b in range(N) for c in range(N) if a + b + c <= N - 1]
    q0 = [sum(int(cf) * x ** a * y ** b * z ** c
              for cf, (a, b, c) in zip(rng.integers(-3, 4, len(monos)), monos)) for _ in range(9)]
    # q(t) = sum_k t^k/k! A^k q0 for the continuous operator (terminates)
    terms = [q0]
    while True:
        f = terms[-1]
        grad = [[sp.diff(f[s], v) for s in range(9)] for v in (x, y, z)]
        nxt = [sp.expand(e) for e in ref.elastic_rate(grad, rho_r, lam_r, mu_r)]
        if all(e == 0 for e in nxt):
            break
        terms.append(nxt)
    dt_r = sp.Rational(dt)
    q1 = [sum(dt_r ** k / sp.factorial(k) * terms[k][s] for k in range(len(terms))) for s in range(9)]
    f0 = [sp.lambdify((x, y, z), e, "numpy") for e in q0]
    f1 = [sp.lambdify((x, y, z), e, "numpy") for e in q1]
    xi, _ = ref.points(N)
    grid = (3, 3, 3)
    q = np.zeros((27, N, N, N, 9))
    exact = np.zeros_like(q)
    for ez in range(3):
        for ey in range(3):
            for ex in range(3):
                e = (ez * 3 + ey) * 3 + ex
                Z, Y, X = np.meshgrid((ez + xi) * h, (ey + xi) * h, (ex + xi) * h, indexing="ij")
                for s in range(9):
                    q[e, ..., s] = np.broadcast_to(f0[s](X, Y, Z), (N, N, N))
                    exact[e, ..., s] = np.broadcast_to(f1[s](X, Y, Z), (N, N, N))
    return q, exact, grid


@pytest.mark.parametrize("N", [2, 3, 4])
def test_polynomial_interior_element_is_exact(N):
    rho, cp, cs, h, dt = 2.0, 3.0, 1.0, 0.5, 0.03  # lambda != mu
    q, exact, grid = _exact_poly_step(N, rho, cp, cs, h, dt, seed=40 + N)
    out = one_step(q, uniform_params(27, N, rho, cp, cs), grid, h, dt)
    centre = 13  # (1,1,1): every neighbour carries the same polynomial
    assert ref.rel_err(out[centre], exact[centre]) <= 1e-13
    # and the corrector did change it (the data is not steady)
    assert ref.rel_err(q[centre], exact[centre]) > 1e-4


# --------------------------------------------------------------------------
# energy identity
def energy_matrix(rho, cp, cs):
    """H with E = 1/2 q^T H q: rho for velocities, the compliance for stresses
    (normal block the inverse of the stiffness, 1/mu for each shear stress)."""
    lam, mu = ref.lame(rho, cp, cs)
    H = np.zeros((9, 9))
    H[:3, :3] = rho * np.eye(3)
    C = lam * np.ones((3, 3)) + 2 * mu * np.eye(3)
    H[3:6, 3:6] = np.linalg.inv(C)
    H[6:, 6:] = np.eye(3) / mu
    return H


def face_values(q, N, nodes="gl"):
    """[E][6][N][N][9] with numpy's Lagrange values at 0 and 1."""
    p = [ref.lagrange_phi_numpy(N, 0.0, nodes), ref.lagrange_phi_numpy(N, 1.0, nodes)]
    out = np.empty((q.shape[0], 6, N, N, 9))
    for side in range(2):
        out[:, 0 + side] = np.einsum("i,ezyis->ezys", p[side], q)
        out[:, 2 + side] = np.einsum("i,eziys->ezys", p[side], q)
        out[:, 4 + side] = np.einsum("i,eiyxs->eyxs", p[side], q)
    return out


def neighbours(grid, e, d):
    gx, gy, gz = grid
    ex, ey, ez = e % gx, (e // gx) % gy, e // (gx * gy)
    c = [ex, ey, ez]
    c[d] = (c[d] + 1) % grid[d]
    return (c[2] * gy + c[1]) * gx + c[0]


@pytest.mark.parametrize("N,grid", [(2, (3, 2, 2)), (3, (2, 3, 2)), (4, (2, 2, 3)), (5, (1, 2, 2))])
def test_energy_identity_on_uniform_material(N, grid):
    rho, cp, cs, h = 2.4, 5.1, 2.2, 0.3
    E = int(np.prod(grid))
    q, _ = periodic_field(N, grid, h, seed=70 + N)
    params = uniform_params(E, N, rho, cp, cs)
    H = energy_matrix(rho, cp, cs)
    for d in range(3):  # the identity needs H B_d symmetric
        A = ref.coefficient_matrices(rho, cp, cs)[d]
        assert np.allclose(H @ A, (H @ A).T, atol=1e-12)
    # semi-discrete rate: the corrector with avg = q, faces of q, dt = 1
    _, w = ref.gl_points(N)
    fq = face_values(q, N)
    rate = oracle.correct(q, params, q, fq, grid, h, 1.0) - q
    W = np.einsum("i,j,k->ijk", w, w, w) * h ** 3
    dEdt = float(np.einsum("zyx,ezyxs,st,ezyxt->", W, q, H, rate))
    # dissipation: every face once (the side-1 face of each element)
    Wf = np.outer(w, w) * h * h
    diss = 0.0
    for e in range(E):
        for d in range(3):
            en = neighbours(grid, e, d)
            jump = fq[en, 2 * d] - fq[e, 2 * d + 1]
            diss += float(np.einsum("ab,abs,st,abt->", Wf, jump, H, jump))
    expected = -0.5 * cp * diss
    assert expected < 0
    assert abs(dEdt - expected) <= 1e-12 * abs(expected) * 10


# --------------------------------------------------------------------------
# N = 1: the first-order Rusanov finite-volume scheme
@pytest.mark.parametrize("d", [0, 1, 2])
def test_one_node_is_first_order_rusanov(d):
    rho, cp, cs, h, dt = 2.4, 5.1, 2.2, 0.2, 0.013
    n = 7
    grid = [1, 1, 1]
    grid[d] = n
    rng = np.random.default_rng(90 + d)
    q = rng.uniform(-1, 1, (n, 1, 1, 1, 9))
    out = one_step(q, uniform_params(n, 1, rho, cp, cs), tuple(grid), h, dt)
    A = ref.coefficient_matrices(rho, cp, cs)[d]  # q_t = A q_x along d
    u = q.reshape(n, 9)
    up, um = np.roll(u, -1, axis=0), np.roll(u, 1, axis=0)
    # classic local Lax-Friedrichs form of q_t = A q_x with speed bound cp
    fv = u + dt / (2 * h) * (up - um) @ A.T + cp * dt / (2 * h) * (up - 2 * u + um)
    assert ref.rel_err(out.reshape(n, 9), fv) <= 1e-14


def test_one_node_heterogeneous_is_path_conservative_rusanov():
    """Element-wise material: the fluctuation form of the Rusanov scheme with
    the mean matrix and the larger P speed on each face."""
    h, dt, n = 0.2, 0.011, 6
    rng = np.random.default_rng(95)
    q = rng.uniform(-1, 1, (n, 1, 1, 1, 9))
    mat = np.stack([rng.uniform(2, 3, n), rng.uniform(4, 6, n), rng.uniform(2, 3, n)], axis=1)
    params = mat.reshape(n, 1, 1, 1, 3)
    out = one_step(q, params, (n, 1, 1), h, dt).reshape(n, 9)
    u = q.reshape(n, 9)
    B = [-ref.coefficient_matrices(*mat[i])[0] for i in range(n)]  # q_t + B q_x = 0
    fv = u.copy()
    for i in range(n):
        r, l = (i + 1) % n, (i - 1) % n
        Br, sr = 0.5 * (B[i] + B[r]), max(mat[i, 1], mat[r, 1])
        Bl, sl = 0.5 * (B[l] + B[i]), max(mat[l, 1], mat[i, 1])
        dminus = 0.5 * (Br - sr * np.eye(9)) @ (u[r] - u[i])  # into cell i from its right
        dplus = 0.5 * (Bl + sl * np.eye(9)) @ (u[i] - u[l])  # into cell i from its left
        fv[i] = u[i] - dt / h * (dminus + dplus)
    assert ref.rel_err(out, fv) <= 1e-14


# --------------------------------------------------------------------------
# dense brute force
def _face_operator(N, d, side, nodes="gl"):
    """Maps an element's flattened [z][y][x] node values to its d-face values
    [a][b] (the two other dimensions, slower first)."""
    phi = ref.lagrange_phi_numpy(N, float(side), nodes).reshape(1, N)
    I = np.eye(N)
    if d == 0:
        return np.kron(np.kron(I, I), phi)  # [z][y]
    if d == 1:
        return np.kron(np.kron(I, phi), I)  # [z][x]
    return np.kron(np.kron(phi, I), I)  # [y][x]


def dense_corrector(q, params, grid, h, dt, nodes="gl"):
    N = q.shape[1]
    E = q.shape[0]
    n3, n2 = N ** 3, N ** 2
    _, w = ref.points(N, nodes)
    L = np.zeros((9 * n3 * E, 9 * n3 * E))
    for e in range(E):
        sl = slice(9 * n3 * e, 9 * n3 * (e + 1))
        L[sl, sl] = ref.dense_operator(N, h, params[e], nodes)
    # predictor: volume operator only, K = N + 1 terms
    avg = ref.dense_time_average(L, q.reshape(-1), dt, N + 1)
    R = L.copy()
    gx, gy, gz = grid
    I9 = np.eye(9)
    for e in range(E):
        ex, ey, ez = e % gx, (e // gx) % gy, e // (gx * gy)
        for d in range(3):
            for side in range(2):
                c = [ex, ey, ez]
                c[d] = (c[d] + (1 if side else -1)) % grid[d]
                en = (c[2] * gy + c[1]) * gx + c[0]
                Pm = _face_operator(N, d, side, nodes)
                Pp = _face_operator(N, d, 1 - side, nodes)
                mm = Pm @ params[e].reshape(n3, 3)
                mp = Pp @ params[en].reshape(n3, 3)
                # lift: node n gets phi_i(side) / (w_i h) F[a,b], i = n's index along d
                idx = np.indices((N, N, N)).reshape(3, -1)  # z, y, x per flat node
                along = idx[2 - d]
                lift = np.diag(1.0 / (w[along] * h)) @ Pm.T
                for ab in range(n2):
                    Bm = -ref.coefficient_matrices(*mm[ab])[d]
                    Bp = -ref.coefficient_matrices(*mp[ab])[d]
                    Bn = (1 if side else -1) * 0.5 * (Bm + Bp)
                    s = max(abs(mm[ab, 1]), abs(mp[ab, 1]))
                    F = 0.5 * (Bn - s * I9)
                    col = lift[:, ab]
                    rows_e = slice(9 * n3 * e, 9 * n3 * (e + 1))
                    # F acts on (q+ - q-) at face point ab
                    sel_p = np.kron(Pp[ab:ab + 1], I9)  # (9, 9 n3) of the neighbour
                    sel_m = np.kron(Pm[ab:ab + 1], I9)
                    blk = np.kron(col.reshape(-1, 1), I9) @ F  # (9 n3, 9)
                    R[rows_e, 9 * n3 * en:9 * n3 * (en + 1)] -= blk @ sel_p
                    R[rows_e, rows_e] += blk @ sel_m
    return (q.reshape(-1) + dt * (R @ avg)).reshape(q.shape)


@pytest.mark.parametrize("N,grid", [(2, (2, 1, 1)), (3, (2, 1, 1)), (2, (1, 2, 1)),
                                    (3, (1, 1, 2)), (2, (2, 2, 1))])
def test_dense_brute_force(N, grid):
    h, dt = 0.25, 0.004
    q, params = periodic_field(N, grid, h, seed=110 + N + 3 * sum(grid))
    out = one_step(q, params, grid, h, dt)
    dense = dense_corrector(q, params, grid, h, dt)
    assert ref.rel_err(out, dense) <= 1e-13
    assert ref.rel_err(out - q, dense - q) <= 1e-12


# --------------------------------------------------------------------------
# mirror symmetry
def mirror_x(a, grid, vec_signs=None):
    gx, gy, gz = grid
    E = a.shape[0]
    b = a.reshape((gz, gy, gx) + a.shape[1:])[:, :, ::-1, :, :, ::-1]
    b = b.reshape((E,) + a.shape[1:])
    if vec_signs is not None:
        b = b * vec_signs
    return np.ascontiguousarray(b)


@pytest.mark.parametrize("N", [2, 4, 5])
def test_mirror_symmetry(N):
    grid, h, dt = (3, 2, 2), 0.25, 0.004
    q, params = periodic_field(N, grid, h, seed=130 + N)
    out = one_step(q, params, grid, h, dt)
    out_m = one_step(mirror_x(q, grid, SIGN_X), mirror_x(params, grid), grid, h, dt)
    assert ref.rel_err(out_m, mirror_x(out, grid, SIGN_X)) <= 1e-13
    assert ref.rel_err(out_m - mirror_x(q, grid, SIGN_X), mirror_x(out - q, grid, SIGN_X)) <= 1e-12


def test_face_params_is_the_face_projection():
    N, E = 5, 3
    rng = np.random.default_rng(7)
    params = rng.uniform(1, 3, (E, N, N, N, 3))
    fp = oracle.face_params(params)
    p = [ref.lagrange_phi_numpy(N, 0.0), ref.lagrange_phi_numpy(N, 1.0)]
    for side in range(2):
        assert ref.rel_err(fp[:, side], np.einsum("i,ezyic->ezyc", p[side], params)) <= 1e-14
        assert ref.rel_err(fp[:, 2 + side], np.einsum("i,ezixc->ezxc", p[side], params)) <= 1e-14
        assert ref.rel_err(fp[:, 4 + side], np.einsum("i,eiyxc->eyxc", p[side], params)) <= 1e-14
