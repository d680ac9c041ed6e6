"""Independent restatements used to pin the oracle (test helpers only).

Everything here is written from textbook definitions, not from the oracle:

* ``elastic_rate``: linear elasticity in tensor form (velocity-stress),
  rho v_t = div(sigma), sigma_t = lambda tr(grad v) I + mu (grad v + grad v^T),
  mapped to the quantity order (v1,v2,v3,s11,s22,s33,s12,s13,s23). It works on
  numbers or on sympy expressions.
* ``lagrange_D_numpy``: derivative matrix from a Vandermonde solve in the
  Legendre basis on numpy's Gauss-Legendre points, or on Gauss-Lobatto points
  from numpy's Legendre-derivative roots (library routines only).
* ``dense_operator``: the whole per-element spatial operator as a dense matrix
  assembled with Kronecker products.
"""
from __future__ import annotations

import math

import numpy as np

# position of the symmetric stress component sigma_ij in the state vector
SIG = {(0, 0): 3, (1, 1): 4, (2, 2): 5, (0, 1): 6, (1, 0): 6, (0, 2): 7,
       (2, 0): 7, (1, 2): 8, (2, 1): 8}


def lame(rho, cp, cs):
    """Lame parameters from density and P/S wave speeds."""
    return rho * (cp * cp - 2 * cs * cs), rho * cs * cs


def elastic_rate(grad, rho, lam, mu):
    """Time derivative of the state from its spatial gradient.

    grad[d][s] = d q_s / d x_d (3 x 9 nested sequence). Returns a list of 9.
    """
    out = [0] * 9
    gradv = [[grad[j][i] for j in range(3)] for i in range(3)]  # dv_i/dx_j
    for i in range(3):
        out[i] = sum(grad[j][SIG[(i, j)]] for j in range(3)) / rho
    div = gradv[0][0] + gradv[1][1] + gradv[2][2]
    for i in range(3):
        for j in range(i, 3):
            val = mu * (gradv[i][j] + gradv[j][i])
            if i == j:
                val = val + lam * div
            out[SIG[(i, j)]] = val
    return out


def coefficient_matrices(rho, cp, cs):
    """A_d (9x9) with q_t = sum_d A_d dq/dx_d, read off elastic_rate."""
    lam, mu = lame(rho, cp, cs)
    A = np.zeros((3, 9, 9))
    for d in range(3):
        for s in range(9):
            g = [[0.0] * 9 for _ in range(3)]
            g[d][s] = 1.0
            A[d][:, s] = elastic_rate(g, rho, lam, mu)
    return A


def gl_points(N):
    t, w = np.polynomial.legendre.leggauss(N)
    return (t + 1) / 2, w / 2


def gll_points(N):
    """Gauss-Lobatto points and weights on [0,1]: the end points and the roots
    of P_{N-1}' (numpy polynomial routines), weights 1/(N(N-1) P_{N-1}(t)^2)."""
    P = np.polynomial.legendre.Legendre.basis(N - 1)
    t = np.concatenate([[-1.0], np.sort(P.deriv().roots().real), [1.0]]) if N > 2 else np.array([-1.0, 1.0])
    w = 1.0 / (N * (N - 1) * P(t) ** 2)
    return (t + 1) / 2, w


def points(N, nodes="gl"):
    return gl_points(N) if nodes == "gl" else gll_points(N)


def lagrange_D_numpy(N, nodes="gl"):
    """D[i,j] = phi_j'(xi_i) via the Legendre Vandermonde matrix V[i,k]=P_k(t_i)."""
    xi, _ = points(N, nodes)
    t = 2 * xi - 1
    V = np.polynomial.legendre.legvander(t, N - 1)
    # phi_j = sum_k C[k,j] P_k with V C = I
    C = np.linalg.solve(V, np.eye(N))
    dV = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1
        dV[:, k] = np.polynomial.legendre.legval(t, np.polynomial.legendre.legder(e)) * 2
    return dV @ C


def lagrange_phi_numpy(N, a, nodes="gl"):
    xi, _ = points(N, nodes)
    t = 2 * xi - 1
    V = np.polynomial.legendre.legvander(t, N - 1)
    C = np.linalg.solve(V, np.eye(N))
    va = np.polynomial.legendre.legvander(np.array([2 * a - 1.0]), N - 1)[0]
    return va @ C


def dense_operator(N, h, params, nodes="gl"):
    """Dense L (9N^3 x 9N^3) of one element, state flattened as [z][y][x][s].

    params: [N][N][N][3] per-node (rho, cp, cs).
    """
    D = lagrange_D_numpy(N, nodes) / h
    I = np.eye(N)
    Dd = [np.kron(np.kron(I, I), D),  # x: fastest node index
          np.kron(np.kron(I, D), I),  # y
          np.kron(np.kron(D, I), I)]  # z
    n3 = N ** 3
    L = np.zeros((9 * n3, 9 * n3))
    flat = params.reshape(n3, 3)
    for d in range(3):
        big = np.kron(Dd[d], np.eye(9))  # derivative of every quantity
        blk = np.zeros((9 * n3, 9 * n3))
        for n in range(n3):
            blk[9 * n:9 * n + 9, 9 * n:9 * n + 9] = coefficient_matrices(*flat[n])[d]
        L += blk @ big
    return L


def dense_time_average(L, q, dt, K):
    """sum_{k<K} dt^k/(k+1)! L^k q by repeated dense matrix-vector products."""
    p = q.copy()
    avg = q.copy()
    for k in range(1, K):
        p = L @ p
        avg = avg + dt ** k / math.factorial(k + 1) * p
    return avg


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.abs(b).max()
    return float(np.abs(a - b).max() / (scale if scale > 0 else 1.0))


def dense_operator_curvilinear(N, params, metric, nodes="gl"):
    """Dense L of one curvilinear element, physical derivative first:
    L = sum_j blockdiag_n(A_j(n)) (Dphys_j kron I_9) with
    Dphys_j = sum_d diag_n(G_n[d][j]) D_d, D_d the reference derivative along
    d (no 1/h: the metric G_n = dxi/dx at node n carries the scale).

    params: [N][N][N][3]; metric: [N][N][N][3][3] (G[d][j] = dxi_d/dx_j).
    """
    D = lagrange_D_numpy(N, nodes)
    I = np.eye(N)
    Dd = [np.kron(np.kron(I, I), D), np.kron(np.kron(I, D), I), np.kron(np.kron(D, I), I)]
    n3 = N ** 3
    G = metric.reshape(n3, 3, 3)
    flat = params.reshape(n3, 3)
    A = [coefficient_matrices(*flat[n]) for n in range(n3)]
    L = np.zeros((9 * n3, 9 * n3))
    for j in range(3):
        Dphys = sum(np.diag(G[:, d, j]) @ Dd[d] for d in range(3))
        blk = np.zeros((9 * n3, 9 * n3))
        for n in range(n3):
            blk[9 * n:9 * n + 9, 9 * n:9 * n + 9] = A[n][j]
        L += blk @ np.kron(Dphys, np.eye(9))
    return L
